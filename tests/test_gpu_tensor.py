"""Tensor-product NED on the tensor cores (ned_mode tensor_bf16): workload 5
geometry (128 x 128 non-equispaced tensor-grid sensors over 20 mm, Nt 2048,
256 x 256 x 512 voxels).

The GEMM path evaluates the NED sum exactly with BF16 operands split into hi
and lo parts and FP32 accumulation; its error is set by the ~2^-16 relative
precision of the split factors (each real product keeps the hi*hi, lo*hi and
hi*lo terms), so the tolerance here is rel-L2 <= 3e-5, and the measured value
is printed per test.
"""
import numpy as np
import pytest

import oracle
from oracle import Problem
from paper_1510_01078_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_BF16 = 3e-5


def rel_l2(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


def problem(case, **kw):
    return Problem(sensor_xy=case["sensor_xy"], h=case["h"], Nt=case["Nt"], dt=case["dt"], c=case["c"],
                   nx=case["nx"], ny=case["ny"], nz=case["nz"], dx=case["dx"], dy=case["dy"], dz=case["dz"], **kw)


@pytest.fixture(scope="module")
def c5_sparse():
    cfg = inputs.make_config(4, with_data=False)
    rng = np.random.default_rng(505)
    ns = np.array([0, 77, 1024, 2047])
    gs = rng.standard_normal((cfg["sensor_xy"].shape[0], len(ns)))
    g = np.zeros((gs.shape[0], cfg["Nt"]))
    g[:, ns] = gs
    return cfg, ns, gs, g


def test_tensor_ned_stage_matches_oracle(nd, c5_sparse):
    cfg, ns, gs, g = c5_sparse
    pr = problem(cfg)
    sub = Problem(**{**pr.__dict__, "Nt": len(ns)})
    jx = np.arange(0, cfg["nx"] // 2 + 1)
    jy = np.arange(-(cfg["ny"] // 2), cfg["ny"] // 2 + 1)
    want = oracle.ned(sub, gs, jx, jy)                              # (129, 257, 4)
    plan = nd.plan_from_config(cfg, ned_mode="tensor_bf16")
    got = plan.ned_stage(torch.as_tensor(g, dtype=torch.float32, device="cuda")).cpu().numpy()[:, :, ns]
    plan.close()
    err = rel_l2(got, want)
    print("tensor_bf16 NED stage rel-L2 vs oracle: %.3e" % err)
    assert err <= TOL_BF16, err


def test_tensor_forward_matches_oracle(nd, c5_sparse):
    cfg, ns, gs, g = c5_sparse
    want = oracle.forward(problem(cfg), gs, ns=ns)
    plan = nd.plan_from_config(cfg, ned_mode="tensor_bf16")
    got = plan.forward(torch.as_tensor(g, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    err = rel_l2(got, want)
    print("tensor_bf16 forward rel-L2 vs oracle: %.3e" % err)
    assert err <= TOL_BF16, err


def test_tensor_matches_nufft_on_dense_data(nd):
    cfg = inputs.make_config(4)
    g = torch.as_tensor(cfg["g"], dtype=torch.float32, device="cuda")
    pt = nd.plan_from_config(cfg, ned_mode="tensor_bf16")
    pn = nd.plan_from_config(cfg)
    a = pt.ned_stage(g).cpu().numpy()
    b = pn.ned_stage(g).cpu().numpy()
    pt.close(); pn.close()
    err = rel_l2(a, b)
    print("tensor_bf16 vs NUFFT NED stage rel-L2 (dense data): %.3e" % err)
    assert err <= TOL_BF16, err


def test_tensor_mode_rejects_other_layouts(nd):
    case = inputs.small_case(16, 16, 16, 40, 32, seed=7)
    with pytest.raises(nd.NednerError) as ei:
        nd.plan_from_config(case, ned_mode="tensor_bf16")
    assert ei.value.status == 1


def test_tensor_kernels_report_no_timeouts(nd, c5_sparse):
    cfg, ns, gs, g = c5_sparse
    plan = nd.plan_from_config(cfg, ned_mode="tensor_bf16")
    x = torch.as_tensor(g, dtype=torch.float32, device="cuda")
    for _ in range(3):
        plan.forward(x)
    assert plan.device_status() == 0        # no bounded mbarrier wait ran out
    plan.close()
