"""Tensor-product NED on the tensor cores (precision modes BF16 and FP16 GEMM): workload 5
geometry (128 x 128 non-equispaced tensor-grid sensors over 20 mm, Nt 2048,
256 x 256 x 512 voxels).

The GEMM path evaluates the NED sum exactly with BF16 operands split into hi
and lo parts and FP32 accumulation; its error is set by the ~2^-16 relative
precision of the split factors (each real product keeps the hi*hi, lo*hi and
hi*lo terms), so the tolerance here is rel-L2 <= 3e-5, and the measured value
is printed per test.  The FP16 mode keeps 11 significant bits per part (its
dropped lo*lo term is ~2^-22 of a product), so its tolerance is the FP32
path's, 1e-5.
"""
import numpy as np
import pytest

import oracle
from oracle import Problem
from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_BF16 = 3e-5
TOL_FP16 = 1e-5
MODES = [("tensor_bf16", TOL_BF16), ("tensor_fp16", TOL_FP16)]


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


@pytest.mark.parametrize("mode,tol", MODES, ids=[m for m, _ in MODES])
def test_tensor_ned_stage_matches_oracle(nd, c5_sparse, mode, tol):
    cfg, ns, gs, g = c5_sparse
    pr = problem(cfg)
    sub = Problem(**{**pr.__dict__, "Nt": len(ns)})
    jx = np.arange(0, cfg["nx"] // 2 + 1)
    jy = np.arange(-(cfg["ny"] // 2), cfg["ny"] // 2 + 1)
    want = oracle.ned(sub, gs, jx, jy)                              # (129, 257, 4)
    plan = nd.plan_from_config(cfg, ned_mode=mode)
    got = plan.ned_stage(torch.as_tensor(g, dtype=torch.float32, device="cuda")).cpu().numpy()[:, :, ns]
    plan.close()
    check(got, want, tol)


@pytest.mark.parametrize("mode,tol", MODES, ids=[m for m, _ in MODES])
def test_tensor_forward_matches_oracle(nd, c5_sparse, mode, tol):
    cfg, ns, gs, g = c5_sparse
    want = oracle.forward(problem(cfg), gs, ns=ns)
    plan = nd.plan_from_config(cfg, ned_mode=mode)
    got = plan.forward(torch.as_tensor(g, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    check(got, want, tol)


@pytest.mark.parametrize("mode,tol", MODES, ids=[m for m, _ in MODES])
def test_tensor_matches_nufft_on_dense_data(nd, mode, tol):
    cfg = inputs.make_config(4)
    g = torch.as_tensor(cfg["g"], dtype=torch.float32, device="cuda")
    pt = nd.plan_from_config(cfg, ned_mode=mode)
    pn = nd.plan_from_config(cfg)
    a = pt.ned_stage(g).cpu().numpy()
    b = pn.ned_stage(g).cpu().numpy()
    pt.close(); pn.close()
    check(a, b, tol)


@pytest.mark.parametrize("factor", [1e-9, 1e9])
def test_fp16_mode_scales_any_data_magnitude(nd, c5_sparse, factor):
    """The FP16 mode's power-of-two data scale: data a billion times smaller
    or larger than the workload's give the same relative accuracy (without the
    scale they would underflow or overflow FP16)."""
    cfg, ns, gs, g = c5_sparse
    pr = problem(cfg)
    sub = Problem(**{**pr.__dict__, "Nt": len(ns)})
    jx = np.arange(0, cfg["nx"] // 2 + 1)
    jy = np.arange(-(cfg["ny"] // 2), cfg["ny"] // 2 + 1)
    want = oracle.ned(sub, gs * factor, jx, jy)
    plan = nd.plan_from_config(cfg, ned_mode="tensor_fp16")
    got = plan.ned_stage(torch.as_tensor(g * factor, dtype=torch.float32, device="cuda")).cpu().numpy()[:, :, ns]
    plan.close()
    check(got, want, TOL_FP16)


@pytest.mark.parametrize("mode", ["tensor_bf16", "tensor_fp16"])
def test_tensor_mode_rejects_other_layouts(nd, mode):
    case = inputs.small_case(16, 16, 16, 40, 32, seed=7)
    with pytest.raises(nd.NednerError) as ei:
        nd.plan_from_config(case, ned_mode=mode)
    assert ei.value.status == 1


@pytest.mark.parametrize("mode", ["tensor_bf16", "tensor_fp16"])
def test_tensor_kernels_report_no_timeouts(nd, c5_sparse, mode):
    cfg, ns, gs, g = c5_sparse
    plan = nd.plan_from_config(cfg, ned_mode=mode)
    x = torch.as_tensor(g, dtype=torch.float32, device="cuda")
    for _ in range(3):
        plan.forward(x)
    assert plan.device_status() == 0        # no bounded mbarrier wait ran out
    plan.close()


@pytest.mark.parametrize("mode", ["tensor_bf16", "tensor_fp16"])
def test_tensor_kernels_time_out_cleanly_and_recover(nd, c5_sparse, mode):
    """The bounded waits of the tensor-core kernels, made to run out: with a
    pipeline-wait limit of zero polls every pipeline wait gives up at once;
    the kernels flag it, drain their own copies and MMAs (those waits keep the
    long limit), free tensor memory and return.  The device status reports the
    timeout, and the same plan then computes the right answer again."""
    cfg, ns, gs, g = c5_sparse
    cfg = dict(cfg, Nt=512, dt=cfg["dt"] * 4)             # one pass of 512 time samples
    g = g[:, :512].copy()
    keep = ns[ns < 512]
    plan = nd.plan_from_config(cfg, ned_mode=mode)
    x = torch.as_tensor(g, dtype=torch.float32, device="cuda")
    plan.debug_set_wait_limit(0)
    plan.ned_stage(x)
    assert plan.device_status() & plan.STATUS_WAIT_TIMEOUT
    plan.debug_set_wait_limit(1 << 26)
    got = plan.ned_stage(x).cpu().numpy()[:, :, keep]
    assert plan.device_status() == 0
    plan.close()
    pr = problem(cfg)
    sub = Problem(**{**pr.__dict__, "Nt": len(keep)})
    jx = np.arange(0, cfg["nx"] // 2 + 1)
    jy = np.arange(-(cfg["ny"] // 2), cfg["ny"] // 2 + 1)
    want = oracle.ned(sub, gs[:, :len(keep)], jx, jy)
    check(got, want, TOL_BF16)
