"""nedner_ned_stage_static: the NED stage for callers that cannot allocate
device memory when they run it (graph capture, an exhausted or foreign pool
allocator, no-allocation-after-start-up pipelines).  Its intermediate lives in
the library's fixed 16 MiB device buffer instead of the plan's workspace.

The test calls it through the C-ABI twice in a row on different data and
compares each result with nedner_ned_stage (the plan-workspace version) at the
tolerance of the other parity tests, then checks that a geometry whose
intermediate does not fit is refused.  This file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


def test_static_scratch_ned_stage_matches_workspace_version(nd):
    case = inputs.small_case(32, 16, 32, 211, 128, seed=31, layout="disc")
    plan = nd.plan_from_config(case)
    rng = np.random.default_rng(32)
    gs = [torch.as_tensor(rng.standard_normal((plan.M, plan.Nt)), dtype=torch.float32, device="cuda")
          for _ in range(2)]
    want = [plan.ned_stage(g).cpu().numpy() for g in gs]
    outs = [torch.empty((plan.nx // 2 + 1, plan.ny + 1, plan.Nt), dtype=torch.complex64, device="cuda")
            for _ in range(2)]
    for g, out in zip(gs, outs):                      # two calls in a row
        nd.ned_stage_static(plan, g, out=out)
    torch.cuda.synchronize()
    for out, w in zip(outs, want):
        check(out.cpu().numpy(), w, TOL)
    assert rel_l2(want[0], want[1]) > 0.1             # the two inputs really differ
    plan.close()


def test_static_scratch_rejects_oversized_geometry(nd):
    cfg = inputs.make_config(1, with_data=False)      # intermediate 68 MB > 16 MiB
    plan = nd.plan_from_config(cfg)
    g = torch.zeros((plan.M, plan.Nt), dtype=torch.float32, device="cuda")
    with pytest.raises(nd.NednerError) as ei:
        nd.ned_stage_static(plan, g)
    assert ei.value.status == 3
    plan.close()


def test_static_scratch_rejects_bad_output_pointers_before_launch(nd):
    """A Ghat that is null or not 16-byte aligned is refused on the host with
    NEDNER_EINVAL; nothing is launched, so the GPU never sees the pointer."""
    import ctypes
    case = inputs.small_case(16, 16, 16, 40, 32, seed=33)
    plan = nd.plan_from_config(case)
    g = torch.zeros((plan.M, plan.Nt), dtype=torch.float32, device="cuda")
    out = torch.empty((plan.nx // 2 + 1, plan.ny + 1, plan.Nt + 2), dtype=torch.complex64, device="cuda")
    lib = nd.library()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gp = ctypes.c_void_p(g.data_ptr())
    assert lib.nedner_ned_stage_static(plan._handle, gp, ctypes.c_void_p(out.data_ptr() + 4), s) == nd.EINVAL
    assert lib.nedner_ned_stage_static(plan._handle, gp, ctypes.c_void_p(out.data_ptr() + 8), s) == nd.EINVAL
    assert lib.nedner_ned_stage_static(plan._handle, gp, None, s) == nd.EINVAL
    assert lib.nedner_ned_stage_static(plan._handle, ctypes.c_void_p(g.data_ptr() + 4),
                                       ctypes.c_void_p(out.data_ptr()), s) == nd.EINVAL
    torch.cuda.synchronize()
    plan.close()


def test_static_scratch_refuses_tensor_core_plans(nd):
    """Plans built for the tensor-core stage (a) are refused with NEDNER_EINVAL."""
    cfg = inputs.make_config(4, with_data=False)
    cfg = dict(cfg, Nt=128, dt=cfg["dt"] * 16)
    plan = nd.plan_from_config(cfg, ned_mode="tensor_bf16")
    g = torch.zeros((plan.M, plan.Nt), dtype=torch.float32, device="cuda")
    with pytest.raises(nd.NednerError) as ei:
        nd.ned_stage_static(plan, g)
    assert ei.value.status == nd.EINVAL
    plan.close()
