"""Device status flags and the profiled transposed entry points.

Non-finite data: a NaN placed in g on the host (or an infinity in p0 or
dL/dp0) reaches every output value through the transforms; the output kernel
of each entry point sets the non-finite flag, which nedner_device_status reads
back (returning NEDNER_ENAN) and clears.  Nothing here faults or hangs the GPU:
the kernels only compute with the non-finite numbers.
"""
import ctypes

import numpy as np
import pytest

from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


@pytest.fixture(scope="module")
def case():
    return inputs.small_case(16, 16, 32, 61, 64, seed=41, layout="disc")


def _status_call(nd, plan):
    f = ctypes.c_int(0)
    st = nd.library().nedner_device_status(plan._handle, ctypes.byref(f))
    return st, f.value


def test_forward_flags_nonfinite_input(nd, case):
    plan = nd.plan_from_config(case)
    g = torch.as_tensor(case["g"], dtype=torch.float32, device="cuda")
    plan.forward(g)
    assert _status_call(nd, plan) == (nd.OK, 0)
    bad = case["g"].astype(np.float32).copy()
    bad[7, 13] = np.nan
    plan.forward(torch.as_tensor(bad, device="cuda"))
    assert _status_call(nd, plan) == (nd.ENAN, plan.STATUS_NONFINITE)
    assert _status_call(nd, plan) == (nd.OK, 0)          # read back and cleared
    plan.forward(g)                                      # a clean call afterwards stays clean
    assert plan.device_status() == 0
    bad[7, 13] = np.inf
    out = torch.empty((case["nz"], case["ny"], case["nx"]), dtype=torch.float32).pin_memory()
    plan.forward_host(torch.as_tensor(bad).pin_memory(), out=out)
    assert plan.device_status() == plan.STATUS_NONFINITE
    plan.close()


def test_adjoint_and_gradient_flag_nonfinite_input(nd, case):
    plan = nd.plan_from_config(case)
    rng = np.random.default_rng(42)
    p = rng.standard_normal((case["nz"], case["ny"], case["nx"])).astype(np.float32)
    g = torch.as_tensor(case["g"], dtype=torch.float32, device="cuda")
    plan.adjoint(torch.as_tensor(p, device="cuda"))
    plan.grad_positions(g, torch.as_tensor(p, device="cuda"))
    assert plan.device_status() == 0
    p[3, 4, 5] = np.inf
    plan.adjoint(torch.as_tensor(p, device="cuda"))
    assert plan.device_status() == plan.STATUS_NONFINITE
    plan.grad_positions(g, torch.as_tensor(p, device="cuda"))
    assert plan.device_status() == plan.STATUS_NONFINITE
    plan.close()


def test_profiled_transposed_calls_match_plain_calls(nd):
    """The profiled adjoint and gradient give the plain calls' results (to
    FP32 rounding: the order of a few sums may differ between runs), and a
    positive time for every stage it launches (the gather summed over its
    passes: several passes here, under a workspace limit; the transposed x-FFT
    runs only with the block gather, else its time is zero)."""
    case = inputs.small_case(32, 32, 32, 400, 256, seed=43, layout="disc")
    rng = np.random.default_rng(44)
    p = torch.as_tensor(rng.standard_normal((case["nz"], case["ny"], case["nx"])), dtype=torch.float32,
                        device="cuda")
    g = torch.as_tensor(case["g"], dtype=torch.float32, device="cuda")
    for limit in (0, 6 << 20):
        plan = nd.plan_from_config(case, max_workspace_bytes=limit)
        a = plan.adjoint(p)
        b = torch.empty_like(a)
        ms = plan.adjoint_profiled(p, b)
        check(b.cpu().numpy(), a.cpu().numpy(), 1e-6)
        assert all(v > 0 for k, v in ms.items() if k != "ned_xfft_adj") and ms["ned_xfft_adj"] >= 0, ms
        c = plan.grad_positions(g, p)
        d = torch.empty_like(c)
        ms = plan.grad_positions_profiled(g, p, d)
        check(d.cpu().numpy(), c.cpu().numpy(), 1e-6)
        assert all(v > 0 for k, v in ms.items() if k != "ned_xfft_adj") and ms["ned_xfft_adj"] >= 0, ms
        plan.close()


def test_plan_info_reports_passes_and_launches(nd):
    """nedner_plan_info: the split stage's chunks and the gathers' passes
    divide the record, and the launch counts follow from them."""
    case = inputs.small_case(32, 32, 32, 400, 256, seed=45, layout="disc")
    for limit in (0, 6 << 20):
        plan = nd.plan_from_config(case, max_workspace_bytes=limit)
        i = plan.info()
        Nt = case["Nt"]
        assert set(i) == set(plan.PLAN_INFO_FIELDS)
        assert i["split"] == 1 and Nt % i["tq"] == 0 and Nt % i["tp_adj"] == 0
        assert i["launches_forward"] == 3 * (Nt // i["tq"]) + 3
        if i["gsplit"]:
            assert i["tp_g"] >= 64 and Nt % i["tp_g"] == 0
            assert i["launches_adjoint"] == 4 + 3 * (Nt // i["tp_adj"])
            assert i["launches_grad_positions"] == 4 + 2 * (Nt // i["tp_g"]) + 1
        else:
            assert i["launches_adjoint"] == 4 + 2 * (Nt // i["tp_adj"])
            assert i["launches_grad_positions"] == 6
        if limit == 0:
            assert i["tq"] == Nt and i["gsplit"] == 1
        else:
            assert i["tq"] < Nt                              # the forward streams under the limit
        plan.close()
