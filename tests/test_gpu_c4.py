"""Differentiation workload (64x64 centre-dense sensors over 20 mm, Nt 1024,
128^3 voxels): least-squares fit of p0 through the forward/adjoint pair,
and sensor-position gradients for the central 32x32 movable sensors checked
against the FP64 oracle's gradient (itself pinned by FP64 central
differences in test_oracle_pins.py)."""
import numpy as np
import pytest

import oracle
from oracle import Problem
from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def test_model_backward_is_unweighted_forward(nd):
    """d<mu, A f>/df = A^T mu = R_unweighted mu (oracle)."""
    case = inputs.small_case(16, 16, 32, 60, 64, seed=41, layout="disc")
    plan = nd.plan_from_config(case, apply_weights=False)
    rng = np.random.default_rng(42)
    mu = rng.standard_normal((len(case["h"]), case["Nt"]))
    f = torch.zeros((case["nz"], case["ny"], case["nx"]), device="cuda", requires_grad=True)
    gpred = nd.model(plan, f)
    (gpred * torch.as_tensor(mu, dtype=torch.float32, device="cuda")).sum().backward()
    want = oracle.forward(problem(case, apply_weights=False), mu)
    check(f.grad.cpu().numpy(), want, 1e-5)
    plan.close()


@pytest.mark.parametrize("method", ["cg", "adam"])
def test_c4_least_squares_fit(nd, method):
    from paper_1510_01078_gb300 import fit
    cfg = inputs.make_config(3)
    plan = nd.plan_from_config(cfg, apply_weights=False)
    g = torch.as_tensor(cfg["g"], dtype=torch.float32, device="cuda")
    out = fit.fit_p0(plan, g, iters=50, method=method, lr=0.01)
    r = out["residual"]
    assert len(r) == 51
    assert r[-1] < 0.6 * r[0], (r[0], r[-1])
    if method == "cg":
        assert all(r[k + 1] <= r[k] * (1 + 1e-4) for k in range(50))      # CGNR: ||r|| non-increasing
    plan.close()


def test_c4_position_gradient_full_size(nd):
    """dL/d(x, y) of the central 32x32 sensors at full workload size, against
    the oracle's gradient of the same loss L = <lambda, R(x) g>."""
    cfg = inputs.make_config(3)
    rng = np.random.default_rng(43)
    lam = rng.standard_normal((cfg["nz"], cfg["ny"], cfg["nx"]))
    mov = cfg["movable"]
    plan = nd.plan_from_config(cfg)
    got = plan.grad_positions(torch.as_tensor(cfg["g"], dtype=torch.float32, device="cuda"),
                              torch.as_tensor(lam, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    want = oracle.grad_positions(problem(cfg), cfg["g"], lam)
    assert mov.sum() == 1024
    check(got[mov], want[mov], 1e-4)


def test_c4_placement_step_lowers_loss(nd):
    """A small gradient step on the movable sensors lowers ||R(x) g - f_true||^2."""
    from paper_1510_01078_gb300 import fit
    cfg = inputs.make_config(3)
    truth = inputs.voxelise(cfg["balls"], cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"])
    plan = nd.plan_from_config(cfg)
    g = torch.as_tensor(cfg["g"], dtype=torch.float32, device="cuda")
    target = torch.as_tensor(truth, dtype=torch.float32, device="cuda")
    xy = torch.as_tensor(cfg["sensor_xy"], dtype=torch.float64)
    mov = torch.as_tensor(cfg["movable"])
    s0 = fit.placement_step(plan, g, target, xy, mov, lr=0.0)
    gnorm = float(s0["grad"].norm())
    assert gnorm > 0
    step = 0.05 * cfg["dx"] / float(s0["grad"].abs().max())
    s1 = fit.placement_step(plan, g, target, xy, mov, lr=step)
    s2 = fit.placement_step(plan, g, target, s1["xy"], mov, lr=0.0)
    assert s2["loss"] < s0["loss"], (s0["loss"], s2["loss"])
    assert torch.equal(s1["xy"][~mov], xy[~mov])
    plan.close()
