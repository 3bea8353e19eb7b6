"""Sensor placement on the GPU (Sec. 6): the position gradient of the
physical forward model A(x) = R_u(x)^T (the unweighted transpose) against
the FP64 oracle, and a few gradient steps of the placement loop raising the
correlation coefficient (Appendix B) of R(x) A(x) f with f."""
import numpy as np
import pytest

import oracle
from oracle import Problem
from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_GRAD = 1e-4


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


def test_model_position_gradient_matches_oracle(nd):
    """d/dx <v, A(x) f> = d/dx <R_u(x) v, f>: the model's backward for the
    positions is nedner_grad_positions with (g, dL/dp0) = (v, f)."""
    case = inputs.small_case(16, 16, 32, 60, 64, seed=71, layout="disc")
    rng = np.random.default_rng(72)
    v = rng.standard_normal((60, case["Nt"]))
    f = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    plan = nd.plan_from_config(case, apply_weights=False)
    xy = torch.as_tensor(case["sensor_xy"], dtype=torch.float64).requires_grad_(True)
    g = nd.model(plan, torch.as_tensor(f, dtype=torch.float32, device="cuda"), xy)
    (g * torch.as_tensor(v, dtype=torch.float32, device="cuda")).sum().backward()
    pr = Problem(sensor_xy=case["sensor_xy"], h=case["h"], Nt=case["Nt"], dt=case["dt"], c=case["c"],
                 nx=case["nx"], ny=case["ny"], nz=case["nz"], dx=case["dx"], dy=case["dy"], dz=case["dz"],
                 apply_weights=False)
    want = oracle.grad_positions(pr, v, f)
    check(xy.grad.numpy(), want, TOL_GRAD)
    plan.close()


def test_model_moves_the_plan(nd):
    """Positions given to model() move the plan (nedner_set_positions); the
    result equals a plan built at those positions."""
    case = inputs.small_case(16, 16, 32, 40, 64, seed=73, layout="scatter")
    rng = np.random.default_rng(74)
    f = torch.as_tensor(rng.standard_normal((32, 16, 16)), dtype=torch.float32, device="cuda")
    plan = nd.plan_from_config(case, apply_weights=False)
    xy2 = case["sensor_xy"] * 0.9
    a = nd.model(plan, f, torch.as_tensor(xy2))
    other = nd.Plan(xy2, case["Nt"], case["dt"], case["c"],
                    (case["nx"], case["ny"], case["nz"], case["dx"], case["dy"], case["dz"]), apply_weights=False)
    b = other.adjoint(f)
    assert torch.equal(a, b)
    plan.close()
    other.close()


def test_placement_steps_raise_the_correlation(nd):
    from paper_1510_01078_gb300 import placement as P
    nx, ny, nz, Nt, dt, c = 32, 32, 64, 128, 20e-9, 1500.0
    X = 6.4e-3
    dx = X / nx
    dz = c * Nt * dt / nz
    g3 = (nx, ny, nz, dx, dx, dz)
    xy, h = P.equi_steradian(128, 0.9 * X, 1.2e-3)
    rng = np.random.default_rng(75)
    balls = inputs.random_balls(4, rng, (0.1e-3, 0.25e-3), 0.8e-3, (0.8e-3, 1.6e-3))
    truth = inputs.voxelise(balls, nx, ny, nz, dx, dx, dz)
    mask = P.upper_half_mask(nz, ny, nx)
    pw = nd.Plan(xy, Nt, dt, c, g3, sensor_w=h)
    pu = nd.Plan(xy, Nt, dt, c, g3, apply_weights=False)
    f = torch.as_tensor(truth, dtype=torch.float32, device="cuda")
    res = P.optimise_placement(pw, pu, f, xy, steps=8, lr=3e-3, mask=mask)
    rho = res["rho"]
    assert len(rho) == 9 and np.all(np.isfinite(rho)) and all(-1 <= r <= 1 for r in rho)
    assert rho[-1] > rho[0], rho
    assert np.abs(res["xy"] - xy).max() > 0
    assert np.abs(res["xy"]).max() < 0.5 * X
    # the analytic-data quality of each layout is a correlation coefficient
    r_es = P.layout_rho(g3, Nt, dt, c, xy, h, balls, truth, mask)
    xg, hg = P.regular_grid(xy.shape[0], 0.9 * X)
    r_g = P.layout_rho(g3, Nt, dt, c, xg, hg, balls, truth, mask)
    assert -1 <= r_es <= 1 and -1 <= r_g <= 1
    pw.close()
    pu.close()
