"""The two-dimensional variant (Sec. 7) on the GPU against the 2-D oracle:
forward and adjoint, weighted and unweighted, scattered sensors; and a small
run of the Sec. 7 comparison."""
import numpy as np
import pytest

from oracle.twod import Problem2D, adjoint2d, forward2d
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


def _case(seed, M=40, nx=64, nz=32, Nt=64):
    rng = np.random.default_rng(seed)
    dx, dt, c = 1e-4, 20e-9, 1500.0
    dz = c * Nt * dt / nz
    X = nx * dx
    x = rng.uniform(-0.49 * X, 0.49 * X, size=M)
    h = rng.uniform(0.5, 1.5, size=M) * X / M
    return Problem2D(sensor_x=x, Nt=Nt, dt=dt, c=c, nx=nx, nz=nz, dx=dx, dz=dz, h=h), rng


@pytest.mark.parametrize("weights", [True, False])
def test_forward_2d_matches_oracle(nd, weights):
    pr, rng = _case(101)
    pr.apply_weights = weights
    g = rng.standard_normal((pr.M, pr.Nt))
    plan = nd.Plan2D(pr.sensor_x, pr.Nt, pr.dt, pr.c, (pr.nx, pr.nz, pr.dx, pr.dz), apply_weights=weights,
                     sensor_w=pr.h)
    got = plan.forward(torch.as_tensor(g, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    check(got, forward2d(pr, g), 1e-5)


@pytest.mark.parametrize("weights", [True, False])
def test_adjoint_2d_matches_oracle(nd, weights):
    pr, rng = _case(102)
    pr.apply_weights = weights
    p = rng.standard_normal((pr.nz, pr.nx))
    plan = nd.Plan2D(pr.sensor_x, pr.Nt, pr.dt, pr.c, (pr.nx, pr.nz, pr.dx, pr.dz), apply_weights=weights,
                     sensor_w=pr.h)
    got = plan.adjoint(torch.as_tensor(p, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    check(got, adjoint2d(pr, p), 1e-5)


def test_set_positions_2d(nd):
    pr, rng = _case(103)
    g = rng.standard_normal((pr.M, pr.Nt))
    plan = nd.Plan2D(pr.sensor_x, pr.Nt, pr.dt, pr.c, (pr.nx, pr.nz, pr.dx, pr.dz), sensor_w=pr.h)
    x2 = pr.sensor_x * 0.8
    plan.set_positions(x2)
    got = plan.forward(torch.as_tensor(g, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    pr.sensor_x = x2
    check(got, forward2d(pr, g), 1e-5)


def test_sec7_comparison_small(nd):
    from paper_1510_01078_gb300 import sec7
    res = sec7.run(nx=128, nz=64, dx=100e-6, Nt=128, n_sensors=16, intervals=range(1, 9))
    assert len(res["equispaced"]) == 8
    for r in res["equispaced"] + [res["equi_angular"]]:
        assert -1.0 <= r["rho"] <= 1.0 and np.isfinite(r["sharpness"]) and r["sharpness"] >= 0
