"""Parity of the transposed CUDA path (nedner_adjoint) and of the
sensor-position gradient (nedner_grad_positions) with the FP64 oracle, the
transposition identity <R g, p> = <g, R^T p> on the GPU's own outputs, and the
autograd wrapper.

Tolerances: adjoint rel-L2 <= 1e-5 (the same FP32 budget as the forward path);
gradient rel-L2 <= 1e-4: it differentiates the window (the derivative taps
carry ~w/2 times the window's relative error) and is a sum over time of
products that cancel strongly.
"""
import numpy as np
import pytest

import oracle
from oracle import Problem
from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5
TOL_GRAD = 1e-4


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


CASES = [
    dict(nx=16, ny=16, nz=32, M=37, Nt=64, seed=21, layout="scatter"),
    dict(nx=32, ny=16, nz=64, M=301, Nt=128, seed=22, layout="disc"),
    dict(nx=16, ny=32, nz=16, M=700, Nt=32, seed=23, layout="scatter"),
    dict(nx=8, ny=8, nz=8, M=5, Nt=16, seed=24, layout="scatter"),
    dict(nx=64, ny=64, nz=32, M=2000, Nt=64, seed=25, layout="disc"),
]
IDS = ["{nx}x{ny}x{nz}_M{M}_Nt{Nt}_{layout}".format(**c) for c in CASES]


@pytest.mark.parametrize("spec", CASES, ids=IDS)
def test_adjoint_matches_oracle(nd, spec):
    case = inputs.small_case(**spec)
    rng = np.random.default_rng(spec["seed"] + 100)
    p = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    want = oracle.adjoint(problem(case), p)
    plan = nd.plan_from_config(case)
    got = plan.adjoint(torch.as_tensor(p, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    check(got, want, TOL)


@pytest.mark.parametrize("spec", CASES[:3], ids=IDS[:3])
@pytest.mark.parametrize("weights", [True, False])
def test_transposition_identity_on_gpu(nd, spec, weights):
    case = inputs.small_case(**spec)
    rng = np.random.default_rng(spec["seed"] + 200)
    g = torch.as_tensor(rng.standard_normal((len(case["h"]), case["Nt"])), dtype=torch.float32, device="cuda")
    p = torch.as_tensor(rng.standard_normal((case["nz"], case["ny"], case["nx"])), dtype=torch.float32,
                        device="cuda")
    plan = nd.plan_from_config(case, apply_weights=weights)
    lhs = float((plan.forward(g).double() * p.double()).sum())
    rhs = float((g.double() * plan.adjoint(p).double()).sum())
    plan.close()
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("spec", CASES[:4], ids=IDS[:4])
def test_grad_positions_matches_oracle(nd, spec):
    case = inputs.small_case(**spec)
    rng = np.random.default_rng(spec["seed"] + 300)
    lam = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    want = oracle.grad_positions(problem(case), case["g"], lam)
    plan = nd.plan_from_config(case)
    got = plan.grad_positions(torch.as_tensor(case["g"], dtype=torch.float32, device="cuda"),
                              torch.as_tensor(lam, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    check(got, want, TOL_GRAD)


def test_adjoint_c2_full_size(nd):
    """Workload 2 geometry at full size (4096 sensors, Nt 512, 128x128x256)."""
    case = inputs.make_config(1, with_data=False)
    rng = np.random.default_rng(42)
    p = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    want = oracle.adjoint(problem(case), p)
    plan = nd.plan_from_config(case)
    got = plan.adjoint(torch.as_tensor(p, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    check(got, want, TOL)


def test_adjoint_options(nd):
    case = inputs.small_case(16, 16, 32, 77, 64, seed=26, layout="disc")
    rng = np.random.default_rng(27)
    p = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    for kw in (dict(apply_weights=False), dict(band_mask=True)):
        want = oracle.adjoint(problem(case, **kw), p)
        plan = nd.plan_from_config(case, **kw)
        got = plan.adjoint(torch.as_tensor(p, dtype=torch.float32, device="cuda")).cpu().numpy()
        plan.close()
        check(got, want, TOL)


def test_autograd_function(nd):
    """torch.autograd: gradients of <lambda, R(x) g> w.r.t. g and x."""
    case = inputs.small_case(16, 16, 32, 30, 64, seed=28, layout="scatter")
    plan = nd.plan_from_config(case)
    rng = np.random.default_rng(29)
    lam = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    g = torch.as_tensor(case["g"], dtype=torch.float32, device="cuda").requires_grad_(True)
    xy = torch.as_tensor(case["sensor_xy"], dtype=torch.float64).requires_grad_(True)
    lam_t = torch.as_tensor(lam, dtype=torch.float32, device="cuda")
    p0 = nd.reconstruct(plan, g, xy)
    (p0 * lam_t).sum().backward()
    want_g = oracle.adjoint(problem(case), lam)
    want_xy = oracle.grad_positions(problem(case), case["g"], lam)
    check(g.grad.cpu().numpy(), want_g, TOL)
    check(xy.grad.numpy(), want_xy, TOL_GRAD)
    plan.close()


def test_adjoint_and_grad_wide_rows(nd):
    """2nx = 512 grid columns: the transposed gather with two time samples per
    lane (64 per CTA of 512 threads), and its gradient."""
    case = inputs.small_case(256, 16, 8, 200, 64, seed=31, layout="scatter")
    rng = np.random.default_rng(131)
    p = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    g = rng.standard_normal((case["sensor_xy"].shape[0], case["Nt"]))
    pr = problem(case)
    plan = nd.plan_from_config(case)
    pt = torch.as_tensor(p, dtype=torch.float32, device="cuda")
    got = plan.adjoint(pt).cpu().numpy()
    check(got, oracle.adjoint(pr, p), TOL)
    gg = plan.grad_positions(torch.as_tensor(g, dtype=torch.float32, device="cuda"), pt).cpu().numpy()
    want = oracle.grad_positions(pr, g, p)
    plan.close()
    check(gg, want, TOL_GRAD)


def test_adjoint_in_passes_under_workspace_limit(nd):
    """A workspace limit that leaves room for only part of the entry buffer
    makes the adjoint run in several passes over the time samples; the result
    is the same as in one pass."""
    case = inputs.small_case(16, 16, 16, 600, 256, seed=32, layout="scatter")
    rng = np.random.default_rng(132)
    p = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    pt = torch.as_tensor(p, dtype=torch.float32, device="cuda")
    full = nd.plan_from_config(case)
    a = full.adjoint(pt).cpu().numpy()
    limit = full.workspace_bytes // 3
    full.close()
    tight = nd.plan_from_config(case, max_workspace_bytes=limit)
    assert tight.workspace_bytes <= limit
    b = tight.adjoint(pt).cpu().numpy()
    tight.close()
    assert rel_l2(b, a) <= 1e-6, rel_l2(b, a)
    check(b, oracle.adjoint(problem(case), p), TOL)


LIMITS = [
    dict(nx=2048, ny=8, nz=8, M=20, Nt=16, seed=41, layout="scatter"),
    dict(nx=8, ny=2048, nz=8, M=20, Nt=16, seed=42, layout="scatter"),
    dict(nx=8, ny=8, nz=2048, M=12, Nt=4096, seed=43, layout="scatter"),
]


@pytest.mark.parametrize("spec", LIMITS, ids=["{nx}x{ny}x{nz}_Nt{Nt}".format(**c) for c in LIMITS])
def test_adjoint_and_grad_at_size_limits(nd, spec):
    """nx, ny or nz at 2048 and Nt at 4096: a transposed gather with two time
    samples per CTA over a row of 4096 columns, one-column y transforms, and
    the transposed line FFT of 8192 points."""
    case = inputs.small_case(**spec)
    rng = np.random.default_rng(spec["seed"] + 500)
    p = rng.standard_normal((case["nz"], case["ny"], case["nx"]))
    pr = problem(case)
    plan = nd.plan_from_config(case)
    pt = torch.as_tensor(p, dtype=torch.float32, device="cuda")
    got = plan.adjoint(pt).cpu().numpy()
    want = oracle.adjoint(pr, p)
    check(got, want, TOL)
    gg = plan.grad_positions(torch.as_tensor(case["g"], dtype=torch.float32, device="cuda"), pt).cpu().numpy()
    want_g = oracle.grad_positions(pr, case["g"], p)
    plan.close()
    check(gg, want_g, TOL_GRAD)
