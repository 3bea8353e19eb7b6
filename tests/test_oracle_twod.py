"""Pins of the 2-D oracle (Sec. 7) against things it does not compute itself:
the 3-D oracle (independent C sums) through the exact embedding of a line
problem, the planar-source closed form (d'Alembert), numpy's FFT for sensors
on the grid, and adjointness."""
import numpy as np
import pytest

import oracle
from oracle.twod import Problem2D, adjoint2d, forward2d, spectrum2d


def _case(seed=3, M=13, nx=16, nz=16, Nt=32, on_grid=False):
    rng = np.random.default_rng(seed)
    dx, dt, c = 1e-4, 20e-9, 1500.0
    dz = c * Nt * dt / nz
    X = nx * dx
    if on_grid:
        x = (np.arange(nx) - nx // 2) * dx
        x[0] += 1e-12 * X
        h = np.full(nx, dx)
    else:
        x = rng.uniform(-0.49 * X, 0.49 * X, size=M)
        h = rng.uniform(0.5, 1.5, size=M) * X / M
    return Problem2D(sensor_x=x, Nt=Nt, dt=dt, c=c, nx=nx, nz=nz, dx=dx, dz=dz, h=h), rng


@pytest.mark.parametrize("weights", [True, False])
def test_line_problem_is_the_row_sum_of_the_3d_problem(weights):
    """Sensors at (x_m, 0) of a 3-D grid with ny rows of dy, areas h_m dy:
    the 3-D NED sum does not depend on jy, so the sum of the 3-D image over
    its rows keeps only jy = 0, whose nu, W and F are the 2-D ones."""
    pr, rng = _case()
    g = rng.standard_normal((pr.M, pr.Nt))
    ny, dy = 8, 1.3e-4
    pr3 = oracle.Problem(sensor_xy=np.stack([pr.sensor_x, np.zeros(pr.M)], 1), h=pr.h * dy, Nt=pr.Nt, dt=pr.dt,
                         c=pr.c, nx=pr.nx, ny=ny, nz=pr.nz, dx=pr.dx, dy=dy, dz=pr.dz, apply_weights=weights)
    pr.apply_weights = weights
    p3 = oracle.forward(pr3, g)
    assert np.allclose(p3.sum(axis=1), forward2d(pr, g), rtol=0, atol=1e-12 * np.abs(p3).max() * ny)


def test_planar_source_is_exact():
    """Sensors on the whole grid line, data of a laterally uniform source,
    g_n = (f(n c dt) + f(-n c dt)) / 2 (d'Alembert): with nz = Nt and
    Z = c Nt dt the reconstruction is f(z) + f(-z) = 2 g(z/c) at every x
    (here f is even on the periodic grid, so g = f and the result is 2 f)."""
    pr, rng = _case(on_grid=True, nx=16, nz=32, Nt=32)
    f = rng.standard_normal(pr.nz)
    f[1:] = 0.5 * (f[1:] + f[1:][::-1])              # even on the periodic grid, so g_n = f_n
    g = np.tile(f, (pr.nx, 1))
    p = forward2d(pr, g)
    assert np.allclose(p, 2.0 * f[:, None] * np.ones((1, pr.nx)), atol=1e-10)


def test_ned_on_the_grid_is_the_fft_and_the_ner_the_c_sums():
    """Sensors on the grid points (h = dx), unweighted: G[jx, n] is the
    centred DFT of the data along x (numpy's FFT), and F[jx, l] its NER sum
    at nu[jx, l], evaluated here by the 3-D oracle's C core (oracle.ner)."""
    pr, rng = _case(on_grid=True, nx=16, nz=8, Nt=16)
    pr.apply_weights = False
    g = rng.standard_normal((pr.nx, pr.Nt))
    G = np.fft.fftshift(np.fft.fft(np.fft.ifftshift(g, axes=0), axis=0), axes=0)     # jx = -nx/2..nx/2-1
    jx = np.arange(-(pr.nx // 2), pr.nx - pr.nx // 2)
    l = np.arange(-(pr.nz // 2), pr.nz - pr.nz // 2)
    JX, L = np.meshgrid(jx, l, indexing="ij")
    from oracle.twod import nu2d
    pr3 = oracle.Problem(sensor_xy=np.zeros((1, 2)), Nt=pr.Nt, dt=pr.dt, c=pr.c, nx=8, ny=8, nz=8, dx=1.0, dy=1.0,
                         dz=1.0)
    want = oracle.ner(pr3, G, nu2d(pr, JX, L))
    assert np.allclose(spectrum2d(pr, g), want, atol=1e-10)


@pytest.mark.parametrize("weights", [True, False])
def test_adjoint_is_the_transpose(weights):
    pr, rng = _case(seed=5)
    pr.apply_weights = weights
    g = rng.standard_normal((pr.M, pr.Nt))
    p = rng.standard_normal((pr.nz, pr.nx))
    a = float((forward2d(pr, g) * p).sum())
    b = float((g * adjoint2d(pr, p)).sum())
    assert a == pytest.approx(b, rel=1e-11)
