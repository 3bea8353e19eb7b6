"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names what it pins.  None of them re-types the oracle's formula:
they use a textbook FFT on special cases where the paper's sums reduce to it
(Sec. 2: on-grid sensors turn Eq. disc_rec into Eq. equiv_rec), closed forms
(geometric series, d'Alembert), transposition identities, finite differences
and the physics of a ball phantom.
"""
import numpy as np
import pytest

import oracle
from oracle import Problem
from paper_1510_01078_gb300 import inputs


def _problem(case, **kw):
    return Problem(sensor_xy=case["sensor_xy"], h=case["h"], Nt=case["Nt"], dt=case["dt"], c=case["c"],
                   nx=case["nx"], ny=case["ny"], nz=case["nz"], dx=case["dx"], dy=case["dy"],
                   dz=case["dz"], **kw)


def _grid_problem(nx, ny, nz, Nt, dt=20e-9, c=1500.0, dx=1e-4):
    qx = np.arange(nx) - nx // 2
    qy = np.arange(ny) - ny // 2
    QY, QX = np.meshgrid(qy, qx, indexing="ij")
    xy = np.stack([QX.ravel() * dx, QY.ravel() * dx], 1)
    return Problem(sensor_xy=xy, h=np.full(nx * ny, dx * dx), Nt=Nt, dt=dt, c=c, nx=nx, ny=ny, nz=nz,
                   dx=dx, dy=dx, dz=c * Nt * dt / nz)


# P1 ------------------------------------------------------------------------
def test_ned_on_grid_is_the_2d_dft():
    """Sensors on Delta_x G_x with h = Delta_x^2: Eq. disc_rec reduces to the
    plain DFT of Eq. equiv_rec (Sec. 2).  Compared with numpy.fft.fft2."""
    nx, ny, Nt = 8, 6, 5
    pr = _grid_problem(nx, ny, 4, Nt)
    rng = np.random.default_rng(0)
    g = rng.standard_normal((pr.M, Nt))
    G = oracle.ned(pr, g)                                       # (nx, ny, Nt), index j + n/2
    B = g.reshape(ny, nx, Nt).transpose(2, 0, 1)                # [n][qy][qx], q = index - n/2
    D = np.fft.fft2(B)                                          # sum exp(-2 pi i (jy qy + jx qx)/n)
    jx = oracle.index_set(nx)
    jy = oracle.index_set(ny)
    for a, kx in enumerate(jx):
        for b, ky in enumerate(jy):
            ref = D[:, ky % ny, kx % nx] * (-1.0) ** (kx + ky)  # exp(+i pi k) from the -n/2 offset
            np.testing.assert_allclose(G[a, b], ref, rtol=0, atol=1e-11 * np.abs(D).max())


def test_ned_shift_and_symmetry():
    """Moving every sensor by one grid step multiplies the NED sum by
    exp(-2 pi i jx / nx); real data give G(-j) = conj G(j)."""
    case = inputs.small_case(8, 8, 8, 37, 6, seed=3)
    pr = _problem(case)
    jx = np.array([-3, -1, 0, 2, 3])
    jy = np.array([-2, 0, 1, 3])
    G0 = oracle.ned(pr, case["g"], jx, jy)
    pr2 = _problem(case)
    pr2.sensor_xy = case["sensor_xy"] + np.array([pr.dx, 0.0])
    G1 = oracle.ned(pr2, case["g"], jx, jy)
    np.testing.assert_allclose(G1, G0 * np.exp(-2j * np.pi * jx / pr.nx)[:, None, None], atol=1e-10)
    Gm = oracle.ned(pr, case["g"], -jx, -jy)
    np.testing.assert_allclose(Gm, np.conj(G0), atol=1e-10)


# P2 ------------------------------------------------------------------------
@pytest.mark.parametrize("nz", [16, 8])
def test_ner_on_axis_is_the_1d_dft(nz):
    """On the j = 0 line with Z = c Nt dt the kappa map gives nu = l
    (Eq. equiv_rec, kappa = sign(l)|l|), so the NER sum is the length-Nt DFT."""
    Nt = 16
    pr = _grid_problem(4, 4, nz, Nt)
    l = oracle.index_set(nz)
    v = oracle.nu(pr, 0, 0, l)
    np.testing.assert_allclose(v, l, rtol=0, atol=1e-12)
    rng = np.random.default_rng(1)
    G = rng.standard_normal(Nt) + 1j * rng.standard_normal(Nt)
    F = oracle.ner(pr, G[None], v[None])[0]
    np.testing.assert_allclose(F, np.fft.fft(G)[l % Nt], atol=1e-11)


# P3 ------------------------------------------------------------------------
def test_ner_single_tone_is_the_dirichlet_kernel():
    """A tone exp(2 pi i nu0 n/Nt) evaluated at non-integer nu gives the
    geometric-series closed form exp(-i pi d (Nt-1)/Nt) sin(pi d)/sin(pi d/Nt),
    d = nu - nu0."""
    Nt = 64
    pr = _grid_problem(4, 4, 8, Nt)
    nu0 = 5.3
    n = np.arange(Nt)
    G = np.exp(2j * np.pi * nu0 * n / Nt)
    nus = np.array([-7.9, -0.25, 3.1, 5.29, 11.77, 40.5])
    F = oracle.ner(pr, G[None], nus[None])[0]
    d = nus - nu0
    ref = np.exp(-1j * np.pi * d * (Nt - 1) / Nt) * np.sin(np.pi * d) / np.sin(np.pi * d / Nt)
    np.testing.assert_allclose(F, ref, atol=1e-10)


def test_ner_adj_at_integer_frequencies_is_the_inverse_dft():
    """At nu = 0..Nt-1 the transposed NER sum sum_l exp(+2 pi i nu_l n/Nt) P_l is
    Nt times the inverse DFT of P."""
    Nt = 32
    pr = _grid_problem(4, 4, 8, Nt)
    rng = np.random.default_rng(5)
    P = rng.standard_normal((2, Nt)) + 1j * rng.standard_normal((2, Nt))
    nus = np.tile(np.arange(Nt, dtype=np.float64), (2, 1))
    T = oracle.ner_adj(pr, P, nus)
    np.testing.assert_allclose(T, Nt * np.fft.ifft(P, axis=1), atol=1e-10)


def test_ner_adj_is_the_conjugate_transpose_of_ner():
    """<ner(G), P> = <G, ner_adj(P)> for non-integer frequencies."""
    Nt = 48
    pr = _grid_problem(4, 4, 8, Nt)
    rng = np.random.default_rng(6)
    G = rng.standard_normal((3, Nt)) + 1j * rng.standard_normal((3, Nt))
    nus = rng.uniform(-30.0, 30.0, (3, 11))
    P = rng.standard_normal((3, 11)) + 1j * rng.standard_normal((3, 11))
    lhs = np.vdot(oracle.ner(pr, G, nus), P)
    rhs = np.vdot(G, oracle.ner_adj(pr, P, nus))
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_kappa_map_and_jacobian_special_values():
    """W(0,0) = 2 and W(j != 0, 0) = 0 (the readings of the 0/0 in 2l/kappa);
    on the j = 0 axis W = 2 for every l; kappa is odd in l and depends on j
    only through |j|."""
    pr = _grid_problem(8, 8, 8, 8)
    assert oracle.jacobian(pr, 0, 0, 0) == 2.0
    assert oracle.jacobian(pr, 3, -2, 0) == 0.0
    np.testing.assert_allclose(oracle.jacobian(pr, 0, 0, np.arange(-4, 4)[np.arange(-4, 4) != 0]), 2.0)
    v = oracle.nu(pr, 3, -2, np.array([-3, 3]))
    assert v[0] == -v[1] and v[1] > 3
    assert oracle.nu(pr, -3, 2, 3) == oracle.nu(pr, 3, -2, 3)
    # |nu| >= |l| with equality on the axis; W <= 2
    assert np.all(oracle.jacobian(pr, 1, 1, np.arange(1, 5)) < 2.0)


# P4 ------------------------------------------------------------------------
def test_ball_nwave_closed_form():
    """The N-wave of a uniform ball integrates to zero over time and peaks
    at A R / (2 r) at t = (r - R)/c."""
    balls = inputs.Balls(np.array([[0.0, 0.0, 5e-3]]), np.array([0.5e-3]), np.array([1.0]))
    dt = 1e-10
    g = inputs.nwave_data(np.array([[0.0, 0.0]]), balls, 60000, dt)[0]
    assert abs(g.sum() * dt) < 1e-3 * np.abs(g).max() * 2 * 0.5e-3 / 1500
    r, R = 5e-3, 0.5e-3
    assert abs(g.max() - R / (2 * r)) < 1e-3 * R / (2 * r)
    assert abs(np.argmax(g) * dt - (r - R) / 1500) < 2 * dt


# IDFT brute force ------------------------------------------------------------
def test_image_from_spectrum_brute_force():
    """The final uniform inverse DFT (Sec. 3 step 3) with voxel centring,
    against a plain loop over every (voxel, frequency) pair."""
    pr = _grid_problem(4, 6, 4, 8)
    rng = np.random.default_rng(2)
    F = rng.standard_normal((4, 6, 4)) + 1j * rng.standard_normal((4, 6, 4))
    p = oracle.image_from_spectrum(pr, F)
    jx, jy, l = oracle.index_set(4), oracle.index_set(6), oracle.index_set(4)
    ref = np.zeros((4, 6, 4))
    for qz in range(4):
        for qy in range(6):
            for qx in range(4):
                s = 0j
                for a, kx in enumerate(jx):
                    for b, ky in enumerate(jy):
                        for c_, kz in enumerate(l):
                            ph = kx * (qx - 2) / 4 + ky * (qy - 3) / 6 + kz * qz / 4
                            s += F[a, b, c_] * np.exp(2j * np.pi * ph)
                ref[qz, qy, qx] = s.real / (4 * 6 * 4)
    np.testing.assert_allclose(p, ref, atol=1e-12)


# P5 ------------------------------------------------------------------------
@pytest.mark.parametrize("weights,mask", [(True, False), (False, False), (True, True)])
def test_adjoint_identity(weights, mask):
    """<R g, p> = <g, R^T p> for random g, p (R real-linear), scattered sensors."""
    case = inputs.small_case(8, 6, 10, 23, 12, seed=5)
    pr = _problem(case, apply_weights=weights, band_mask=mask)
    rng = np.random.default_rng(6)
    g = rng.standard_normal((pr.M, pr.Nt))
    p = rng.standard_normal((pr.nz, pr.ny, pr.nx))
    lhs = np.sum(oracle.forward(pr, g) * p)
    rhs = np.sum(g * oracle.adjoint(pr, p))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs) + 1e-300) + 1e-14
    assert abs(lhs) > 1e-6


# P6 ------------------------------------------------------------------------
def test_plane_source_exact_recovery():
    """A laterally uniform source f(z) seen by sensors covering the grid
    (h = Delta_x^2): only the j = 0 line is non-zero, nu = l, W = 2, and with
    nz = Nt, dz = c dt the reconstruction is 2 g(t = z/c) = f(z) + f(-z)
    (d'Alembert), exactly."""
    nx, ny, Nt = 6, 4, 32
    pr = _grid_problem(nx, ny, Nt, Nt)
    rng = np.random.default_rng(7)
    f = rng.standard_normal(Nt)
    g = np.tile(f, (pr.M, 1))
    p0 = oracle.forward(pr, g)
    np.testing.assert_allclose(p0, np.broadcast_to((2 * f)[:, None, None], p0.shape), atol=1e-11)


def test_plane_source_bandlimited_recovery_coarse_depth():
    """Same with nz < Nt: a data trace band-limited to |nu| < nz/2 is
    recovered as 2 g sampled at z = qz dz (the depth grid is coarser than c dt)."""
    nx, ny, Nt, nz = 4, 4, 64, 16
    pr = _grid_problem(nx, ny, nz, Nt)
    n = np.arange(Nt)
    f = 0.3 + np.cos(2 * np.pi * 3 * n / Nt + 0.4) - 0.5 * np.sin(2 * np.pi * 7 * n / Nt)
    g = np.tile(f, (pr.M, 1))
    p0 = oracle.forward(pr, g)
    zq = np.arange(nz) * Nt / nz
    want = 2 * (0.3 + np.cos(2 * np.pi * 3 * zq / Nt + 0.4) - 0.5 * np.sin(2 * np.pi * 7 * zq / Nt))
    np.testing.assert_allclose(p0, np.broadcast_to(want[:, None, None], p0.shape), atol=1e-11)


# P8 ------------------------------------------------------------------------
def test_position_gradient_matches_finite_differences():
    """dL/dx_m for L = <lambda, R(x) g>, against central differences of the
    oracle's forward (step 1e-6 X)."""
    case = inputs.small_case(6, 6, 8, 5, 10, seed=9)
    pr = _problem(case)
    rng = np.random.default_rng(10)
    lam = rng.standard_normal((pr.nz, pr.ny, pr.nx))
    g = case["g"]
    grad = oracle.grad_positions(pr, g, lam)
    h = 1e-6 * pr.X
    fd = np.zeros_like(grad)
    for m in range(pr.M):
        for d in range(2):
            xp = case["sensor_xy"].copy(); xp[m, d] += h
            xm = case["sensor_xy"].copy(); xm[m, d] -= h
            pp = _problem(case); pp.sensor_xy = xp
            pm = _problem(case); pm.sensor_xy = xm
            fd[m, d] = (np.sum(lam * oracle.forward(pp, g)) - np.sum(lam * oracle.forward(pm, g))) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


# P9 ------------------------------------------------------------------------
def test_ball_phantom_recovery():
    """Physics pin of the kappa map, the Jacobian and the scale: a ball seen by
    a dense grid of sensors (aperture half-angle ~ 70 degrees) is reconstructed
    at the right place with roughly the right amplitude.  A flipped nu sign
    moves it to the far end of the depth range, a dropped Jacobian halves the
    amplitude and a wrong lateral scale smears it."""
    nx = ny = 64
    nz = 64
    dx = 0.1e-3
    c = 1500.0
    Nt = 128
    dt = nz * dx / (c * Nt)          # dz = dx
    pr = _grid_problem(nx, ny, nz, Nt, dt=dt, dx=dx)
    centre, R = np.array([0.0, 0.0, 1.0e-3]), 0.4e-3
    balls = inputs.Balls(centre[None], np.array([R]), np.array([1.0]))
    g = inputs.nwave_data(pr.sensor_xy, balls, Nt, dt, c)
    p0 = oracle.forward(pr, g)
    truth = inputs.voxelise(balls, nx, ny, nz, dx, dx, pr.dz)
    x = (np.arange(nx) - nx // 2) * dx
    z = np.arange(nz) * pr.dz
    Zg, Yg, Xg = np.meshgrid(z, x, x, indexing="ij")
    r = np.sqrt(Xg ** 2 + Yg ** 2 + (Zg - centre[2]) ** 2)
    core = p0[r < R / 2].mean()
    far = p0[(r > 2.5 * R) & (Zg < pr.Z / 2)]
    assert 0.5 < core < 1.2, core
    assert abs(far.mean()) < 0.02 and np.sqrt(np.mean(far ** 2)) < 0.1
    upper = slice(0, nz // 2)
    cc = np.corrcoef(p0[upper].ravel(), truth[upper].ravel())[0, 1]
    assert cc > 0.7, cc
    # nothing of comparable size at the mirrored depth Z - z_c
    mirror = p0[np.sqrt(Xg ** 2 + Yg ** 2 + (Zg - (pr.Z - centre[2])) ** 2) < R / 2].mean()
    assert abs(mirror) < 0.1 * core


def test_line_spectrum_matches_spectrum():
    case = inputs.small_case(6, 8, 8, 11, 10, seed=12)
    pr = _problem(case)
    F = oracle.spectrum(pr, case["g"])
    jx = np.array([-3, 0, 2]); jy = np.array([1, -4, 3])
    ls = oracle.index_set(pr.nz)
    S = oracle.line_spectrum(pr, case["g"], jx, jy, ls)
    for i in range(3):
        np.testing.assert_allclose(S[i], F[jx[i] + 3, jy[i] + 4], atol=1e-12)


# band mask and sparse time samples -------------------------------------------
def test_band_mask_keeps_the_half_open_band():
    """The band mask keeps nu in the half-open band [-Nt/2, Nt/2) of G_Ky
    (Sec. 2).  On the j = 0 line with Z = c Nt dt, nu = l exactly; with
    nz = 4 Nt some l lie outside the band.  The masked coefficient must be
    zero exactly for l >= Nt/2 and l < -Nt/2, keep the tie l = -Nt/2, and
    equal the unmasked coefficient everywhere else."""
    Nt, nz = 16, 64
    pr = _grid_problem(4, 4, nz, Nt)
    pm = _grid_problem(4, 4, nz, Nt)
    pm.band_mask = True
    l = oracle.index_set(nz)
    np.testing.assert_allclose(oracle.nu(pr, 0, 0, l), l, rtol=0, atol=1e-12)
    c0 = oracle.coef(pr, np.zeros_like(l), np.zeros_like(l), l)
    cm = oracle.coef(pm, np.zeros_like(l), np.zeros_like(l), l)
    outside = (l >= Nt // 2) | (l < -(Nt // 2))
    assert outside.sum() == nz - Nt
    assert np.all(cm[outside] == 0.0)
    np.testing.assert_array_equal(cm[~outside], c0[~outside])
    assert cm[l == -(Nt // 2)][0] == c0[l == -(Nt // 2)][0] and c0[l == -(Nt // 2)][0] != 0.0
    assert cm[l == Nt // 2 - 1][0] != 0.0 and cm[l == Nt // 2][0] == 0.0
    # off the axis the band edge moves to smaller |l|: with jx = 2 on a grid of
    # X = 4 dx and Z = c Nt dt, nu^2 = l^2 + (2 Z / X)^2, so the kept set is
    # l^2 < (Nt/2)^2 - (2 Z / X)^2 (no ties there); W(j != 0, 0) = 0 besides
    lat = 2.0 * pr.Z / pr.X
    keep = l.astype(float) ** 2 < (Nt / 2) ** 2 - lat ** 2
    assert 0 < keep.sum() < Nt
    c2 = oracle.coef(pm, np.full_like(l, 2), np.zeros_like(l), l)
    np.testing.assert_array_equal(c2 != 0.0, keep & (l != 0))


def test_sparse_time_samples_equal_dense_zero_filled():
    """The ``ns`` path (data non-zero only at the listed time samples, passed
    as len(ns) columns) gives the same reconstruction as the dense data with
    zeros elsewhere.  ns is unsorted and contains both 0 and Nt - 1."""
    case = inputs.small_case(8, 8, 16, 29, 32, seed=21, layout="disc")
    pr = _problem(case)
    rng = np.random.default_rng(22)
    ns = np.array([17, 0, 31, 5, 22])
    gs = rng.standard_normal((pr.M, len(ns)))
    g = np.zeros((pr.M, pr.Nt))
    g[:, ns] = gs
    dense = oracle.forward(pr, g)
    sparse = oracle.forward(pr, gs, ns=ns)
    assert np.abs(dense).max() > 1e-3
    np.testing.assert_allclose(sparse, dense, rtol=0, atol=1e-12 * np.abs(dense).max())
    # and at the spectrum level, with the band mask on
    pm = _problem(case, band_mask=True)
    np.testing.assert_allclose(oracle.spectrum(pm, gs, ns=ns), oracle.spectrum(pm, g), rtol=0,
                               atol=1e-12 * np.abs(oracle.spectrum(pm, g)).max())


def test_spectrum_block_matches_spectrum():
    """The product-set subset evaluation equals the full spectrum on its lines."""
    case = inputs.small_case(6, 8, 8, 11, 10, seed=13)
    pr = _problem(case)
    F = oracle.spectrum(pr, case["g"])
    jx = np.array([-3, 0, 2]); jy = np.array([1, -4]); ls = np.array([-4, 0, 3])
    S = oracle.spectrum_block(pr, case["g"], jx, jy, ls)
    np.testing.assert_allclose(S, F[np.ix_(jx + 3, jy + 4, ls + 4)], atol=1e-12)


def test_line_restricted_transposes_equal_the_full_ones():
    """adjoint and grad_positions restricted to a product set of lines (and a
    subset of sensors) equal the full sums when the volume's spectrum vanishes
    outside that set: the volume is the real part of an inverse DFT of a
    spectrum supported on jx x jy, whose mirror -jx x -jy the set contains."""
    case = inputs.small_case(16, 8, 16, 40, 32, seed=61, layout="disc")
    pr = _problem(case)
    rng = np.random.default_rng(62)
    jx = np.array([-3, 2]); jy = np.array([1, 3])
    lx = np.concatenate([jx, -jx]); ly = np.concatenate([jy, -jy])
    B = np.zeros((pr.nz, pr.ny, pr.nx), dtype=np.complex128)
    for a in jx:
        for b in jy:
            B[:, b % pr.ny, a % pr.nx] = rng.standard_normal(pr.nz) + 1j * rng.standard_normal(pr.nz)
    p = np.real(np.fft.ifftn(B)) * pr.nx * pr.ny * pr.nz
    sens = np.array([0, 7, 19, 39])
    full = oracle.adjoint(pr, p)
    part = oracle.adjoint(pr, p, lx, ly, sens)
    np.testing.assert_allclose(part, full[sens], rtol=0, atol=1e-10 * np.abs(full).max())
    gf = oracle.grad_positions(pr, case["g"], p)
    gp = oracle.grad_positions(pr, case["g"], p, lx, ly, sens)
    np.testing.assert_allclose(gp, gf[sens], rtol=0, atol=1e-10 * np.abs(gf).max())
    # a set that misses the mirror lines gives a different (wrong) answer
    wrong = oracle.adjoint(pr, p, jx, jy, sens)
    assert np.abs(wrong - full[sens]).max() > 1e-3 * np.abs(full).max()
