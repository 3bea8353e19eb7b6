"""Pins of the oracle's utilities (data low-pass of Sec. 8, Tenenbaum
sharpness of Appendix B, MIPs) against closed forms, brute force and a
library routine."""
import math

import numpy as np
import pytest

from oracle import utilities as U


def test_nearest_neighbour_on_a_grid_is_the_step():
    s = 0.37e-3
    q = (np.arange(7) - 3) * s
    YY, XX = np.meshgrid(q, q, indexing="ij")
    xy = np.stack([XX.ravel(), YY.ravel()], 1)
    assert np.allclose(U.nearest_neighbour_distance(xy), s, rtol=1e-12)
    assert np.isinf(U.nearest_neighbour_distance(xy[:1]))[0]


def test_nearest_neighbour_matches_a_kd_tree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(3)
    xy = rng.uniform(-1e-2, 1e-2, size=(500, 2))
    d, _ = spatial.cKDTree(xy).query(xy, k=2)
    assert np.allclose(U.nearest_neighbour_distance(xy), d[:, 1], rtol=1e-12)


def test_lowpass_passes_tones_below_and_removes_tones_above_the_cut():
    """Two sensors 0.3 mm apart: f_cut = c / (2 * 0.3 mm) = 2.5 MHz; with
    Nt = 256 and dt = 20 ns the bin spacing is 1/(Nt dt) = 195.3 kHz, so bins
    |k| <= floor(12.8) = 12 are kept."""
    Nt, dt, c = 256, 20e-9, 1500.0
    xy = np.array([[0.0, 0.0], [0.3e-3, 0.0]])
    assert list(U.lowpass_bins(xy, Nt, dt, c)) == [12, 12]
    n = np.arange(Nt)
    lo = np.cos(2 * np.pi * 12 * n / Nt + 0.3) + 0.5
    hi = np.sin(2 * np.pi * 13 * n / Nt)
    g = np.stack([lo + hi, 2 * hi])
    out = U.lowpass(g, xy, dt, c)
    assert np.allclose(out[0], lo, atol=1e-12)
    assert np.allclose(out[1], 0.0, atol=1e-12)
    # idempotent, and a projection (no gain above one)
    assert np.allclose(U.lowpass(out, xy, dt, c), out, atol=1e-12)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((2, Nt))
    f = U.lowpass(r, xy, dt, c)
    assert (f * f).sum() <= (r * r).sum()
    assert np.isclose((f * (r - f)).sum(), 0.0, atol=1e-9)       # orthogonal projection


def test_lowpass_of_a_lone_sensor_is_the_identity_and_bins_clip_at_nyquist():
    rng = np.random.default_rng(6)
    g = rng.standard_normal((1, 64))
    assert np.allclose(U.lowpass(g, np.zeros((1, 2)), 20e-9, 1500.0), g, atol=1e-12)
    xy = np.array([[0.0, 0.0], [1e-9, 0.0]])                      # 1 nm apart: cut far above Nyquist
    assert list(U.lowpass_bins(xy, 64, 20e-9, 1500.0)) == [32, 32]


def test_tenenbaum_closed_forms():
    ny, nx = 9, 12
    assert U.tenenbaum(np.full((ny, nx), 3.5)) == 0.0
    # ramp a x + b y: Sobel responses 8a and 8b at every valid pixel
    a, b = 0.7, -1.3
    y, x = np.mgrid[0:ny, 0:nx]
    F = U.tenenbaum(a * x + b * y)
    assert F == pytest.approx(64 * (a * a + b * b) * (nx - 2) * (ny - 2) / (nx * ny), rel=1e-12)
    # a unit impulse two pixels from the border: the responses are the
    # operator's own entries, sum of squares 12 for each direction
    d = np.zeros((ny, nx))
    d[4, 5] = 1.0
    assert U.tenenbaum(d) == pytest.approx(24.0 / (nx * ny), rel=1e-12)


def test_mip_finds_a_planted_maximum():
    rng = np.random.default_rng(8)
    v = rng.uniform(0, 1, size=(5, 6, 7))
    v[3, 2, 4] = 5.0
    for axis, pos in ((0, (2, 4)), (1, (3, 4)), (2, (3, 2))):
        m = U.mip(v, axis)
        assert m[pos] == 5.0 and (m <= 5.0).all()
        assert m.shape == tuple(s for i, s in enumerate(v.shape) if i != axis)
        assert np.all(m >= np.take(v, 0, axis=axis))


def test_linear_interpolation_oracle_against_direct_sums():
    """The FFT-with-linear-interpolation oracle (Table 1's comparison method)
    at grid frequencies nu = mu / sigma equals the direct NER sum there, and
    in between it is the straight line between the direct sums at the two
    neighbouring grid frequencies (direct sums from the C core)."""
    import oracle
    from oracle import comparison as C
    pr = oracle.Problem(sensor_xy=np.zeros((1, 2)), Nt=64, dt=20e-9, c=1500.0, nx=8, ny=8, nz=16,
                        dx=1e-4, dy=1e-4, dz=1500.0 * 64 * 20e-9 / 16)
    rng = np.random.default_rng(9)
    G = rng.standard_normal((3, 64)) + 1j * rng.standard_normal((3, 64))
    for sigma in (1, 2):
        grid = np.array([[-7.0, 0.0, 3.0, 31.5 if sigma == 2 else 31.0]] * 3) / 1.0
        grid = np.round(grid * sigma) / sigma
        assert np.allclose(C.ner_linear(pr, G, grid, sigma), oracle.ner(pr, G, grid), atol=1e-10)
        nus = rng.uniform(-40, 40, size=(3, 5))
        got = C.ner_linear(pr, G, nus, sigma)
        v = sigma * nus
        lo, t = np.floor(v) / sigma, v - np.floor(v)
        want = (1 - t) * oracle.ner(pr, G, lo) + t * oracle.ner(pr, G, lo + 1.0 / sigma)
        assert np.allclose(got, want, atol=1e-10)
        # and it is not the direct sum off the grid
        assert np.abs(got - oracle.ner(pr, G, nus)).max() > 1e-3
