"""Host checks of the sensor-placement helpers (Sec. 6, Appendix A and B):
the equi-steradian layout against the solid-angle rule that defines it and
against plane geometry, the r^3 weighting against the areas it stands for,
and the correlation coefficient against numpy's."""
import math

import numpy as np
import pytest

from paper_1510_01078_gb300 import placement as P

D, R0 = 18e-3, 5e-3


@pytest.fixture(scope="module", params=[64, 1024, 4096])
def layout(request):
    N = request.param
    xy, h, sl = P.equi_steradian(N, D, R0, return_slices=True)
    return N, xy, h, sl


def test_every_sensor_gets_one_unit_solid_angle(layout):
    """Appendix A: omega j_k = 2 pi (cos theta_{k-1} - cos theta_k), omega = Omega / N,
    Omega = 2 pi (1 - cos theta_max); the slices tile the cap from the axis."""
    N, xy, h, sl = layout
    tmax = math.atan(0.5 * D / R0)
    omega = 2 * math.pi * (1 - math.cos(tmax)) / N
    assert sl[0]["theta_in"] == 0.0 and sl[0]["j"] == 1
    for a, b in zip(sl[:-1], sl[1:]):
        assert b["theta_in"] == pytest.approx(a["theta_out"], abs=1e-15)
    for s in sl:
        solid = 2 * math.pi * (math.cos(s["theta_in"]) - math.cos(s["theta_out"]))
        assert solid == pytest.approx(omega * s["j"], rel=1e-9)
    assert sum(s["j"] for s in sl) == xy.shape[0]


def test_slice_counts_are_powers_of_two_that_at_most_double(layout):
    _, _, _, sl = layout
    js = [s["j"] for s in sl]
    assert all(j & (j - 1) == 0 for j in js)
    assert all(b in (a, 2 * a) for a, b in zip(js[:-1], js[1:]))
    assert js[:5] == [1, 2, 4, 8, 16]            # the first slices double each time (ring diameter vs neighbour)


def test_points_lie_on_their_slices_and_inside_the_disc(layout):
    """Sensor k,i at (pol, az) = (mid polar angle, phi_{i,k}) projected from
    (0, 0, R0) onto the plane: radius R0 tan(pol); all inside the disc of
    diameter D; the count is N rounded to whole slices (within one slice)."""
    N, xy, h, sl = layout
    r = np.sqrt((xy ** 2).sum(1))
    assert r.max() < 0.5 * D
    i = 0
    for s in sl:
        rr = r[i:i + s["j"]]
        assert np.allclose(rr, R0 * math.tan(s["pol"]), rtol=1e-12, atol=1e-15)
        if s["j"] > 1:
            assert s["pol"] == pytest.approx(0.5 * (s["theta_in"] + s["theta_out"]), rel=1e-12)
        i += s["j"]
    assert abs(xy.shape[0] - N) <= sl[-1]["j"]


def test_azimuths_follow_the_previous_slice(layout):
    """phi_{i,k} = 2 pi i / j_k + pi / j_k + phi_r with phi_r the previous slice's
    last azimuth plus half its spacing (the reading of the garbled phi_r)."""
    _, xy, _, sl = layout
    for a, b in zip(sl[:-1], sl[1:]):
        phi_r = a["phi"][-1] + math.pi / a["j"]
        want = 2 * math.pi * np.arange(b["j"]) / b["j"] + math.pi / b["j"] + phi_r
        assert np.allclose(b["phi"], want, rtol=0, atol=1e-12)
        d = np.diff(b["phi"])
        assert np.allclose(d, 2 * math.pi / b["j"])


def test_r_cubed_weights_stand_for_the_plane_area_of_each_slice(layout):
    """Sec. 6.2: the projected density of an equal-solid-angle layout is
    proportional to r0 / r^3, so h_m proportional to r^3 gives each slice
    about the plane area of its annulus [R0 tan theta_in, R0 tan theta_out];
    the weights sum to the disc area.  (Weights proportional to r^2 would
    miss the annulus areas by the factor r0 / r.)"""
    N, xy, h, sl = layout
    assert h.sum() == pytest.approx(math.pi * D * D / 4, rel=1e-12)
    rr = np.sqrt((xy ** 2).sum(1) + R0 * R0)
    assert np.allclose(h / h.sum(), rr ** 3 / (rr ** 3).sum(), rtol=1e-12)
    # per slice: sum of h against the annulus area, up to one common factor
    # (the disc beyond the last slice is not covered)
    i, ratio = sl[0]["j"], []
    for s in sl[1:]:
        area = math.pi * R0 * R0 * (math.tan(s["theta_out"]) ** 2 - math.tan(s["theta_in"]) ** 2)
        ratio.append(h[i:i + s["j"]].sum() / area)
        i += s["j"]
    ratio = np.array(ratio)
    assert np.allclose(ratio, np.median(ratio), rtol=0.02 if N >= 1024 else 0.06)
    # the same with r^2 weights is far from constant over the slices
    i, r2 = sl[0]["j"], []
    for s in sl[1:]:
        area = math.pi * R0 * R0 * (math.tan(s["theta_out"]) ** 2 - math.tan(s["theta_in"]) ** 2)
        r2.append((rr[i:i + s["j"]] ** 2).sum() / area)
        i += s["j"]
    r2 = np.array(r2)
    assert r2.max() / r2.min() > 1.2


def test_regular_grid():
    xy, h = P.regular_grid(1000, D)
    assert xy.shape == (32 * 32, 2) and np.abs(xy).max() < 0.5 * D
    assert h.sum() == pytest.approx(D * D, rel=1e-12)
    assert np.allclose(np.unique(np.round(np.diff(np.unique(xy[:, 0])), 15)), D / 32)


def test_corrcoef_matches_numpy_and_its_limits():
    rng = np.random.default_rng(7)
    a = rng.standard_normal((6, 5, 4))
    b = 0.3 * a + rng.standard_normal((6, 5, 4))
    assert P.corrcoef(a, b) == pytest.approx(np.corrcoef(a.ravel(), b.ravel())[0, 1], rel=1e-12)
    assert P.corrcoef(a, 3 * a + 2) == pytest.approx(1.0, abs=1e-14)
    assert P.corrcoef(a, -a) == pytest.approx(-1.0, abs=1e-14)
    m = P.upper_half_mask(6, 5, 4)
    assert m[:3].all() and not m[3:].any()
    assert P.corrcoef(a, b, m) == pytest.approx(np.corrcoef(a[:3].ravel(), b[:3].ravel())[0, 1], rel=1e-12)
    torch = pytest.importorskip("torch")
    ta, tb = torch.as_tensor(a), torch.as_tensor(b)
    assert float(P.corrcoef(ta, tb, torch.as_tensor(m))) == pytest.approx(P.corrcoef(a, b, m), rel=1e-12)


def test_bad_arguments():
    with pytest.raises(ValueError):
        P.equi_steradian(0, D, R0)
    with pytest.raises(ValueError):
        P.equi_steradian(10, -1.0, R0)


def test_equi_angular_layout():
    """Equal angles between neighbouring sensor lines seen from (0, r0), all
    inside the detection region, and h proportional to r^2 stands for the
    sensor's share of the line (the local spacing grows like r^2 / r0)."""
    N, D, r0 = 32, 40e-3, 6e-3
    x, h = P.equi_angular(N, D, r0)
    th = np.arctan(x / r0)
    assert np.allclose(np.diff(th), 2 * math.atan(0.5 * D / r0) / N, rtol=1e-12)
    assert np.abs(x).max() < 0.5 * D and np.allclose(x, -x[::-1], atol=1e-15)
    assert h.sum() == pytest.approx(D, rel=1e-12)
    spacing = 0.5 * (x[2:] - x[:-2])
    ratio = h[1:-1] / spacing
    assert np.allclose(ratio, np.median(ratio), rtol=0.04)
    # the discretisation error of that statement falls with N
    x2, h2 = P.equi_angular(4 * N, D, r0)
    r2 = h2[1:-1] / (0.5 * (x2[2:] - x2[:-2]))
    assert np.abs(r2 / np.median(r2) - 1).max() < 0.25 * np.abs(ratio / np.median(ratio) - 1).max()
    assert h.max() / h.min() == pytest.approx((x.max() ** 2 + r0 ** 2) / (x[N // 2] ** 2 + r0 ** 2), rel=1e-12)
