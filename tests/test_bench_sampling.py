"""The sampled accuracy check of bench.py, on the CPU: the spectrum that the
check reads off a volume equals the oracle's spectrum on the sampled lines
when the volume is the oracle's own reconstruction, and a planted error in
the volume shows up in the sampled rel-L2 at the size it has over the whole
volume (Parseval)."""
import numpy as np

import bench
import oracle
from paper_1510_01078_gb300 import inputs


def _cfg():
    case = inputs.small_case(16, 8, 16, 23, 32, seed=51, layout="disc")
    return dict(case, seed=51)


def test_spectrum_of_volume_recovers_the_oracle_spectrum():
    cfg = _cfg()
    pr = bench.oracle_problem(cfg)
    p0 = oracle.forward(pr, cfg["g"])
    jx, jy = bench.sample_lines(cfg, 0.2, seed=3)
    assert len(jx) * len(jy) >= 8 and -8 not in jx and -4 not in jy
    F = oracle.spectrum_block(pr, cfg["g"], jx, jy, oracle.index_set(cfg["nz"]))
    got = bench.spectrum_of_volume(p0, jx, jy)
    np.testing.assert_allclose(got[:, :, 1:], F[:, :, 1:], rtol=0, atol=1e-11 * np.abs(F).max())
    rl2, mx = bench.sampled_errors(p0, jx, jy, F)
    assert rl2 < 1e-12 and mx < 1e-12


def test_sampled_error_sees_a_planted_error():
    cfg = _cfg()
    pr = bench.oracle_problem(cfg)
    p0 = oracle.forward(pr, cfg["g"])
    rng = np.random.default_rng(4)
    noise = rng.standard_normal(p0.shape)
    bad = p0 + 1e-3 * np.linalg.norm(p0) / np.linalg.norm(noise) * noise      # whole-volume rel-L2 1e-3
    jx, jy = bench.sample_lines(cfg, 0.5, seed=5)
    F = oracle.spectrum_block(pr, cfg["g"], jx, jy, oracle.index_set(cfg["nz"]))
    rl2, _ = bench.sampled_errors(bad, jx, jy, F)
    assert 3e-4 < rl2 < 3e-3, rl2


def test_lateral_crop_keeps_spacing_density_and_aperture():
    full = inputs.make_config(2, with_data=False)
    lat = inputs.make_config(2, with_data=False, lateral=128)
    assert (lat["nx"], lat["ny"], lat["nz"], lat["Nt"]) == (128, 128, full["nz"], full["Nt"])
    assert lat["dx"] == full["dx"] and lat["dy"] == full["dy"] and lat["dz"] == full["dz"]
    half = 0.5 * lat["nx"] * lat["dx"]
    xy_full, xy_lat = full["sensor_xy"], lat["sensor_xy"]
    assert np.abs(xy_lat).max() < half
    # exactly the full layout's sensors inside the square, with their weights
    keep = np.all(np.abs(xy_full) < 0.98 * half, axis=1)
    np.testing.assert_array_equal(xy_lat, xy_full[keep])
    np.testing.assert_array_equal(lat["h"], full["h"][keep])
    b = lat["balls"]
    assert np.all(np.abs(b.centres[:, :2]) + b.radii[:, None] < half)
    assert lat["name"] == "c3_paper_scale_lat128"
