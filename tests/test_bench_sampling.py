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
