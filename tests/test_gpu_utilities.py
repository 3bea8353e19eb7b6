"""GPU utilities against the oracle: the data low-pass of Sec. 8 (cut-off
bins bit for bit, the filtered data to FP32 FFT rounding), the Tenenbaum
sharpness of Appendix B and maximum intensity projections."""
import numpy as np
import pytest

from oracle import utilities as U
from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


@pytest.mark.parametrize("layout", ["c2", "disc", "equi_steradian"])
def test_lowpass_bins_match_oracle(nd, layout):
    if layout == "c2":
        cfg = inputs.make_config(1, with_data=False)
    elif layout == "disc":
        cfg = inputs.small_case(64, 64, 32, 3000, 512, seed=81, layout="disc")
    else:
        from paper_1510_01078_gb300 import placement as P
        cfg = inputs.small_case(64, 64, 32, 10, 512, seed=82, layout="scatter")
        xy, h = P.equi_steradian(1024, 0.9 * cfg["nx"] * cfg["dx"], 2e-3)
        cfg = dict(cfg, sensor_xy=xy, h=h)
    plan = nd.plan_from_config(cfg)
    got = plan.lowpass_bins()
    want = U.lowpass_bins(cfg["sensor_xy"], cfg["Nt"], cfg["dt"], cfg["c"])
    assert np.array_equal(got, want)
    assert got.min() < cfg["Nt"] // 2            # the cut is active somewhere
    plan.close()


@pytest.mark.parametrize("M,Nt", [(301, 128), (64, 2048), (7, 64)])
def test_lowpass_matches_oracle(nd, M, Nt):
    cfg = inputs.small_case(32, 32, 32, M, Nt, seed=83 + M, layout="disc")
    rng = np.random.default_rng(84)
    g = rng.standard_normal((M, Nt))
    plan = nd.plan_from_config(cfg)
    gt = torch.as_tensor(g, dtype=torch.float32, device="cuda")
    out = plan.lowpass(gt).cpu().numpy()
    want = U.lowpass(g.astype(np.float32).astype(np.float64), cfg["sensor_xy"], cfg["dt"], cfg["c"])
    check(out, want, 1e-5)
    # in place
    plan.lowpass(gt, out=gt)
    assert np.array_equal(gt.cpu().numpy(), out)
    plan.close()


def test_tenenbaum_matches_oracle(nd):
    rng = np.random.default_rng(85)
    imgs = rng.standard_normal((3, 37, 53)).astype(np.float32)
    F = nd.tenenbaum(torch.as_tensor(imgs, device="cuda")).cpu().numpy()
    want = np.array([U.tenenbaum(im) for im in imgs.astype(np.float64)])
    check(F, want, 1e-6)
    one = float(nd.tenenbaum(torch.as_tensor(imgs[1], device="cuda")))
    assert one == F[1]                            # fixed summation order: same bits
    # degenerate sizes: no valid pixel
    z = nd.tenenbaum(torch.zeros((2, 2, 9), device="cuda")).cpu().numpy()
    assert np.array_equal(z, [0.0, 0.0])


def test_mip_matches_oracle(nd):
    rng = np.random.default_rng(86)
    v = rng.standard_normal((19, 33, 70)).astype(np.float32)
    vt = torch.as_tensor(v, device="cuda")
    for axis in (0, 1, 2):
        assert np.array_equal(nd.mip(vt, axis).cpu().numpy(), U.mip(v, axis))


def test_utilities_reject_bad_arguments(nd):
    import ctypes
    lib = nd.library()
    assert lib.nedner_mip(None, 4, 4, 4, 0, None, None) == nd.EINVAL
    v = torch.zeros((4, 4, 4), device="cuda")
    o = torch.zeros((4, 4), device="cuda")
    assert lib.nedner_mip(ctypes.c_void_p(v.data_ptr()), 4, 4, 4, 3, ctypes.c_void_p(o.data_ptr()), None) == nd.EINVAL
    assert lib.nedner_tenenbaum(None, -1, 4, 4, None, None) == nd.EINVAL
    assert lib.nedner_tenenbaum(None, 0, 4, 4, None, None) == nd.OK
    assert lib.nedner_lowpass(None, None, None, None) == nd.EINVAL
