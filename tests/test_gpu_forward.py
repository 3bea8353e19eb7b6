"""Parity of the CUDA forward path (nedner_forward, nedner_ned_stage) with the
FP64 oracle, element by element, on seeded inputs.

Tolerance: relative L2 error <= 1e-5 over the whole output for the FP32 path
with the Kaiser-Bessel window, w = 12, sigma = 2.  The window's own
interpolation error there is ~1e-11, so the budget is FP32 rounding: about
1e-7 per operation through a spread of 144 taps and five FFT passes of length
up to 4096 (log2 N ~ 12 stages each), i.e. a few 1e-6.
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    assert torch.cuda.is_available()
    return nedner


def problem(case, **kw):
    return Problem(sensor_xy=case["sensor_xy"], h=case["h"], Nt=case["Nt"], dt=case["dt"], c=case["c"],
                   nx=case["nx"], ny=case["ny"], nz=case["nz"], dx=case["dx"], dy=case["dy"], dz=case["dz"], **kw)


def gpu_forward(nd, case, g=None, **kw):
    plan = nd.plan_from_config(case, **kw)
    gg = torch.as_tensor(np.asarray(case["g"] if g is None else g, dtype=np.float32), device="cuda")
    out = plan.forward(gg)
    torch.cuda.synchronize()
    res = out.cpu().numpy().astype(np.float64)
    plan.close()
    return res


SMALL = [
    dict(nx=16, ny=16, nz=32, M=37, Nt=64, seed=1, layout="scatter"),
    dict(nx=32, ny=16, nz=64, M=301, Nt=128, seed=2, layout="disc"),
    dict(nx=16, ny=32, nz=16, M=1000, Nt=32, seed=3, layout="scatter"),
    dict(nx=8, ny=8, nz=8, M=5, Nt=16, seed=4, layout="scatter"),
    dict(nx=32, ny=32, nz=32, M=333, Nt=256, seed=5, layout="disc", data="balls"),
    dict(nx=16, ny=16, nz=16, M=256, Nt=32, seed=6, layout="grid"),
]


@pytest.mark.parametrize("spec", SMALL, ids=lambda s: "{nx}x{ny}x{nz}_M{M}_Nt{Nt}_{layout}".format(**s))
def test_forward_matches_oracle_small(nd, spec):
    case = inputs.small_case(**spec)
    want = oracle.forward(problem(case), case["g"])
    got = gpu_forward(nd, case)
    check(got, want, TOL)


@pytest.mark.parametrize("spec", SMALL[:3], ids=lambda s: "{nx}x{ny}_M{M}_Nt{Nt}".format(**s))
def test_ned_stage_matches_oracle(nd, spec):
    case = inputs.small_case(**spec)
    pr = problem(case)
    jx = np.arange(0, pr.nx // 2 + 1)
    jy = np.arange(-(pr.ny // 2), pr.ny // 2 + 1)
    want = oracle.ned(pr, case["g"], jx, jy)
    plan = nd.plan_from_config(case)
    got = plan.ned_stage(torch.as_tensor(case["g"], dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    check(got, want, TOL)


def test_forward_c1_tiny(nd):
    """Workload 1: 16x16 centre-dense tensor sensors, Nt 64, 16x16x32 voxels, two balls."""
    case = inputs.make_config(0)
    want = oracle.forward(problem(case), case["g"])
    got = gpu_forward(nd, case)
    check(got, want, TOL)


def test_forward_c2_full_size(nd):
    """Workload 2 at full size (64x64 sensors, Nt 512, 128x128x256), dense noisy data."""
    case = inputs.make_config(1)
    want = oracle.forward(problem(case), case["g"])
    got = gpu_forward(nd, case)
    check(got, want, TOL)


def test_forward_c3_full_size_sparse_time(nd):
    """Workload 3 geometry at full size (16384 scattered sensors, Nt 2048,
    256x256x512) with data non-zero at four time samples only, so the oracle's
    direct sums finish in seconds; every voxel is compared."""
    case = inputs.make_config(2, with_data=False)
    rng = np.random.default_rng(77)
    ns = np.array([3, 400, 1023, 1990])
    gs = rng.standard_normal((case["sensor_xy"].shape[0], len(ns)))
    g = np.zeros((gs.shape[0], case["Nt"]))
    g[:, ns] = gs
    want = oracle.forward(problem(case), gs, ns=ns)
    got = gpu_forward(nd, case, g=g)
    check(got, want, TOL)


# nx, ny or nz at the plan's maximum of 2048, and Nt at its maximum of 4096: a
# spread row of 2nx = 4096 columns (4 time samples per spread CTA, 2 columns in the
# x complex-to-real transform), a y-FFT and y-IFFT of one column, and a line FFT of
# 2Nt = 8192 points (512 threads) with a z-IFFT of 2048.
LIMITS = [
    dict(nx=2048, ny=8, nz=8, M=20, Nt=16, seed=41, layout="scatter"),
    dict(nx=8, ny=2048, nz=8, M=20, Nt=16, seed=42, layout="scatter"),
    dict(nx=8, ny=8, nz=2048, M=12, Nt=4096, seed=43, layout="scatter"),
]
LIMIT_IDS = ["{nx}x{ny}x{nz}_M{M}_Nt{Nt}".format(**c) for c in LIMITS]


@pytest.mark.parametrize("spec", LIMITS, ids=LIMIT_IDS)
def test_forward_at_size_limits(nd, spec):
    case = inputs.small_case(**spec)
    want = oracle.forward(problem(case), case["g"])
    got = gpu_forward(nd, case)
    check(got, want, TOL)


@pytest.mark.parametrize("opt", ["unweighted", "band_mask", "gauss16", "kb8"])
def test_forward_options(nd, opt):
    case = inputs.small_case(16, 16, 32, 77, 64, seed=11, layout="disc")
    kw, okw, tol = {}, {}, TOL
    if opt == "unweighted":
        kw["apply_weights"] = okw["apply_weights"] = False
    elif opt == "band_mask":
        kw["band_mask"] = okw["band_mask"] = True
    elif opt == "gauss16":
        kw["window"] = ("gauss", 16)
        tol = 1e-4                      # Gaussian w = 16 interpolation error ~ 3e-8 per axis, times FP32
    elif opt == "kb8":
        kw["window"] = ("kb", 8)
        tol = 1e-4                      # KB w = 8 interpolation error ~ 2e-7
    want = oracle.forward(problem(case, **okw), case["g"])
    got = gpu_forward(nd, case, **kw)
    check(got, want, tol)


def test_forward_no_sensors(nd):
    case = inputs.small_case(16, 16, 16, 0, 32, seed=12)
    plan = nd.plan_from_config(case)
    out = plan.forward(torch.zeros((0, 32), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
    plan.close()


def test_forward_is_linear_and_repeatable(nd):
    case = inputs.small_case(16, 16, 32, 50, 64, seed=13)
    plan = nd.plan_from_config(case)
    g = torch.as_tensor(case["g"], dtype=torch.float32, device="cuda")
    a = plan.forward(g).clone()
    b = plan.forward(2.0 * g)
    c = plan.forward(g)
    torch.cuda.synchronize()
    assert rel_l2((b / 2).cpu().numpy(), a.cpu().numpy()) < 1e-6
    assert rel_l2(c.cpu().numpy(), a.cpu().numpy()) < 1e-6
    plan.close()


def test_set_positions_matches_fresh_plan(nd):
    case = inputs.small_case(16, 16, 32, 40, 64, seed=14)
    plan = nd.plan_from_config(case)
    xy2 = case["sensor_xy"] * 0.9 + 1e-5
    plan.set_positions(xy2)
    g = torch.as_tensor(case["g"], dtype=torch.float32, device="cuda")
    a = plan.forward(g).cpu().numpy()
    case2 = dict(case, sensor_xy=xy2)
    want = oracle.forward(problem(case2), case["g"])
    check(a, want, TOL)
    plan.close()


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_forward_host_matches_device_call(nd, pinned):
    """nedner_forward_host (host buffers uploaded on several copy streams, the
    last stage run per block of depth planes, each downloaded as it is written)
    gives the device call's result on the C2 geometry."""
    case = inputs.make_config(1, with_data=False)
    rng = np.random.default_rng(77)
    g = rng.standard_normal((case["sensor_xy"].shape[0], case["Nt"])).astype(np.float32)
    plan = nd.plan_from_config(case)
    want = plan.forward(torch.as_tensor(g, device="cuda")).cpu().numpy()
    gh = torch.as_tensor(g)
    out = torch.empty((case["nz"], case["ny"], case["nx"]), dtype=torch.float32)
    if pinned:
        gh, out = gh.pin_memory(), out.pin_memory()
    for _ in range(2):                                     # the first call sets up, the second reuses
        out.zero_()
        plan.forward_host(gh, out=out)
        torch.cuda.synchronize()
        assert np.array_equal(out.numpy(), want)
    plan.close()


def test_forward_host_small_and_ragged(nd):
    """Host-buffer call on a small case (fewer depth planes than copy streams would split evenly), against the oracle."""
    case = inputs.small_case(16, 16, 32, 61, 64, seed=9, layout="disc")
    g = np.asarray(case["g"], dtype=np.float32)
    plan = nd.plan_from_config(case)
    out = plan.forward_host(torch.as_tensor(g).pin_memory())
    torch.cuda.synchronize()
    plan.close()
    check(out.numpy(), oracle.forward(problem(case), g), TOL)


def test_forward_streams_in_time_chunks_under_a_workspace_limit(nd):
    """Under a workspace limit the split stage (a) runs in chunks of time
    samples (the oversampled grid is held for one chunk at a time) instead of
    failing.  Each time sample's arithmetic is the same in any chunking, so the
    result equals the unlimited plan's bit for bit, and the oracle's."""
    case = inputs.make_config(1, with_data=False)           # 64x64 sensors, Nt 512, 128x128x256
    rng = np.random.default_rng(78)
    g = rng.standard_normal((case["sensor_xy"].shape[0], case["Nt"])).astype(np.float32)
    full = nd.plan_from_config(case)
    lim = nd.plan_from_config(case, max_workspace_bytes=150 << 20)
    assert lim.workspace_bytes <= 150 << 20 < full.workspace_bytes
    x = torch.as_tensor(g, device="cuda")
    a = full.forward(x).cpu().numpy()
    b = lim.forward(x).cpu().numpy()
    full.close(); lim.close()
    assert np.array_equal(a, b)
    small = inputs.small_case(32, 32, 32, 300, 256, seed=79, layout="disc")
    plan = nd.plan_from_config(small, max_workspace_bytes=6 << 20)          # two chunks of 128 samples
    got = plan.forward(torch.as_tensor(small["g"], dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    check(got, oracle.forward(problem(small), small["g"]), TOL)
