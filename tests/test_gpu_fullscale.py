"""Parity at full workload size with the workloads' own dense data (balls +
20 dB noise), checked against the FP64 oracle on seeded samples that it can
compute one by one.

- Workload 3 (16384 scattered sensors, Nt 2048, 256 x 256 x 512 voxels):
  * stage (a) alone, nedner_ned_stage, on about 1 % of the half-lattice lines
    (a product set of jx in 0..nx/2 and jy in -ny/2..ny/2), all 2048 samples;
  * the whole reconstruction: the spectrum of the GPU's p0 on about 1 % of
    the lateral lines (no Nyquist index) at every depth frequency, against
    the oracle's direct sums there (p0 is the real part of an inverse DFT of a
    Hermitian spectrum, so its DFT gives that spectrum back exactly);
  * nedner_adjoint and nedner_grad_positions on a volume whose spectrum lives
    on 8 x 8 lateral lines (every depth frequency), for 256 seeded sensors:
    the oracle sums only over those lines, which is exact for such a volume.
- Workload 5 (128 x 128 tensor-grid sensors, Nt 2048, 256 x 256 x 512) in the
  FP32 NUFFT and both tensor-core precision modes (BF16 and FP16 split
  GEMMs): the sampled spectrum of the whole reconstruction, so every pass of
  512 time samples sees dense data.

Tolerances as in the other parity tests: rel-L2 1e-5 (FP32 path), 1e-4 for the
position gradient, 3e-5 for the BF16 split GEMMs (1e-5 for FP16); max-abs is reported beside.
"""
import numpy as np
import pytest

import bench
import oracle
from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5
TOL_GRAD = 1e-4
TOL_BF16 = 3e-5


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


@pytest.fixture(scope="module")
def c3():
    return inputs.make_config(2)


@pytest.fixture(scope="module")
def c5():
    return inputs.make_config(4)


def test_c3_ned_stage_dense_data_sampled_lines(nd, c3):
    rng = np.random.default_rng(301)
    ax = np.sort(rng.choice(c3["nx"] // 2 + 1, size=13, replace=False))              # jx = a
    by = np.sort(rng.choice(c3["ny"] + 1, size=26, replace=False))                   # jy = b - ny/2
    plan = nd.plan_from_config(c3)
    g = torch.as_tensor(np.asarray(c3["g"], dtype=np.float32), device="cuda")
    Gh = plan.ned_stage(g)
    got = Gh[torch.as_tensor(ax, device="cuda")][:, torch.as_tensor(by, device="cuda")].cpu().numpy()
    del Gh
    plan.close()
    want = oracle.ned(bench.oracle_problem(c3), c3["g"], ax, by - c3["ny"] // 2)     # (13, 26, 2048)
    check(got, want, TOL)


def _sampled_forward(nd, cfg, mode, seed, tol):
    plan = nd.plan_from_config(cfg, ned_mode=mode)
    g = torch.as_tensor(np.asarray(cfg["g"], dtype=np.float32), device="cuda")
    p0 = plan.forward(g).cpu().numpy().astype(np.float64)
    plan.close()
    jx, jy, F, _, _ = bench.oracle_sample(cfg, 0.01, seed)
    got = bench.spectrum_of_volume(p0, jx, jy)
    check(got[:, :, 1:], F[:, :, 1:], tol)


def test_c3_forward_dense_data_sampled_spectrum(nd, c3):
    _sampled_forward(nd, c3, "nufft", 302, TOL)


def test_c5_tensor_bf16_forward_dense_data_sampled_spectrum(nd, c5):
    _sampled_forward(nd, c5, "tensor_bf16", 501, TOL_BF16)


def test_c5_tensor_fp16_forward_dense_data_sampled_spectrum(nd, c5):
    _sampled_forward(nd, c5, "tensor_fp16", 503, TOL)


def test_c5_nufft_forward_dense_data_sampled_spectrum(nd, c5):
    _sampled_forward(nd, c5, "nufft", 502, TOL)


def _band_volume(cfg, seed):
    """A real volume whose spectrum lives on the lines jx x jy (random complex
    values at every depth frequency) and their mirrors; returns the volume and
    the product set that holds both."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    jx = rng.choice(np.arange(1, nx // 2), size=4, replace=False) * rng.choice([-1, 1], size=4)
    jy = rng.choice(np.arange(1, ny // 2), size=4, replace=False) * rng.choice([-1, 1], size=4)
    B = np.zeros((nz, ny, nx), dtype=np.complex128)
    for a in jx:
        for b in jy:
            B[:, b % ny, a % nx] = rng.standard_normal(nz) + 1j * rng.standard_normal(nz)
    p = np.real(np.fft.ifftn(B)) * (nx * ny * nz) ** 0.5
    return p, np.concatenate([jx, -jx]), np.concatenate([jy, -jy])


def test_c3_adjoint_full_size_sampled_sensors(nd, c3):
    p, lx, ly = _band_volume(c3, 303)
    plan = nd.plan_from_config(c3)
    got = plan.adjoint(torch.as_tensor(p, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    sens = np.sort(np.random.default_rng(304).choice(c3["sensor_xy"].shape[0], size=256, replace=False))
    want = oracle.adjoint(bench.oracle_problem(c3), p, lx, ly, sens)
    check(got[sens], want, TOL)


def test_c3_position_gradient_full_size_sampled_sensors(nd, c3):
    p, lx, ly = _band_volume(c3, 305)
    plan = nd.plan_from_config(c3)
    g = torch.as_tensor(np.asarray(c3["g"], dtype=np.float32), device="cuda")
    got = plan.grad_positions(g, torch.as_tensor(p, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    sens = np.sort(np.random.default_rng(306).choice(c3["sensor_xy"].shape[0], size=256, replace=False))
    want = oracle.grad_positions(bench.oracle_problem(c3), np.asarray(c3["g"], dtype=np.float32), p, lx, ly, sens)
    check(got[sens], want, TOL_GRAD)
