"""The NER value evaluation (csrc/ner_eval.cuh: float-float nu, the w-tap
interpolation with the mirrored tap polynomials, the phase exp(-i pi nu))
compiled with g++ and run on the host (tests/host_fft/ner_harness.cpp), with
the plan's own tap polynomials (window.cpp):
  - nu_l = sign(l) sqrt(axy + az l^2) in float-float against FP64;
  - the NER values of one line against the direct sum of Eq. NER_NUFFT,
    F(nu) = sum_n G[n] exp(-2 pi i nu n / Nt), from the line's oversampled
    spectrum built here with numpy (centred, deconvolved, zero-padded to 2 Nt,
    FFT), for |nu| up to 1600 on a 4096-point grid, where single-float nu
    would lose the fractional grid offset."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1510_01078_gb300", "csrc")
F = ctypes.POINTER(ctypes.c_float)


def _compile(tmp_path_factory, name, sources, std="c++20"):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp(name) / ("lib%s.so" % name))
    cmd = [gxx, "-std=" + std, "-O2", "-shared", "-fPIC", "-Wno-unknown-pragmas", "-I", os.path.join(HERE, "host_fft"),
           "-I", CSRC] + sources + ["-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return ctypes.CDLL(out)


@pytest.fixture(scope="module")
def ner(tmp_path_factory):
    h = _compile(tmp_path_factory, "ner", [os.path.join(CSRC, "window.cpp"), os.path.join(HERE, "host_fft", "ner_harness.cpp")])
    h.host_nu_abs.argtypes = [ctypes.c_double, ctypes.c_float, ctypes.c_float, ctypes.c_int, F, F]
    h.host_ner_values.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, ctypes.c_float, ctypes.c_float] + \
        [ctypes.c_int] * 3 + [F, F]
    h.host_ner_values.restype = ctypes.c_int
    return h


@pytest.fixture(scope="module")
def wm(tmp_path_factory):
    h = _compile(tmp_path_factory, "wm", [os.path.join(CSRC, "window.cpp"),
                                          os.path.join(HERE, "host_fft", "window_math_harness.cpp")], std="c++17")
    h.hw_phihat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    h.hw_phihat.restype = ctypes.c_double
    return h


def ff(x):
    hi = np.float32(x)
    return hi, np.float32(x - float(hi))


def test_float_float_nu(ner):
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(2000):
        az = float(rng.uniform(0.2, 3.0))
        axy = float(rng.uniform(0.0, 4e6))
        l = int(rng.integers(-1024, 1025))
        hi, lo = ff(axy)
        az_hi, az_lo = ff(az)
        a, b = ctypes.c_float(), ctypes.c_float()
        ner.host_nu_abs(az, hi, lo, l, a, b)
        exact = np.sqrt((float(hi) + float(lo)) + (float(az_hi) + float(az_lo)) * l * l)
        worst = max(worst, abs((a.value + b.value) - exact) / max(exact, 1e-30))
    assert worst <= 1e-13, worst


@pytest.mark.parametrize("Nt,axy,w,kind", [(512, 37.3, 12, 0), (2048, 3.9e5, 12, 0), (2048, 2.5e6, 12, 0),
                                           (512, 100.0, 8, 0), (512, 100.0, 16, 0), (1024, 7e4, 16, 1),
                                           (64, 3.0, 12, 0)])
def test_ner_values_match_the_direct_sum(ner, wm, Nt, axy, w, kind):
    rng = np.random.default_rng(Nt + w)
    Lt = 2 * Nt
    G = rng.standard_normal(Nt) + 1j * rng.standard_normal(Nt)
    n = np.arange(Nt)
    deconv = np.array([1.0 / wm.hw_phihat(kind, w, 2.0, (k - Nt / 2) / Lt) for k in n])
    LA = np.zeros(Lt, complex)
    LA[(n - Nt // 2) % Lt] = G * deconv                  # centred, deconvolved, zero-padded
    B = np.fft.fft(LA)
    Bf = np.empty(2 * Lt, np.float32)
    Bf[0::2], Bf[1::2] = B.real, B.imag
    nz = 512
    l0, nl = -nz // 2, nz + 1
    out = np.empty(2 * nl, np.float32)
    hi, lo = ff(axy)
    assert ner.host_ner_values(kind, w, Nt, 1.0, hi, lo, 0, l0, nl, Bf.ctypes.data_as(F), out.ctypes.data_as(F)) == 0
    got = out[0::2].astype(np.float64) + 1j * out[1::2]
    l = np.arange(l0, l0 + nl)
    nu = np.sign(l) * np.sqrt((float(hi) + float(lo)) + l * l.astype(np.float64))   # nu(l = 0) = 0
    want = np.exp(-2j * np.pi * np.outer(nu, n) / Nt) @ G
    tol = 1e-6 if kind == 0 else 1e-5
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= tol
    assert float(np.abs(got - want).max()) <= 1e-7 * float(np.abs(G).sum()) * (1 if kind == 0 else 10)
