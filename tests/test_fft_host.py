"""The device FFT engine (csrc/fft.cuh, block_fft_ip) compiled with g++ and
run on CPU threads (one std::thread per CUDA thread, __syncthreads as a
barrier; tests/host_fft), against numpy's FFT, for every (values per thread,
threads) pair the kernels launch it with and every power-of-two length they
use.  Covers the in-place padded passes, the last radix-2 pass left to the
caller (skip_r2), and the zero-padded first pass, whose skipped points are
filled with NaN here to show they are never read.  No GPU needed."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1510_01078_gb300", "csrc")
TOL = 1e-6            # FP32 passes, up to 13 radix stages; measured <= 2e-7

# (values per thread, threads): the spread (32, 256/512; 16/32, 256), the
# y-FFT (16/32, 256), the NER (16, 256/512), the inverse image FFTs (16, 128),
# the transposed gather (16, 256; 32, 256/512)
CONFIGS = [(16, 128), (16, 256), (16, 512), (32, 256), (32, 512)]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("host_fft") / "libhostfft.so")
    cmd = [gxx, "-std=c++20", "-O2", "-pthread", "-shared", "-fPIC", "-Wno-unknown-pragmas",
           "-I", os.path.join(HERE, "host_fft"), "-I", CSRC, os.path.join(HERE, "host_fft", "harness.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    h = ctypes.CDLL(out)
    F = ctypes.POINTER(ctypes.c_float)
    h.host_block_fft.argtypes = [ctypes.c_int] * 7 + [F, F]
    h.host_block_fft.restype = ctypes.c_int
    return h


def run(lib, x, d, per, nt, skip_r2=False, zp=False):
    N, nb = x.shape
    xi = np.empty((N, nb, 2), np.float32)
    xi[..., 0], xi[..., 1] = x.real, x.imag
    out = np.empty_like(xi)
    F = ctypes.POINTER(ctypes.c_float)
    r = lib.host_block_fft(N, nb, d, per, nt, int(skip_r2), int(zp), xi.ctypes.data_as(F), out.ctypes.data_as(F))
    assert r == 0, (N, nb, per, nt)
    return out[..., 0].astype(np.float64) + 1j * out[..., 1]


def data(N, nb, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, nb)) + 1j * rng.standard_normal((N, nb))


def dft(x, d):
    return np.fft.fft(x, axis=0) if d < 0 else np.fft.ifft(x, axis=0) * x.shape[0]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cases():
    for per, nt in CONFIGS:
        cap = per * nt
        for ln in range(1, 14):
            N = 1 << ln
            if N > cap:
                break
            widest = cap // N
            for nb in sorted({1, min(widest, 4), widest}):
                yield per, nt, N, nb


@pytest.mark.parametrize("per,nt", CONFIGS, ids=["per%d_nt%d" % c for c in CONFIGS])
def test_block_fft_matches_numpy(lib, per, nt):
    worst = 0.0
    for p, t, N, nb in cases():
        if (p, t) != (per, nt):
            continue
        x = data(N, nb, N * 31 + nb)
        for d in (-1, 1):
            e = rel(run(lib, x, d, per, nt), dft(x, d))
            worst = max(worst, e)
            assert e <= TOL, (N, nb, d, e)
    assert worst > 0.0


@pytest.mark.parametrize("N,nb,per,nt", [(32, 32, 16, 128), (512, 32, 32, 512), (512, 8, 16, 256),
                                         (8192, 1, 16, 512)])
def test_last_radix2_pass_left_to_the_caller(lib, N, nb, per, nt):
    """skip_r2 (log2 N = 1 mod 4): X[k] = s[k] + w^k s[k + N/2],
    X[k + N/2] = s[k] - w^k s[k + N/2], w = exp(dir 2 pi i / N)."""
    x = data(N, nb, N + nb)
    for d in (-1, 1):
        s = run(lib, x, d, per, nt, skip_r2=True)
        k = np.arange(N // 2)[:, None]
        w = np.exp(d * 2j * np.pi * k / N)
        X = np.concatenate([s[:N // 2] + w * s[N // 2:], s[:N // 2] - w * s[N // 2:]])
        assert rel(X, dft(x, d)) <= TOL


@pytest.mark.parametrize("N,nb,per,nt", [(16, 1, 16, 256), (64, 4, 16, 256), (1024, 4, 16, 256), (4096, 1, 16, 256),
                                         (8192, 1, 16, 512), (2048, 2, 16, 256)])
def test_zero_padded_first_pass(lib, N, nb, per, nt):
    """Points N/4 <= p < 3N/4 are zero by contract and hold NaN in the buffer:
    a finite, correct result shows the first pass never reads them."""
    x = data(N, nb, 3 * N + nb)
    x[N // 4:3 * N // 4] = 0
    for d in (-1, 1):
        y = run(lib, x, d, per, nt, zp=True)
        assert np.isfinite(y).all()
        assert rel(y, dft(x, d)) <= TOL


@pytest.mark.parametrize("N", [4, 8, 16, 256, 512, 4096])
def test_complex_to_real_pairs(lib, N):
    """c2r_pair (the x complex-to-real stage's input): with Z formed from the
    half spectrum X[0..N/2] pair by pair, z = IFFT_{N/2}(Z) interleaved
    (x[2p] = Re z[p], x[2p+1] = Im z[p]) equals N irfft(X), which likewise drops
    the imaginary parts of X[0] and X[N/2]."""
    F = ctypes.POINTER(ctypes.c_float)
    lib.host_c2r_pairs.argtypes = [ctypes.c_int, F, F]
    rng = np.random.default_rng(N)
    X = rng.standard_normal(N // 2 + 1) + 1j * rng.standard_normal(N // 2 + 1)
    Xi = np.empty((N // 2 + 1, 2), np.float32)
    Xi[:, 0], Xi[:, 1] = X.real, X.imag
    Z = np.empty((N // 2, 2), np.float32)
    assert lib.host_c2r_pairs(N, Xi.ctypes.data_as(F), Z.ctypes.data_as(F)) == 0
    z = np.fft.ifft(Z[:, 0] + 1j * Z[:, 1]) * (N // 2)
    x = np.empty(N)
    x[0::2], x[1::2] = z.real, z.imag
    want = np.fft.irfft(X, n=N) * N
    assert np.linalg.norm(x - want) / np.linalg.norm(want) <= 1e-6


@pytest.mark.parametrize("N", [4, 8, 16, 256, 512, 4096])
def test_real_to_complex_unpack(lib, N):
    """r2c_unpack (the transposed x stage): from Z = FFT_{N/2} of the packed real
    samples z[p] = x[2p] + i x[2p+1], X[0..N/2] equals numpy's rfft(x)."""
    F = ctypes.POINTER(ctypes.c_float)
    lib.host_r2c_unpack.argtypes = [ctypes.c_int, F, F]
    rng = np.random.default_rng(N + 1)
    x = rng.standard_normal(N)
    Z = np.fft.fft(x[0::2] + 1j * x[1::2])
    Zi = np.empty((N // 2, 2), np.float32)
    Zi[:, 0], Zi[:, 1] = Z.real, Z.imag
    out = np.empty((N // 2 + 1, 2), np.float32)
    assert lib.host_r2c_unpack(N, Zi.ctypes.data_as(F), out.ctypes.data_as(F)) == 0
    want = np.fft.rfft(x)
    got = out[:, 0] + 1j * out[:, 1]
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-6
