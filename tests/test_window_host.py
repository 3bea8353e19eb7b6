"""The register-window helpers of the spread (csrc/spread_window.cuh) and of
the transposed gather (csrc/gather_window.cuh) compiled with g++ and run on
the host (tests/host_fft/window_harness.cpp), against direct FP64 sums.

Spread: every lane sweeps the entries of a column segment [c0, c1) in
first-column order; each column of the segment must hold
sum_e tap_e[col - bx4_e] g_e once the sweep ends, and no column outside the
segment may be written.  Gather (its transpose): every entry of a run gets
sum_k tap[k] r[(bx4 + k) mod Lx] for two tap sets.  Both lane layouts (one
and two time samples per lane), every tap count WT the kernels instantiate,
segments at the row's ends (entries repeated at bx - Lx), empty segments,
and runs that wrap around x = Lx.  Also the spread stage's output step
(the folded last x-FFT pass and the split of packed time-sample pairs)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1510_01078_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("host_window") / "libwin.so")
    cmd = [gxx, "-std=c++20", "-O2", "-shared", "-fPIC", "-Wno-unknown-pragmas", "-I", os.path.join(HERE, "host_fft"),
           "-I", CSRC, os.path.join(HERE, "host_fft", "window_harness.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    h = ctypes.CDLL(out)
    I, F = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)
    h.host_sweep.argtypes = [ctypes.c_int] * 7 + [I, F, F, F]
    h.host_sweep.restype = ctypes.c_int
    return h


def taps_for(w):
    return ((w + 3) + 3) // 4 * 4          # w taps after up to 3 leading zeros, rounded up to 4


def entries(rng, w, WT, Lx, c0, c1, n):
    """Entries reaching into [c0, c1): first column bx in [c0 - w + 1, c1), sorted;
    bx < 0 stands for an entry wrapped around x = Lx."""
    lo = c0 - w + 1
    bx = np.sort(rng.integers(lo, max(lo + 1, c1), n)) if n else np.zeros(0, np.int64)
    bx4 = bx & ~3
    taps = np.zeros((n, WT), np.float32)
    for e in range(n):
        off = int(bx[e] - bx4[e])
        taps[e, off:off + w] = rng.uniform(0.1, 1.0, w)
    return bx4.astype(np.int32), taps


def reference(bx4, taps, g, Lx, c0, c1):
    lanes = g.shape[1]
    Z = np.zeros((Lx, lanes))
    for e in range(len(bx4)):
        for k in range(taps.shape[1]):
            col = int(bx4[e]) + k
            if c0 <= col < c1:
                Z[col] += float(taps[e, k]) * g[e].astype(np.float64)
    return Z


def sweep(lib, two, WT, Lx, C, c0, c1, bx4, taps, g):
    I, F = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)
    lanes = 64 if two else C
    out = np.empty((Lx, lanes), np.float32)
    bx4 = np.ascontiguousarray(bx4, np.int32)
    taps = np.ascontiguousarray(taps, np.float32)
    g = np.ascontiguousarray(g, np.float32)
    r = lib.host_sweep(int(two), WT, Lx, C, c0, c1, len(bx4), bx4.ctypes.data_as(I), taps.ctypes.data_as(F),
                       g.ctypes.data_as(F), out.ctypes.data_as(F))
    assert r == 0
    return out


def segments(Lx):
    yield 0, Lx // 4                       # starts at the row's first column (wrapped entries)
    yield Lx // 4, Lx // 4 + 37            # interior, ragged width
    yield 3 * Lx // 4, Lx                  # ends at the row's last column
    yield 5, 6                             # one column
    yield 10, 10                           # empty


@pytest.mark.parametrize("two", [True, False], ids=["two_per_lane", "one_per_lane"])
@pytest.mark.parametrize("w", [4, 6, 8, 10, 12, 14, 16])
def test_window_sweep_matches_direct_accumulation(lib, two, w):
    WT = taps_for(w)
    rng = np.random.default_rng(100 * w + two)
    for Lx in (64, 512):
        for C in ((64,) if two else (2, 8, 32)):
            lanes = 64 if two else C
            for c0, c1 in segments(Lx):
                for n in (0, 1, 7, 60):
                    bx4, taps = entries(rng, w, WT, Lx, c0, c1, n)
                    g = rng.standard_normal((n, lanes)).astype(np.float32)
                    got = sweep(lib, two, WT, Lx, C, c0, c1, bx4, taps, g)
                    inside = got[c0:c1]
                    assert np.isfinite(inside).all(), (w, Lx, C, c0, c1, n)
                    want = reference(bx4, taps, g, Lx, c0, c1)[c0:c1]
                    scale = max(1.0, float(np.abs(want).max()) if want.size else 1.0)
                    assert float(np.abs(inside - want).max(initial=0.0)) <= 1e-5 * scale, (w, Lx, C, c0, c1, n)
                    outside = np.concatenate([got[:c0], got[c1:]])
                    assert np.isnan(outside).all(), (w, Lx, C, c0, c1, n)


def gather(lib, two, WT, Lx, C, bx4, ta, tb, row):
    I, F = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)
    lanes = 64 if two else C
    n = len(bx4)
    oa = np.empty((n, lanes), np.float32)
    ob = np.empty((n, lanes), np.float32)
    bx4 = np.ascontiguousarray(bx4, np.int32)
    ta = np.ascontiguousarray(ta, np.float32)
    tb = np.ascontiguousarray(tb, np.float32)
    row = np.ascontiguousarray(row, np.float32)
    lib.host_gather.argtypes = [ctypes.c_int] * 5 + [I, F, F, F, F, F]
    r = lib.host_gather(int(two), WT, Lx, C, n, bx4.ctypes.data_as(I), ta.ctypes.data_as(F), tb.ctypes.data_as(F),
                        row.ctypes.data_as(F), oa.ctypes.data_as(F), ob.ctypes.data_as(F))
    assert r == 0
    return oa, ob


@pytest.mark.parametrize("two", [True, False], ids=["two_per_lane", "one_per_lane"])
@pytest.mark.parametrize("w", [4, 6, 8, 10, 12, 14, 16])
def test_gather_window_matches_direct_sums(lib, two, w):
    WT = taps_for(w)
    rng = np.random.default_rng(200 * w + two)
    for Lx in (64, 512):
        for C in ((64,) if two else (2, 16, 32)):
            lanes = 64 if two else C
            row = rng.standard_normal((Lx, lanes)).astype(np.float32)
            for n in (1, 5, 80):
                # a run of a row's entries, first columns sorted in [0, Lx); taps past
                # Lx - 1 read the row modulo Lx
                bx = np.sort(rng.integers(0, Lx, n))
                bx4 = (bx & ~3).astype(np.int32)
                ta = np.zeros((n, WT), np.float32)
                tb = np.zeros((n, WT), np.float32)
                for e in range(n):
                    off = int(bx[e] - bx4[e])
                    ta[e, off:off + w] = rng.uniform(0.1, 1.0, w)
                    tb[e, off:off + w] = rng.uniform(-1.0, 1.0, w)
                oa, ob = gather(lib, two, WT, Lx, C, bx4, ta, tb, row)
                cols = (bx4[:, None] + np.arange(WT)[None, :]) % Lx
                r64 = row.astype(np.float64)
                wa = np.einsum("ek,ekt->et", ta.astype(np.float64), r64[cols])
                wb = np.einsum("ek,ekt->et", tb.astype(np.float64), r64[cols])
                assert np.isfinite(oa).all() and np.isfinite(ob).all()
                assert float(np.abs(oa - wa).max()) <= 1e-5 * max(1.0, float(np.abs(wa).max())), (w, Lx, C, n)
                assert float(np.abs(ob - wb).max()) <= 1e-5 * max(1.0, float(np.abs(wb).max())), (w, Lx, C, n)


@pytest.mark.parametrize("Lx,nb", [(64, 4), (256, 32), (512, 32), (512, 1), (4096, 2)])
@pytest.mark.parametrize("fold", [False, True], ids=["last_pass_done", "last_pass_folded"])
def test_spread_output_step(lib, Lx, nb, fold):
    """The spread stage's output step (spread_output in csrc/spread_window.cuh):
    from the x-transformed row of packed time-sample pairs z = x[2b] + i x[2b+1]
    (with fold, the row before its last radix-2 pass, s[k] = (X[k] + X[k+N/2])/2,
    s[k+N/2] = (X[k] - X[k+N/2]) / (2 w^k)), it must write, for jx = 0..Lx/4, the
    FFT of each real time sample's row times the deconvolution factor."""
    F = ctypes.POINTER(ctypes.c_float)
    lib.host_spread_output.argtypes = [ctypes.c_int] * 3 + [F, F, F]
    rng = np.random.default_rng(Lx + nb + fold)
    x = rng.standard_normal((Lx, 2 * nb))
    X = np.fft.fft(x[:, 0::2] + 1j * x[:, 1::2], axis=0)
    if fold:
        H = Lx // 2
        w = np.exp(-2j * np.pi * np.arange(H)[:, None] / Lx)
        X = np.concatenate([(X[:H] + X[H:]) / 2, (X[:H] - X[H:]) / (2 * w)])
    Zin = np.empty((Lx, nb, 2), np.float32)
    Zin[..., 0], Zin[..., 1] = X.real, X.imag
    nxh = Lx // 4 + 1
    dec = rng.uniform(0.5, 2.0, nxh).astype(np.float32)
    out = np.empty((nxh, 2 * nb, 2), np.float32)
    assert lib.host_spread_output(Lx, nb, int(fold), Zin.ctypes.data_as(F), dec.ctypes.data_as(F),
                                  out.ctypes.data_as(F)) == 0
    got = out[..., 0] + 1j * out[..., 1]
    want = np.fft.fft(x, axis=0)[:nxh] * dec[:, None]
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-6


@pytest.mark.parametrize("w", [4, 6, 8, 10, 12, 14, 16])
def test_block_spread_accumulates_exact_taps(lib, w):
    """The block spread's accumulation (block_taps16, the plan's table entry,
    and block_entry16 in csrc/spread_window.cuh):
    a warp's 16-column block [c0, c0 + 16) gets, from every entry whose w taps
    start anywhere in [c0 - w + 1, c0 + 15], exactly the taps that land in the
    block (all w of them for entries inside, the overlapping part at both
    edges), against a direct FP64 sum; also for a block at a negative first
    column (the second copy of a wrapped entry) and an empty entry list."""
    I, F = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)
    lib.host_block_sweep.argtypes = [ctypes.c_int] * 3 + [I, F, F, F]
    PW = (w + 3) // 4 * 4
    rng = np.random.default_rng(100 + w)
    for c0, n in [(0, 60), (496, 40), (-16, 9), (64, 0), (240, 200)]:
        bx = np.sort(rng.integers(c0 - w + 1, c0 + 16, n)).astype(np.int32)
        bx[:min(n, 2)] = c0 - w + 1                        # entries touching the block with one tap
        bx[-min(n, 2):] = c0 + 15 if n else bx[-min(n, 2):]
        taps = np.zeros((n, PW), np.float32)
        taps[:, :w] = rng.uniform(0.1, 1.0, (n, w))
        g = rng.standard_normal((n, 64)).astype(np.float32)
        out = np.empty((16, 64), np.float32)
        assert lib.host_block_sweep(w, c0, n, bx.ctypes.data_as(I), taps.ctypes.data_as(F), g.ctypes.data_as(F),
                                    out.ctypes.data_as(F)) == 0
        want = np.zeros((16, 64))
        for e in range(n):
            for k in range(w):
                col = int(bx[e]) + k - c0
                if 0 <= col < 16:
                    want[col] += float(taps[e, k]) * g[e].astype(np.float64)
        np.testing.assert_allclose(out, want, rtol=0, atol=2e-5 * max(1.0, np.abs(want).max()))
