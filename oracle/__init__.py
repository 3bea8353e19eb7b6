"""FP64 CPU oracle for the NEDNER reconstruction (arXiv:1510.01078).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the heavy sums live in
``nedner_oracle.c`` (plain C, FP64, OpenMP), the rest is numpy.

What it computes (Sec. 2, Eq. exact and Eq. disc_rec, written in physical
units; sound speed c, the paper sets c = 1):

    X = nx dx, Y = ny dy, Z = nz dz
    j = (jx, jy) in G_x = {-nx/2..nx/2-1} x {-ny/2..ny/2-1},  l in {-nz/2..nz/2-1}
    G[j, n]  = sum_m w_m g[m, n] exp(-2 pi i (jx x_m / X + jy y_m / Y))      NED sum
    nu[j, l] = sign(l) c Nt dt sqrt((jx/X)^2 + (jy/Y)^2 + (l/Z)^2)          kappa map
    F[j, l]  = coef[j, l] sum_{n<Nt} G[j, n] exp(-2 pi i nu[j, l] n / Nt)    NER sum
    p0[q]    = Re (1/(nx ny nz)) sum_{j,l} F[j, l] exp(+2 pi i (jx (qx - nx/2)/nx
                                              + jy (qy - ny/2)/ny + l qz/nz))

with w_m = h_m / (dx dy) and coef = W s, W = 2|l/Z| / |k| (the factor 2 l / kappa
of Eq. exact), W(0, 0) = 2, W(j != 0, 0) = 0, s = c dt / dz (the Riemann-sum
step of the temporal integral in depth units).  With ``apply_weights=False``
w_m = 1 and coef = 1.  With ``band_mask=True`` coef is zeroed where nu falls
outside the half-open band [-Nt/2, Nt/2).

The voxel (qx, qy, qz) sits at x = (qx - nx/2) dx, y = (qy - ny/2) dy, z = qz dz.
The final uniform inverse DFT uses numpy's FFT as a library step.

Every function is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nedner_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libnedner_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C core with gcc (FP64, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64, I, D = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_ned.argtypes = [I64, P, P, I, P, D, D, I, P, I, P, P, I]
        lib.orc_ned.restype = I
        lib.orc_ner.argtypes = [I64, I, I, P, P, I, P, P, I]
        lib.orc_ner.restype = None
        lib.orc_ner_adj.argtypes = [I64, I, P, I, P, P, I]
        lib.orc_ner_adj.restype = None
        lib.orc_ned_adj.argtypes = [I64, P, P, I, D, D, I, P, I, P, P, P, I]
        lib.orc_ned_adj.restype = I
        lib.orc_ned_grad.argtypes = [I64, P, P, I, P, D, D, I, P, I, P, P, P, I]
        lib.orc_ned_grad.restype = I
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _nthreads() -> int:
    return int(os.environ.get("NEDNER_ORACLE_THREADS", "0"))


# --------------------------------------------------------------------------
# problem description
# --------------------------------------------------------------------------
@dataclass
class Problem:
    """Geometry of one reconstruction (Sec. 2).

    sensor_xy: (M, 2) sensor positions in metres, inside (-X/2, X/2)^2.
    h: (M,) detector areas h_m (Eq. disc_rec); None means X*Y/M each.
    Nt, dt: number and spacing of time samples, t_n = n dt, n = 0..Nt-1.
    c: sound speed.  nx, ny, nz and dx, dy, dz: output grid.
    """
    sensor_xy: np.ndarray
    Nt: int
    dt: float
    c: float
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    h: Optional[np.ndarray] = None
    apply_weights: bool = True
    band_mask: bool = False

    @property
    def M(self) -> int:
        return int(np.asarray(self.sensor_xy).shape[0])

    @property
    def X(self) -> float:
        return self.nx * self.dx

    @property
    def Y(self) -> float:
        return self.ny * self.dy

    @property
    def Z(self) -> float:
        return self.nz * self.dz

    def areas(self) -> np.ndarray:
        if self.h is None:
            return np.full(self.M, self.X * self.Y / max(self.M, 1))
        return np.asarray(self.h, dtype=np.float64)

    def sensor_factor(self) -> np.ndarray:
        """w_m = h_m / Delta_x^{d-1} of Eq. disc_rec (ones when unweighted)."""
        if not self.apply_weights:
            return np.ones(self.M)
        return self.areas() / (self.dx * self.dy)


def index_set(n: int) -> np.ndarray:
    """G = {-n/2, ..., n/2 - 1} (Sec. 2, the grids G_x and G_Ky)."""
    return np.arange(-(n // 2), n - n // 2, dtype=np.int64)


# --------------------------------------------------------------------------
# the kappa mapping and the Jacobian factor (Sec. 2, Eq. exact / Eq. equiv_rec)
# --------------------------------------------------------------------------
def nu(pr: Problem, jx, jy, l) -> np.ndarray:
    """Temporal frequency index nu = sign(l) c Nt dt |k| of the wavenumber
    k = (jx/X, jy/Y, l/Z); the kappa_{j,l} = sign(l) sqrt(j^2 + l^2) of
    Eq. equiv_rec written in physical units (bins of the length-Nt DFT)."""
    jx = np.asarray(jx, dtype=np.float64)
    jy = np.asarray(jy, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    k = np.sqrt((jx / pr.X) ** 2 + (jy / pr.Y) ** 2 + (l / pr.Z) ** 2)
    return np.sign(l) * pr.c * pr.Nt * pr.dt * k


def jacobian(pr: Problem, jx, jy, l) -> np.ndarray:
    """W = 2 l / kappa of Eq. exact, i.e. 2 |l/Z| / |k|.  At l = 0 it is 0/0:
    W(j != 0, 0) = 0 (the limit kz -> 0 at fixed lateral k) and W(0, 0) = 2
    (the limit along kz)."""
    jx = np.asarray(jx, dtype=np.float64)
    jy = np.asarray(jy, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    jx, jy, l = np.broadcast_arrays(jx, jy, l)
    k = np.sqrt((jx / pr.X) ** 2 + (jy / pr.Y) ** 2 + (l / pr.Z) ** 2)
    W = np.zeros(k.shape)
    nz = k > 0
    W[nz] = 2.0 * np.abs(l[nz] / pr.Z) / k[nz]
    W[~nz] = 2.0
    return W


def coef(pr: Problem, jx, jy, l) -> np.ndarray:
    """Per-(j, l) factor of the NER sum: W * c dt / dz (or 1 unweighted), with
    the optional band mask."""
    jx, jy, l = np.broadcast_arrays(np.asarray(jx), np.asarray(jy), np.asarray(l))
    if pr.apply_weights:
        C = jacobian(pr, jx, jy, l) * (pr.c * pr.dt / pr.dz)
    else:
        C = np.ones(jx.shape)
    if pr.band_mask:
        v = nu(pr, jx, jy, l)
        keep = (v >= -pr.Nt / 2 - 1e-9) & (v < pr.Nt / 2 - 1e-9)
        C = np.where(keep, C, 0.0)
    return C


# --------------------------------------------------------------------------
# direct sums (C core)
# --------------------------------------------------------------------------
def ned(pr: Problem, g: np.ndarray, jx=None, jy=None) -> np.ndarray:
    """NED sum of Eq. disc_rec: G[a, b, n] for jx[a], jy[b] (default: G_x)."""
    jx = index_set(pr.nx) if jx is None else np.asarray(jx, dtype=np.int64)
    jy = index_set(pr.ny) if jy is None else np.asarray(jy, dtype=np.int64)
    xy = np.ascontiguousarray(pr.sensor_xy, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(pr.M, pr.Nt)
    w = np.ascontiguousarray(pr.sensor_factor(), dtype=np.float64)
    jx32 = np.ascontiguousarray(jx, dtype=np.int32)
    jy32 = np.ascontiguousarray(jy, dtype=np.int32)
    out = np.zeros((len(jx), len(jy), pr.Nt), dtype=np.complex128)
    rc = _load().orc_ned(pr.M, _p(xy), _p(w), pr.Nt, _p(g), pr.X, pr.Y,
                         len(jx32), _p(jx32), len(jy32), _p(jy32), _p(out), _nthreads())
    if rc != 0:
        raise MemoryError("orc_ned: allocation failed")
    return out


def ner(pr: Problem, G: np.ndarray, nus: np.ndarray, ns=None) -> np.ndarray:
    """NER sum of Eq. disc_rec: F[j, l] = sum_n G[j, n] exp(-2 pi i nu[j, l] n / Nt).
    With ``ns`` given, G's columns are the time samples ns (the others zero)."""
    nn = pr.Nt if ns is None else len(ns)
    G = np.ascontiguousarray(G, dtype=np.complex128).reshape(-1, nn)
    nus = np.ascontiguousarray(nus, dtype=np.float64).reshape(G.shape[0], -1)
    out = np.zeros(nus.shape, dtype=np.complex128)
    ns32 = None if ns is None else np.ascontiguousarray(ns, dtype=np.int32)
    _load().orc_ner(G.shape[0], pr.Nt, nn, None if ns32 is None else _p(ns32), _p(G), nus.shape[1],
                    _p(nus), _p(out), _nthreads())
    return out


def ner_adj(pr: Problem, P: np.ndarray, nus: np.ndarray) -> np.ndarray:
    """Conjugate transpose of ``ner``: T[j, n] = sum_l exp(+2 pi i nu n / Nt) P[j, l]."""
    P = np.ascontiguousarray(P, dtype=np.complex128).reshape(nus.shape)
    nus = np.ascontiguousarray(nus, dtype=np.float64)
    out = np.zeros((nus.shape[0], pr.Nt), dtype=np.complex128)
    _load().orc_ner_adj(nus.shape[0], pr.Nt, _p(P), nus.shape[1], _p(nus), _p(out), _nthreads())
    return out


# --------------------------------------------------------------------------
# the reconstruction R, its transpose and the sensor-position gradient
# --------------------------------------------------------------------------
def _grid_indices(pr: Problem):
    jx = index_set(pr.nx)
    jy = index_set(pr.ny)
    l = index_set(pr.nz)
    JX, JY, L = np.meshgrid(jx, jy, l, indexing="ij")
    return jx, jy, l, JX, JY, L


def spectrum(pr: Problem, g: np.ndarray, ns=None) -> np.ndarray:
    """F[jx, jy, l] over G_x x G_Ky: the right-hand side of Eq. disc_rec times
    the Riemann step (Sec. 2).  ``ns``: optional list of the time samples where
    g may be non-zero (g then has len(ns) columns); the sums skip the zeros."""
    jx, jy, l, JX, JY, L = _grid_indices(pr)
    if ns is None:
        G = ned(pr, g, jx, jy)                               # (nx, ny, Nt)
        nn = pr.Nt
    else:
        nn = len(ns)
        sub = Problem(**{**pr.__dict__, "Nt": nn})
        G = ned(sub, g, jx, jy)                              # (nx, ny, nn)
    nus = nu(pr, JX, JY, L).reshape(pr.nx * pr.ny, pr.nz)
    F = ner(pr, G.reshape(pr.nx * pr.ny, nn), nus, ns)
    return F.reshape(pr.nx, pr.ny, pr.nz) * coef(pr, JX, JY, L)


def line_spectrum(pr: Problem, g: np.ndarray, jx, jy, ls) -> np.ndarray:
    """F at the lines (jx[i], jy[i]) and depth frequencies ls (any integers):
    the same sums as ``spectrum`` evaluated on a subset; used for sampled
    parity checks at sizes where the whole spectrum is too slow."""
    jx = np.asarray(jx, dtype=np.int64)
    jy = np.asarray(jy, dtype=np.int64)
    ls = np.asarray(ls, dtype=np.int64)
    out = np.zeros((len(jx), len(ls)), dtype=np.complex128)
    for i in range(len(jx)):
        G = ned(pr, g, jx[i:i + 1], jy[i:i + 1]).reshape(1, pr.Nt)
        nus = nu(pr, jx[i], jy[i], ls).reshape(1, -1)
        out[i] = ner(pr, G, nus)[0] * coef(pr, jx[i], jy[i], ls)
    return out


def spectrum_block(pr: Problem, g: np.ndarray, jx, jy, ls) -> np.ndarray:
    """F[a, b, c] at jx[a], jy[b] (every pair: the lines of a product set) and
    depth frequencies ls[c]: the sums of ``spectrum`` on a subset of lines,
    one NED call for all of them.  Used for sampled checks where the whole
    spectrum is too slow; the work is proportional to len(jx) * len(jy)."""
    jx = np.asarray(jx, dtype=np.int64)
    jy = np.asarray(jy, dtype=np.int64)
    ls = np.asarray(ls, dtype=np.int64)
    G = ned(pr, g, jx, jy)                                   # (len(jx), len(jy), Nt)
    JX, JY, L = np.meshgrid(jx, jy, ls, indexing="ij")
    nus = nu(pr, JX, JY, L).reshape(len(jx) * len(jy), len(ls))
    F = ner(pr, G.reshape(len(jx) * len(jy), pr.Nt), nus)
    return F.reshape(len(jx), len(jy), len(ls)) * coef(pr, JX, JY, L)


def _centre_sign(pr: Problem, JX, JY):
    # exp(2 pi i jx (qx - nx/2)/nx) = (-1)^jx exp(2 pi i jx qx / nx)
    return np.where(((JX + JY) % 2) == 0, 1.0, -1.0)


def image_from_spectrum(pr: Problem, F: np.ndarray) -> np.ndarray:
    """Uniform inverse 3D DFT of Sec. 3, step 3 (library FFT), real part,
    voxel-centred as documented in the module docstring.  Returns (nz, ny, nx)."""
    jx, jy, l, JX, JY, L = _grid_indices(pr)
    A = np.zeros((pr.nz, pr.ny, pr.nx), dtype=np.complex128)
    A[np.mod(L, pr.nz), np.mod(JY, pr.ny), np.mod(JX, pr.nx)] = F * _centre_sign(pr, JX, JY)
    return np.real(np.fft.ifftn(A))


def forward(pr: Problem, g: np.ndarray, ns=None) -> np.ndarray:
    """p0 = R g (Sec. 2 Eq. disc_rec followed by Sec. 3 step 3).  (nz, ny, nx).
    ``ns`` as in ``spectrum``."""
    return image_from_spectrum(pr, spectrum(pr, g, ns))


def _dual_spectrum(pr: Problem, p: np.ndarray, sign: int, JX=None, JY=None, L=None) -> np.ndarray:
    """(1/N) sum_q p[q] exp(sign * i theta(k, q)) on G_x x G_Ky, (nx, ny, nz)
    (or on the index arrays JX, JY, L)."""
    if JX is None:
        jx, jy, l, JX, JY, L = _grid_indices(pr)
    p = np.asarray(p, dtype=np.float64).reshape(pr.nz, pr.ny, pr.nx)
    N = pr.nx * pr.ny * pr.nz
    A = np.fft.fftn(p) / N if sign < 0 else np.fft.ifftn(p)
    return A[np.mod(L, pr.nz), np.mod(JY, pr.ny), np.mod(JX, pr.nx)] * _centre_sign(pr, JX, JY)


def _line_subset(pr: Problem, jx, jy):
    """Lateral index sets of the transposed sums: all of G_x, or the product
    set jx x jy (the spectrum is then taken as zero on every other line)."""
    if jx is None:
        return _grid_indices(pr)
    jx = np.asarray(jx, dtype=np.int64)
    jy = np.asarray(jy, dtype=np.int64)
    l = index_set(pr.nz)
    JX, JY, L = np.meshgrid(jx, jy, l, indexing="ij")
    return jx, jy, l, JX, JY, L


def _sensor_subset(pr: Problem, sensors):
    xy = np.asarray(pr.sensor_xy, dtype=np.float64)
    w = pr.sensor_factor()
    if sensors is not None:
        sensors = np.asarray(sensors, dtype=np.int64)
        xy, w = xy[sensors], w[sensors]
    return np.ascontiguousarray(xy), np.ascontiguousarray(w, dtype=np.float64)


def adjoint(pr: Problem, p0: np.ndarray, jx=None, jy=None, sensors=None) -> np.ndarray:
    """R^T p (real transpose of ``forward``):
    g[m, n] = w_m Re sum_{j,l} coef P[j, l] exp(+2 pi i (nu n / Nt + j.x_m)),
    P[j, l] = (1/N) sum_q p[q] exp(-i theta(j, l; q)).  Returns (M, Nt).
    With ``jx``, ``jy`` the sum runs over the lines of the product set jx x jy
    only (exact when the spectrum of p vanishes on the other lines); with
    ``sensors`` only those rows of g are computed."""
    jx, jy, l, JX, JY, L = _line_subset(pr, jx, jy)
    P = _dual_spectrum(pr, p0, -1, JX, JY, L) * coef(pr, JX, JY, L)
    nl = len(jx) * len(jy)
    nus = nu(pr, JX, JY, L).reshape(nl, pr.nz)
    T = ner_adj(pr, P.reshape(nl, pr.nz), nus)                  # (lines, Nt)
    T = np.ascontiguousarray(T.reshape(len(jx), len(jy), pr.Nt))
    xy, w = _sensor_subset(pr, sensors)
    jx32 = np.ascontiguousarray(jx, dtype=np.int32)
    jy32 = np.ascontiguousarray(jy, dtype=np.int32)
    out = np.zeros((len(w), pr.Nt), dtype=np.float64)
    rc = _load().orc_ned_adj(len(w), _p(xy), _p(w), pr.Nt, pr.X, pr.Y, len(jx32), _p(jx32),
                             len(jy32), _p(jy32), _p(T), _p(out), _nthreads())
    if rc != 0:
        raise MemoryError("orc_ned_adj: allocation failed")
    return out


def grad_positions(pr: Problem, g: np.ndarray, dL_dp0: np.ndarray, jx=None, jy=None, sensors=None) -> np.ndarray:
    """dL/d(x_m, y_m) for p0 = R g with dL/dp0 given; the areas h_m are held
    fixed.  Differentiates the NED exponent of Eq. disc_rec.  Returns (M, 2).
    ``jx``, ``jy`` and ``sensors`` restrict the sums as in ``adjoint``."""
    jx, jy, l, JX, JY, L = _line_subset(pr, jx, jy)
    Lam = _dual_spectrum(pr, dL_dp0, +1, JX, JY, L) * coef(pr, JX, JY, L)
    nl = len(jx) * len(jy)
    nus = nu(pr, JX, JY, L).reshape(nl, pr.nz)
    # S[j, n] = sum_l coef Lam exp(-2 pi i nu n / Nt)
    S = np.conj(ner_adj(pr, np.conj(Lam).reshape(nl, pr.nz), nus))
    S = np.ascontiguousarray(S.reshape(len(jx), len(jy), pr.Nt))
    xy, w = _sensor_subset(pr, sensors)
    gg = np.asarray(g, dtype=np.float64).reshape(pr.M, pr.Nt)
    if sensors is not None:
        gg = gg[np.asarray(sensors, dtype=np.int64)]
    gg = np.ascontiguousarray(gg)
    jx32 = np.ascontiguousarray(jx, dtype=np.int32)
    jy32 = np.ascontiguousarray(jy, dtype=np.int32)
    out = np.zeros((len(w), 2), dtype=np.float64)
    rc = _load().orc_ned_grad(len(w), _p(xy), _p(w), pr.Nt, _p(gg), pr.X, pr.Y, len(jx32),
                              _p(jx32), len(jy32), _p(jy32), _p(S), _p(out), _nthreads())
    if rc != 0:
        raise MemoryError("orc_ned_grad: allocation failed")
    return out


__all__ = ["Problem", "build", "index_set", "nu", "jacobian", "coef", "ned", "ner",
           "ner_adj", "spectrum", "line_spectrum", "spectrum_block", "image_from_spectrum", "forward",
           "adjoint", "grad_positions"]
