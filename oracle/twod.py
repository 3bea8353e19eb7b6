"""FP64 oracle of the two-dimensional variant (Sec. 7): sensors at x_m on the
line z = 0, an image (nz, nx).

TEST INFRASTRUCTURE, like the rest of this package.  Plain numpy, direct
sums (a matrix product serves as the sum over sensors); the final uniform
inverse DFT is numpy's FFT.  Eq. disc_rec with one lateral axis, in physical
units as the 3-D oracle:

    X = nx dx, Z = nz dz,  jx in {-nx/2..nx/2-1},  l in {-nz/2..nz/2-1}
    G[jx, n]  = sum_m w_m g[m, n] exp(-2 pi i jx x_m / X),     w_m = h_m / dx
    nu[jx, l] = sign(l) c Nt dt sqrt((jx/X)^2 + (l/Z)^2)
    F[jx, l]  = C[jx, l] sum_{n<Nt} G[jx, n] exp(-2 pi i nu n / Nt),
                C = W c dt / dz,  W = 2 |l/Z| / |k|,  W(0, 0) = 2,  W(jx != 0, 0) = 0
    p2[qz, qx] = Re (1/(nx nz)) sum_{jx, l} F exp(2 pi i (jx (qx - nx/2)/nx + l qz/nz))

Unweighted (``apply_weights=False``): w_m = 1 and C = 1.  ``adjoint2d`` is the
exact transpose for real inner products.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class Problem2D:
    sensor_x: np.ndarray
    Nt: int
    dt: float
    c: float
    nx: int
    nz: int
    dx: float
    dz: float
    h: Optional[np.ndarray] = None
    apply_weights: bool = True

    @property
    def M(self) -> int:
        return int(np.asarray(self.sensor_x).shape[0])

    @property
    def X(self) -> float:
        return self.nx * self.dx

    @property
    def Z(self) -> float:
        return self.nz * self.dz

    def weights(self) -> np.ndarray:
        if not self.apply_weights:
            return np.ones(self.M)
        h = np.full(self.M, self.X / max(self.M, 1)) if self.h is None else np.asarray(self.h, dtype=np.float64)
        return h / self.dx


def _indices(pr: Problem2D):
    jx = np.arange(-(pr.nx // 2), pr.nx - pr.nx // 2)
    l = np.arange(-(pr.nz // 2), pr.nz - pr.nz // 2)
    JX, L = np.meshgrid(jx, l, indexing="ij")
    return jx, l, JX, L


def coef2d(pr: Problem2D, JX, L) -> np.ndarray:
    if not pr.apply_weights:
        return np.ones(JX.shape)
    k = np.sqrt((JX / pr.X) ** 2 + (L / pr.Z) ** 2)
    W = np.where(k > 0, 2.0 * np.abs(L / pr.Z) / np.where(k > 0, k, 1.0), 2.0)
    return W * pr.c * pr.dt / pr.dz


def nu2d(pr: Problem2D, JX, L) -> np.ndarray:
    return np.sign(L) * pr.c * pr.Nt * pr.dt * np.sqrt((JX / pr.X) ** 2 + (L / pr.Z) ** 2)


def _ex(pr: Problem2D, jx):
    x = np.asarray(pr.sensor_x, dtype=np.float64)
    return np.exp(-2j * np.pi * np.outer(x, jx) / pr.X)                       # (M, nx)


def _et(pr: Problem2D, nus):
    n = np.arange(pr.Nt)
    return np.exp(-2j * np.pi * nus[..., None] * n / pr.Nt)                   # (..., Nt)


def _centre(pr: Problem2D, JX):
    return np.where(JX % 2 == 0, 1.0, -1.0)          # exp(2 pi i jx (qx - nx/2)/nx) = (-1)^jx exp(2 pi i jx qx/nx)


def spectrum2d(pr: Problem2D, g) -> np.ndarray:
    jx, l, JX, L = _indices(pr)
    g = np.asarray(g, dtype=np.float64).reshape(pr.M, pr.Nt)
    G = _ex(pr, jx).T @ (pr.weights()[:, None] * g)                          # (nx, Nt)
    E = _et(pr, nu2d(pr, JX, L))                                             # (nx, nz, Nt)
    return np.einsum("an,aln->al", G, E) * coef2d(pr, JX, L)


def forward2d(pr: Problem2D, g) -> np.ndarray:
    jx, l, JX, L = _indices(pr)
    F = spectrum2d(pr, g) * _centre(pr, JX)
    A = np.zeros((pr.nz, pr.nx), dtype=np.complex128)
    A[np.mod(L, pr.nz), np.mod(JX, pr.nx)] = F
    return np.real(np.fft.ifft2(A))


def adjoint2d(pr: Problem2D, p) -> np.ndarray:
    """g[m, n] = w_m Re sum_{jx, l} C exp(-2 pi i (jx x_m/X + nu n/Nt)) P[jx, l] / (nx nz),
    P[jx, l] = sum_q p[q] (-1)^jx exp(2 pi i (jx qx/nx + l qz/nz)): the transpose of forward2d."""
    jx, l, JX, L = _indices(pr)
    p = np.asarray(p, dtype=np.float64).reshape(pr.nz, pr.nx)
    B = np.fft.ifft2(p) * (pr.nx * pr.nz)                                    # sum_q p exp(+2 pi i ...)
    P = B[np.mod(L, pr.nz), np.mod(JX, pr.nx)] * _centre(pr, JX) * coef2d(pr, JX, L) / (pr.nx * pr.nz)
    E = _et(pr, nu2d(pr, JX, L))                                             # (nx, nz, Nt)
    T = np.einsum("al,aln->an", P, E)                                        # (nx, Nt)
    return pr.weights()[:, None] * np.real(_ex(pr, jx) @ T)


__all__ = ["Problem2D", "coef2d", "nu2d", "spectrum2d", "forward2d", "adjoint2d"]
