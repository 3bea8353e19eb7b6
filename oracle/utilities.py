"""FP64 oracle of the utilities around the reconstruction: the data low-pass
of Sec. 8, the Tenenbaum sharpness of Appendix B and maximum intensity
projections.

TEST INFRASTRUCTURE, like the rest of this package (only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU legs use it).  Plain
numpy; numpy's FFT is the one library step (the DFT of each series).

- nearest-neighbour distance: for every sensor, the minimum Euclidean
  distance to any other sensor (brute force over all pairs);
- low-pass: f_cut,m = c / (2 dx_m); the length-Nt DFT G[k] of series m keeps
  the bins whose frequency |k'| / (Nt dt) <= f_cut,m, k' = k for k <= Nt/2
  and k - Nt above (the bin's two-sided index), i.e. |k'| <= floor(f_cut,m
  Nt dt); the others are set to zero and the series is the real part of the
  inverse DFT.  A lone sensor is not filtered;
- Tenenbaum: F = (1 / (nx ny)) sum over the pixels whose 3 x 3 neighbourhood
  lies in the image of (S * U)^2 + (S^T * U)^2, S = [-1 0 1; -2 0 2; -1 0 1]
  (Appendix B, Eq. for F_Tenenbaum, normalised by the number of elements);
- MIP: the maximum along one axis of a (nz, ny, nx) volume.
"""
from __future__ import annotations

import numpy as np

SOBEL = np.array([[-1.0, 0.0, 1.0], [-2.0, 0.0, 2.0], [-1.0, 0.0, 1.0]])


def nearest_neighbour_distance(xy) -> np.ndarray:
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    M = xy.shape[0]
    d = np.full(M, np.inf)
    for m in range(M):
        ex = xy[:, 0] - xy[m, 0]
        ey = xy[:, 1] - xy[m, 1]
        r2 = ex * ex + ey * ey
        r2[m] = np.inf
        if M > 1:
            d[m] = np.sqrt(r2.min())
    return d


def lowpass_bins(xy, Nt: int, dt: float, c: float) -> np.ndarray:
    """Highest kept two-sided bin of each sensor's filter (Nt/2: none cut)."""
    d = nearest_neighbour_distance(xy)
    k = np.full(d.shape[0], Nt // 2, dtype=np.int64)
    ok = np.isfinite(d) & (d > 0)
    kf = np.floor(c / (2.0 * d[ok]) * Nt * dt)
    k[ok] = np.minimum(Nt // 2, kf).astype(np.int64)
    return k


def lowpass(g, xy, dt: float, c: float) -> np.ndarray:
    g = np.asarray(g, dtype=np.float64)
    M, Nt = g.shape
    K = lowpass_bins(xy, Nt, dt, c)
    kk = np.arange(Nt)
    two_sided = np.minimum(kk, Nt - kk)
    out = np.empty_like(g)
    for m in range(M):
        G = np.fft.fft(g[m])
        G[two_sided > K[m]] = 0.0
        out[m] = np.real(np.fft.ifft(G))
    return out


def tenenbaum(U) -> float:
    U = np.asarray(U, dtype=np.float64)
    ny, nx = U.shape
    F = 0.0
    for y in range(1, ny - 1):
        for x in range(1, nx - 1):
            patch = U[y - 1:y + 2, x - 1:x + 2]
            gx = float((SOBEL * patch).sum())
            gy = float((SOBEL.T * patch).sum())
            F += gx * gx + gy * gy
    return F / (nx * ny)


def mip(vol, axis: int) -> np.ndarray:
    return np.asarray(vol).max(axis=axis)


__all__ = ["nearest_neighbour_distance", "lowpass_bins", "lowpass", "tenenbaum", "mip", "SOBEL"]
