"""FP64 oracle of the comparison method of Sec. 5.1 (Table 1): the NER sums
evaluated by an FFT of each line followed by linear interpolation.

TEST INFRASTRUCTURE, like the rest of this package.

For each lateral line j the samples G[j, n], n < Nt, are zero-padded at the
end to sigma Nt (sigma = 1: no padding) and transformed,
    B[mu] = sum_{n < Nt} G[j, n] exp(-2 pi i mu n / (sigma Nt)),
which is the NER sum at the grid frequencies nu = mu / sigma; between them
the value at nu is the linear interpolation of B at v = sigma nu:
    F_lin(nu) = (1 - t) B[floor v] + t B[floor v + 1],   t = v - floor v
(indices modulo sigma Nt).  No window, no deconvolution, no centring.  The
rest of the reconstruction (Jacobian, scale, inverse 3-D DFT) is that of the
main oracle.  numpy's FFT is the library step.
"""
from __future__ import annotations

import numpy as np

from . import Problem, _grid_indices, coef, image_from_spectrum, ned, nu


def ner_linear(pr: Problem, G: np.ndarray, nus: np.ndarray, sigma: int) -> np.ndarray:
    """F_lin[j, l] for the lines G (rows, Nt columns) at the frequencies nus."""
    G = np.asarray(G, dtype=np.complex128).reshape(-1, pr.Nt)
    nus = np.asarray(nus, dtype=np.float64).reshape(G.shape[0], -1)
    Lt = sigma * pr.Nt
    B = np.fft.fft(G, n=Lt, axis=1)
    v = sigma * nus
    i0 = np.floor(v)
    t = v - i0
    i0 = i0.astype(np.int64)
    rows = np.arange(G.shape[0])[:, None]
    return (1.0 - t) * B[rows, np.mod(i0, Lt)] + t * B[rows, np.mod(i0 + 1, Lt)]


def forward_linear(pr: Problem, g: np.ndarray, sigma: int) -> np.ndarray:
    """p0 with the NER sums replaced by ``ner_linear`` (the FFT method of
    Table 1 with oversampling sigma).  (nz, ny, nx)."""
    jx, jy, l, JX, JY, L = _grid_indices(pr)
    G = ned(pr, g, jx, jy).reshape(pr.nx * pr.ny, pr.Nt)
    nus = nu(pr, JX, JY, L).reshape(pr.nx * pr.ny, pr.nz)
    F = ner_linear(pr, G, nus, sigma).reshape(pr.nx, pr.ny, pr.nz) * coef(pr, JX, JY, L)
    return image_from_spectrum(pr, F)


__all__ = ["ner_linear", "forward_linear"]
