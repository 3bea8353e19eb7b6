"""The two-dimensional comparison of Sec. 7 on synthetic data: 32 sensors on a
line above an image of 1024 x 256 pixels, equispaced with intervals 1..32
(the detection region swept from 32 to 1024 pixels, centred) against the
equi-angular layout of Sec. 6.1, each reconstruction scored by the
correlation coefficient inside a circular region of interest and by the
Tenenbaum sharpness on the smallest rectangle holding it (Appendix B).

The paper's phantom is a licensed tree image simulated with k-Wave; here a
"tree" of discs (crown) and a vertical bar (trunk, the edge a small aperture
cannot see) stands in, and the data are the physical forward model of the
library, A = R_u^T (the transpose of the unweighted 2-D reconstruction), of
that image, with white noise at 30 dB SNR.  Reconstructions use the weighted
2-D plan (h = interval x dx for the equispaced layouts, h proportional to
r^2 for the equi-angular one).
"""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np

from . import nedner
from .placement import corrcoef, equi_angular


def tree_phantom(nx: int, nz: int, dx: float, dz: float) -> np.ndarray:
    """(nz, nx) image: a crown of discs and a trunk bar below it (depth z
    grows with the row index)."""
    X = nx * dx
    x = (np.arange(nx) - nx // 2) * dx
    z = np.arange(nz) * dz
    ZZ, XX = np.meshgrid(z, x, indexing="ij")
    Z = nz * dz
    f = np.zeros((nz, nx))
    crown = [(0.0, 0.22 * Z, 0.075 * Z, 1.0), (-0.06 * Z, 0.27 * Z, 0.05 * Z, 0.8), (0.07 * Z, 0.26 * Z, 0.045 * Z, 0.9),
             (0.0, 0.16 * Z, 0.04 * Z, 0.7)]
    for cx, cz, r, a in crown:
        f[(XX - cx) ** 2 + (ZZ - cz) ** 2 < r * r] = a
    trunk = (np.abs(XX) < 0.012 * Z) & (ZZ > 0.28 * Z) & (ZZ < 0.42 * Z)
    f[trunk] = 0.9
    assert X > 0
    return f


def _roi(nx, nz, dx, dz):
    Z = nz * dz
    x = (np.arange(nx) - nx // 2) * dx
    z = np.arange(nz) * dz
    ZZ, XX = np.meshgrid(z, x, indexing="ij")
    cz, r = 0.29 * Z, 0.16 * Z
    mask = XX ** 2 + (ZZ - cz) ** 2 < r * r
    rows = np.where(mask.any(axis=1))[0]
    cols = np.where(mask.any(axis=0))[0]
    return mask, (rows[0], rows[-1] + 1, cols[0], cols[-1] + 1), cz


def run(nx: int = 1024, nz: int = 256, dx: float = 50e-6, Nt: int = 512, c: float = 1500.0, n_sensors: int = 32,
        intervals=range(1, 33), snr_db: Optional[float] = 30.0, seed: int = 1517) -> Dict:
    import torch
    dz = dx
    dt = nz * dz / (c * Nt)                          # Z = c Nt dt
    grid = (nx, nz, dx, dz)
    f = tree_phantom(nx, nz, dx, dz)
    ft = torch.as_tensor(f, dtype=torch.float32, device="cuda")
    mask, (z0, z1, x0, x1), cz = _roi(nx, nz, dx, dz)
    mt = torch.as_tensor(mask, device="cuda")
    rng = np.random.default_rng(seed)

    def score(x, h):
        pu = nedner.Plan2D(x, Nt, dt, c, grid, apply_weights=False)
        g = pu.adjoint(ft)
        pu.close()
        if snr_db is not None:
            rms = float(torch.sqrt((g.double() ** 2).mean()))
            noise = rng.normal(0.0, rms * 10.0 ** (-snr_db / 20.0), size=tuple(g.shape))
            g = g + torch.as_tensor(noise, dtype=torch.float32, device="cuda")
        pw = nedner.Plan2D(x, Nt, dt, c, grid, sensor_w=h)
        p = pw.forward(g.contiguous())
        pw.close()
        rho = float(corrcoef(p, ft, mt))
        sharp = float(nedner.tenenbaum(p[z0:z1, x0:x1].contiguous()))
        return rho, sharp

    out = {"image": [nz, nx], "dx": dx, "Nt": Nt, "sensors": n_sensors, "snr_db": snr_db,
           "roi": "circle of radius %.3g m at depth %.3g m; sharpness on rows %d:%d, columns %d:%d"
                  % (0.16 * nz * dz, cz, z0, z1, x0, x1),
           "equispaced": []}
    for k in intervals:
        x = (np.arange(n_sensors) - 0.5 * (n_sensors - 1)) * k * dx
        rho, sharp = score(x, np.full(n_sensors, k * dx))
        out["equispaced"].append({"interval": int(k), "rho": round(rho, 5), "sharpness": round(sharp, 6)})
    best = max(out["equispaced"], key=lambda r: r["rho"])
    out["best_equispaced"] = best
    xe, he = equi_angular(n_sensors, 0.95 * nx * dx, cz)
    rho, sharp = score(xe, he)
    out["equi_angular"] = {"rho": round(rho, 5), "sharpness": round(sharp, 6), "h_max_over_min": float(he.max() / he.min())}
    out["closer_to_full_correlation_pct"] = round(100.0 * (1.0 - (1.0 - rho) / (1.0 - best["rho"])), 1)
    out["sharpness_above_every_equispaced"] = bool(sharp > max(r["sharpness"] for r in out["equispaced"]))
    return out


if __name__ == "__main__":
    import json
    from . import build
    build.build()
    print(json.dumps(run()))
