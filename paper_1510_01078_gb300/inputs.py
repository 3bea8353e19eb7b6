"""Seeded synthetic inputs: sensor layouts, ball phantoms and their data.

This module holds no reconstruction arithmetic.  It is the one module that
both the CUDA path's tests/benchmark and the FP64 oracle draw inputs from.

Layouts follow the paper's setup (Sec. 4 and Sec. 6: a planar sensor with
centre-dense, non-equispaced positions and a detector area h_m per sensor,
Eq. disc_rec).  The data model is the closed-form pressure of a uniform ball in
3D (the solution of the wave equation of Sec. 2 with a ball-shaped initial
pressure): at distance r from the centre of a ball of radius R and amplitude A,

    p(t) = A (r - c t) / (2 r)   for |r - c t| < R,   0 otherwise,

the "N-shaped" signal.  The paper's own data (k-Wave simulations and chick
embryo measurements) are not available; these stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np

C_SOUND = 1500.0


# --------------------------------------------------------------------------
# sensor layouts
# --------------------------------------------------------------------------
def law_coords(n: int, L: float, power: float = 1.5, rng: Optional[np.random.Generator] = None) -> np.ndarray:
    """Centre-dense 1-D coordinates x_i = (L/2) sign(u_i) |u_i|^power.

    u_i are the midpoints -1 + (2 i + 1)/n (deterministic), or uniform draws in
    (-1, 1) when ``rng`` is given.  All |x_i| < L/2.
    """
    if rng is None:
        u = -1.0 + (2.0 * np.arange(n) + 1.0) / n
    else:
        u = np.sort(rng.uniform(-1.0, 1.0, size=n))
    return 0.5 * L * np.sign(u) * np.abs(u) ** power


def cell_widths(x: np.ndarray, X: float) -> np.ndarray:
    """1-D midpoint cell widths of sorted coordinates, the outer cells extended
    to +-X/2, so that the widths sum to X."""
    x = np.asarray(x, dtype=np.float64)
    edges = np.concatenate([[-X / 2], 0.5 * (x[1:] + x[:-1]), [X / 2]])
    return np.diff(edges)


def tensor_sensors(nsx: int, nsy: int, L: float, X: float, power: float = 1.5):
    """Tensor product of two centre-dense coordinate sets; h_m = product of
    the 1-D cell widths (sums to X^2).  Sensor m = iy * nsx + ix."""
    xs = law_coords(nsx, L, power)
    ys = law_coords(nsy, L, power)
    hx = cell_widths(xs, X)
    hy = cell_widths(ys, X)
    YY, XX = np.meshgrid(ys, xs, indexing="ij")
    HY, HX = np.meshgrid(hy, hx, indexing="ij")
    xy = np.stack([XX.ravel(), YY.ravel()], axis=1)
    return xy, (HX * HY).ravel(), xs, ys


def disc_sensors(M: int, R: float, a: float, rng: np.random.Generator):
    """M scattered sensors in a disc of radius R with areal density
    proportional to 1 / (1 + (r/a)^2) (centre-dense).  Radii by inverse CDF,
    r = a sqrt(exp(U ln(1 + (R/a)^2)) - 1); h_m proportional to 1/density,
    normalised to the disc area pi R^2."""
    U = rng.uniform(0.0, 1.0, size=M)
    r = a * np.sqrt(np.exp(U * np.log1p((R / a) ** 2)) - 1.0)
    th = rng.uniform(0.0, 2.0 * np.pi, size=M)
    xy = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    inv = 1.0 + (r / a) ** 2
    h = inv / inv.sum() * np.pi * R * R
    return xy, h


def scattered_square(M: int, X: float, rng: np.random.Generator, margin: float = 0.999):
    """M uniform sensors in the open square (-X/2, X/2)^2 with equal areas."""
    xy = rng.uniform(-0.5 * X * margin, 0.5 * X * margin, size=(M, 2))
    return xy, np.full(M, X * X / max(M, 1))


# --------------------------------------------------------------------------
# phantoms and data
# --------------------------------------------------------------------------
@dataclass
class Balls:
    centres: np.ndarray   # (B, 3) metres, z > 0 below the sensor plane
    radii: np.ndarray     # (B,)
    amps: np.ndarray      # (B,)


def random_balls(n: int, rng: np.random.Generator, r_range, xy_half: float, z_range, amp_range=(1.0, 1.0)) -> Balls:
    cx = rng.uniform(-xy_half, xy_half, size=n)
    cy = rng.uniform(-xy_half, xy_half, size=n)
    cz = rng.uniform(z_range[0], z_range[1], size=n)
    R = rng.uniform(r_range[0], r_range[1], size=n)
    A = rng.uniform(amp_range[0], amp_range[1], size=n)
    return Balls(np.stack([cx, cy, cz], axis=1), R, A)


def nwave_data(sensor_xy: np.ndarray, balls: Balls, Nt: int, dt: float, c: float = C_SOUND,
               chunk: int = 1024) -> np.ndarray:
    """g[m, n] = sum over balls of A (r - c t_n) / (2 r) for |r - c t_n| < R.

    Each ball's signal is non-zero only for |r - c t_n| < R, so only the
    samples of that window (plus one on each side) are evaluated; the values
    and the order in which the balls are added are those of the plain sum."""
    xy = np.asarray(sensor_xy, dtype=np.float64)
    M = xy.shape[0]
    g = np.zeros((M, Nt), dtype=np.float64)
    ct = c * dt * np.arange(Nt, dtype=np.float64)
    cdt = c * dt
    for b in range(len(balls.radii)):
        cx, cy, cz = balls.centres[b]
        R, A = balls.radii[b], balls.amps[b]
        K = int(np.ceil(2.0 * R / cdt)) + 4                 # samples of a window, with margin
        for s in range(0, M, chunk):
            r = np.sqrt((xy[s:s + chunk, 0] - cx) ** 2 + (xy[s:s + chunk, 1] - cy) ** 2 + cz * cz)
            n0 = np.floor((r - R) / cdt).astype(np.int64) - 1
            idx = n0[:, None] + np.arange(K)[None, :]
            ok = (idx >= 0) & (idx < Nt)
            idc = np.clip(idx, 0, Nt - 1)
            d = r[:, None] - ct[idc]
            inside = ok & (np.abs(d) < R)
            rows = np.broadcast_to(np.arange(s, s + len(r))[:, None], idc.shape)
            g[rows[inside], idc[inside]] += (A * d / (2.0 * r[:, None]))[inside]
    return g


def add_noise(g: np.ndarray, snr_db: float, rng: np.random.Generator) -> np.ndarray:
    """Additive white Gaussian noise with sigma = RMS(g) 10^(-snr/20)."""
    rms = float(np.sqrt(np.mean(g * g))) if g.size else 0.0
    return g + rng.normal(0.0, rms * 10.0 ** (-snr_db / 20.0), size=g.shape)


def voxelise(balls: Balls, nx, ny, nz, dx, dy, dz) -> np.ndarray:
    """True initial pressure on the output grid (nz, ny, nx): sum of uniform
    balls sampled at voxel centres x = (qx - nx/2) dx, y = (qy - ny/2) dy, z = qz dz."""
    x = (np.arange(nx) - nx // 2) * dx
    y = (np.arange(ny) - ny // 2) * dy
    z = np.arange(nz) * dz
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    f = np.zeros((nz, ny, nx))
    for b in range(len(balls.radii)):
        cx, cy, cz = balls.centres[b]
        inside = (Xg - cx) ** 2 + (Yg - cy) ** 2 + (Zg - cz) ** 2 < balls.radii[b] ** 2
        f += np.where(inside, balls.amps[b], 0.0)
    return f


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
CONFIG_NAMES = ["c1_tiny_fp64", "c2_fp32_64x64", "c3_paper_scale", "c4_differentiation", "c5_tensor_gemm"]


def make_config(idx: int, with_data: bool = True, Nt: Optional[int] = None,
                lateral: Optional[int] = None) -> Dict:
    """Workload ``idx`` (0..4); seed 1510 + idx.  Returns a dict with the
    geometry (sensor_xy, h, Nt, dt, c, nx, ny, nz, dx, dy, dz), the phantom and,
    if ``with_data``, the float64 data g (M, Nt).  ``Nt`` shortens (or
    lengthens) the record, nz scaled with it so that dz stays the same: the
    same lateral geometry and kernels on a smaller case.  ``lateral`` (a power
    of two below nx, square lateral grids only) keeps the central lateral x
    lateral voxels at the same spacing, with the sensors and balls inside that
    square: the same record, depth and sensor density on fewer lines."""
    nt_req = Nt
    rng = np.random.default_rng(1510 + idx)
    c = C_SOUND
    extra: Dict = {}
    if idx == 0:
        # 16x16 centre-dense tensor grid over 4 mm; Nt 64 at 50 ns; 16x16x32 voxels
        X = 4e-3
        xy, h, xs, ys = tensor_sensors(16, 16, X, X)
        Nt, dt, nx, ny, nz = 64, 50e-9, 16, 16, 32
        balls = random_balls(2, rng, (0.2e-3, 0.4e-3), 1.2e-3, (0.6e-3, 1.8e-3))
        snr = None
        extra = {"xs": xs, "ys": ys}
    elif idx == 1:
        # 64x64 tensor grid over 20 mm; Nt 512 at 16.7 ns; 128x128x256 voxels
        X = 20e-3
        xy, h, xs, ys = tensor_sensors(64, 64, X, X)
        Nt, dt, nx, ny, nz = 512, 16.7e-9, 128, 128, 256
        balls = random_balls(20, rng, (0.1e-3, 0.5e-3), X / 4, (1e-3, 6e-3), (0.5, 1.0))
        snr = 20.0
        extra = {"xs": xs, "ys": ys}
    elif idx == 2:
        # 16384 scattered sensors in a 30 mm disc; Nt 2048 at 8.3 ns; 256x256x512
        X = 30e-3
        xy, h = disc_sensors(16384, X / 2, 5e-3, rng)
        Nt, dt, nx, ny, nz = 2048, 8.3e-9, 256, 256, 512
        balls = random_balls(200, rng, (0.05e-3, 0.4e-3), X / 4, (1e-3, 12e-3), (0.5, 1.0))
        snr = 20.0
    elif idx == 3:
        # 64x64 tensor grid over 20 mm; Nt 1024 at 16.7 ns; 128^3; central 32x32 movable
        X = 20e-3
        xy, h, xs, ys = tensor_sensors(64, 64, X, X)
        Nt, dt, nx, ny, nz = 1024, 16.7e-9, 128, 128, 128
        balls = random_balls(20, rng, (0.1e-3, 0.5e-3), X / 4, (1e-3, 6e-3), (0.5, 1.0))
        snr = 20.0
        iy, ix = np.divmod(np.arange(64 * 64), 64)
        movable = (ix >= 16) & (ix < 48) & (iy >= 16) & (iy < 48)
        extra = {"xs": xs, "ys": ys, "movable": movable}
    elif idx == 4:
        # 128x128 non-equispaced tensor grid over 20 mm; Nt 2048 at 8.3 ns; 256x256x512
        X = 20e-3
        xy, h, xs, ys = tensor_sensors(128, 128, X, X)
        Nt, dt, nx, ny, nz = 2048, 8.3e-9, 256, 256, 512
        balls = random_balls(200, rng, (0.05e-3, 0.4e-3), X / 4, (1e-3, 12e-3), (0.5, 1.0))
        snr = 20.0
        extra = {"xs": xs, "ys": ys}
    else:
        raise ValueError("config index must be 0..4")
    Nt0 = Nt
    if nt_req is not None and nt_req != Nt:
        if nt_req < 16 or nt_req & (nt_req - 1) or (nz * nt_req) % Nt:
            raise ValueError("Nt must be a power of two >= 16 that keeps nz whole")
        nz = nz * nt_req // Nt
        Nt = int(nt_req)
    dx = X / nx
    dy = X / ny
    dz = c * Nt * dt / nz          # Z = c Nt dt: the record spans the periodic depth range
    name = CONFIG_NAMES[idx] + ("" if nt_req is None or nt_req == Nt0 else "_nt%d" % Nt)
    if lateral is not None and lateral != nx:
        if nx != ny or lateral < 8 or lateral > nx or lateral & (lateral - 1):
            raise ValueError("lateral must be a power of two >= 8 below nx, on a square grid")
        half = 0.5 * lateral * dx
        keep = np.all(np.abs(xy) < 0.98 * half, axis=1)
        xy, h = xy[keep], h[keep]
        inside = np.all(np.abs(balls.centres[:, :2]) + balls.radii[:, None] < half, axis=1)
        balls = Balls(balls.centres[inside], balls.radii[inside], balls.amps[inside])
        extra = {}                        # a cropped tensor grid is no longer the workload's grid
        nx = ny = int(lateral)
        name += "_lat%d" % nx
    cfg = dict(name=name, sensor_xy=xy, h=h, Nt=Nt, dt=dt, c=c, nx=nx, ny=ny, nz=nz,
               dx=dx, dy=dy, dz=dz, balls=balls, snr_db=snr, seed=1510 + idx, **extra)
    if with_data:
        g = nwave_data(xy, balls, Nt, dt, c)
        if snr is not None:
            g = add_noise(g, snr, rng)
        cfg["g"] = g
    return cfg


def small_case(nx: int, ny: int, nz: int, M: int, Nt: int, seed: int, layout: str = "scatter",
               data: str = "random", dt: float = 20e-9, X: Optional[float] = None) -> Dict:
    """A seeded test geometry of arbitrary (small) size: ``layout`` 'scatter'
    (uniform in the square), 'disc' (centre-dense) or 'grid' (sensors on the
    output grid, h = dx dy); ``data`` 'random' (standard normal) or 'balls'."""
    rng = np.random.default_rng(seed)
    c = C_SOUND
    if X is None:
        X = nx * 0.1e-3
    Y = X * ny / nx
    dx, dy = X / nx, Y / ny
    dz = c * Nt * dt / nz
    if layout == "scatter":
        xy = np.stack([rng.uniform(-0.4999 * X, 0.4999 * X, M), rng.uniform(-0.4999 * Y, 0.4999 * Y, M)], 1)
        h = np.full(M, X * Y / max(M, 1))
    elif layout == "disc":
        xy, h = disc_sensors(M, 0.4999 * min(X, Y), 0.15 * min(X, Y), rng)
    elif layout == "grid":
        qx = np.arange(nx) - nx // 2
        qy = np.arange(ny) - ny // 2
        QY, QX = np.meshgrid(qy, qx, indexing="ij")
        xy = np.stack([QX.ravel() * dx, QY.ravel() * dy], 1)
        # the grid point -X/2 lies on the boundary; nudge it inside the open square
        xy = np.clip(xy, -0.5 * X + 1e-12 * X, None)
        h = np.full(xy.shape[0], dx * dy)
        M = xy.shape[0]
    else:
        raise ValueError(layout)
    if data == "random":
        g = rng.standard_normal((M, Nt))
    elif data == "balls":
        balls = random_balls(3, rng, (2 * dx, 4 * dx), X / 4, (0.1 * nz * dz, 0.4 * nz * dz))
        g = nwave_data(xy, balls, Nt, dt, c)
    else:
        raise ValueError(data)
    return dict(name=f"small_{nx}x{ny}x{nz}_M{M}_Nt{Nt}", sensor_xy=xy, h=h, Nt=Nt, dt=dt, c=c,
                nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, g=g, seed=seed)


__all__ = ["law_coords", "cell_widths", "tensor_sensors", "disc_sensors", "scattered_square",
           "Balls", "random_balls", "nwave_data", "add_noise", "voxelise", "make_config",
           "small_case", "CONFIG_NAMES", "C_SOUND"]
