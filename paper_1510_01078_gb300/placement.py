"""Sensor placement (Sec. 6): the equi-steradian layout of Appendix A, the
h_m proportional to r^3 weighting of Sec. 6.2, the correlation coefficient of
Appendix B (Eq. corrcoeff), and a gradient-descent refinement of the sensor
positions through the library's position gradient.

The paper places a limited number of sensors by a geometric rule: every unit
of solid angle seen from a point of interest at depth r0 gets one sensor, so
the layout is dense under that point and sparse further out (a mock
hemispherical detector).  ``equi_steradian`` builds that layout.

``optimise_placement`` poses the same question as an optimisation: the
positions x are moved to maximise the correlation coefficient between a
target volume f and its reconstruction R(x) A(x) f, where A(x) = R_u(x)^T is
the physical forward model (the transpose of the unweighted reconstruction,
data of an initial pressure at the sensors x) and R(x) the weighted
reconstruction.  Both depend on x; their position derivatives are the
library's nedner_grad_positions on the weighted and on the unweighted plan
(d/dx <v, A(x) f> = d/dx <R_u(x) v, f>).  The weights h_m are held fixed
while the sensors move.

Readings of Appendix A where the text is ambiguous or garbled:
- the first slice, the cap of exactly one unit solid angle, holds one sensor
  on the axis (its mid polar angle would put a single point off the axis);
  slice k >= 2 spans [theta_{k-1}, theta_k] and its j_k sensors sit at the
  mid polar angle (theta_{k-1} + theta_k) / 2;
- the doubling test compares distances on the sensor plane: r_s is the chord
  between neighbouring sensors of the trial slice (j_k = j_{k-1}), the
  slice's diameter when it has one sensor, and r_k the distance from a
  sensor of the trial slice to the nearest sensor of slice k-1; j_k is
  doubled (once) when r_s > 1.8 r_k;
- phi_r, the azimuth offset, is the previous slice's last azimuth plus half
  of its spacing;
- slices are added while their mid polar angle stays inside the cap of half
  angle theta_max = atan(D / (2 r0)), so all sensors lie in the disc of
  diameter D and the count is N rounded to what the slices give.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional

import numpy as np

from . import nedner


# --------------------------------------------------------------------------
# layouts (Appendix A, Sec. 6.2)
# --------------------------------------------------------------------------
def _ring(rho: float, j: int, phi_r: float) -> np.ndarray:
    """j points at radius rho on the plane, azimuths 2 pi i / j + pi / j + phi_r."""
    phi = 2.0 * np.pi * np.arange(j) / j + np.pi / j + phi_r
    return np.stack([rho * np.cos(phi), rho * np.sin(phi)], axis=1), phi


def equi_steradian(N: int, D: float, r0: float, return_slices: bool = False):
    """Equi-steradian layout (Appendix A) for about N sensors in a disc of
    diameter D on the plane z = 0, seen from the point of interest (0, 0, r0).

    Returns (xy (M, 2) metres, h (M,)) with h_m proportional to r_m^3, r_m the
    distance from the point of interest (Sec. 6.2), normalised to the disc
    area pi D^2 / 4; with ``return_slices`` also a list of per-slice dicts
    (theta_in, theta_out, pol, j, phi)."""
    if N < 1 or not (D > 0 and r0 > 0):
        raise ValueError("need N >= 1, D > 0, r0 > 0")
    theta_max = math.atan(0.5 * D / r0)
    Omega = 2.0 * math.pi * (1.0 - math.cos(theta_max))
    omega = Omega / N
    # slice 1: the cap of one unit solid angle, one sensor on the axis
    c_in = 1.0 - omega / (2.0 * math.pi)
    slices = [dict(theta_in=0.0, theta_out=math.acos(c_in), pol=0.0, j=1, phi=np.array([math.pi]))]
    pts: List[np.ndarray] = [np.zeros((1, 2))]
    prev_xy = pts[0]
    j_prev, phi_last = 1, math.pi
    while True:
        phi_r = phi_last + math.pi / j_prev

        def trial(j):
            c_out = c_in - omega * j / (2.0 * math.pi)
            if c_out <= -1.0:
                return None
            t_in, t_out = math.acos(c_in), math.acos(c_out)
            pol = 0.5 * (t_in + t_out)
            if pol >= theta_max or pol >= 0.5 * math.pi:
                return None
            rho = r0 * math.tan(pol)
            xy, phi = _ring(rho, j, phi_r)
            return c_out, t_in, t_out, pol, rho, xy, phi

        t = trial(j_prev)
        if t is None:
            break
        _, _, _, _, rho, xy, _ = t
        r_s = 2.0 * rho * math.sin(math.pi / j_prev) if j_prev > 1 else 2.0 * rho
        d = np.sqrt(((xy[:, None, :] - prev_xy[None, :, :]) ** 2).sum(-1))
        r_k = float(d.min(axis=1).min())
        j = 2 * j_prev if r_s > 1.8 * r_k else j_prev
        if j != j_prev:
            t = trial(j)
            if t is None:
                break
        c_out, t_in, t_out, pol, rho, xy, phi = t
        slices.append(dict(theta_in=t_in, theta_out=t_out, pol=pol, j=j, phi=phi))
        pts.append(xy)
        prev_xy = xy
        j_prev, phi_last, c_in = j, float(phi[-1]), c_out
    xy = np.concatenate(pts, axis=0)
    r = np.sqrt((xy ** 2).sum(1) + r0 * r0)
    h = r ** 3
    h = h / h.sum() * (math.pi * D * D / 4.0)
    if return_slices:
        return xy, h, slices
    return xy, h


def equi_angular(N: int, D: float, r0: float):
    """Equi-angular layout on a line (Sec. 6.1, the 2-D variant): N sensors
    whose lines to the point of interest (0, r0) enclose equal angles, the
    angle of the detection region 2 atan(D / (2 r0)) split into N equal parts
    with a sensor at each part's middle angle, x_i = r0 tan(theta_i); h_i
    proportional to r_i^2 (Sec. 6.2, 2-D), normalised to D."""
    if N < 1 or not (D > 0 and r0 > 0):
        raise ValueError("need N >= 1, D > 0, r0 > 0")
    tmax = math.atan(0.5 * D / r0)
    theta = -tmax + (np.arange(N) + 0.5) * (2.0 * tmax / N)
    x = r0 * np.tan(theta)
    h = x * x + r0 * r0
    return x, h / h.sum() * D


def regular_grid(M: int, D: float):
    """The regular comparison layout with about M sensors: an n x n grid of
    cell centres over the square of side D (n = round(sqrt M)), h = (D/n)^2."""
    n = max(1, int(round(math.sqrt(M))))
    q = (np.arange(n) + 0.5) / n * D - 0.5 * D
    YY, XX = np.meshgrid(q, q, indexing="ij")
    xy = np.stack([XX.ravel(), YY.ravel()], axis=1)
    return xy, np.full(n * n, (D / n) ** 2)


# --------------------------------------------------------------------------
# quality measure (Appendix B, Eq. corrcoeff)
# --------------------------------------------------------------------------
def corrcoef(u1, u2, mask=None):
    """rho(U1, U2) = Cov(U1, U2) / sqrt(Var U1 Var U2) over the elements
    (those where ``mask`` is true); torch tensors (differentiable) or arrays."""
    try:
        import torch
        is_t = isinstance(u1, torch.Tensor)
    except ImportError:                                   # pragma: no cover
        is_t = False
    if mask is not None:
        u1, u2 = u1[mask], u2[mask]
    if is_t:
        a = u1.reshape(-1).double()
        b = u2.reshape(-1).double()
        a = a - a.mean()
        b = b - b.mean()
        return (a * b).sum() / torch.sqrt((a * a).sum() * (b * b).sum())
    a = np.asarray(u1, dtype=np.float64).ravel()
    b = np.asarray(u2, dtype=np.float64).ravel()
    a = a - a.mean()
    b = b - b.mean()
    return float((a * b).sum() / math.sqrt((a * a).sum() * (b * b).sum()))


def upper_half_mask(nz: int, ny: int, nx: int):
    """Voxels at depth index < nz/2 (the part of the periodic depth range that
    holds the phantom; the mirror image fills the rest)."""
    m = np.zeros((nz, ny, nx), dtype=bool)
    m[: nz // 2] = True
    return m


# --------------------------------------------------------------------------
# placement by gradient descent through the position gradient
# --------------------------------------------------------------------------
def optimise_placement(plan_w: "nedner.Plan", plan_u: "nedner.Plan", f, sensor_xy, steps: int = 20,
                       lr: float = 1e-3, movable=None, mask=None, margin: float = 0.999) -> Dict:
    """Moves the sensors to maximise rho(R(x) A(x) f, f) over ``mask``.

    plan_w: weighted plan (apply_weights on, the sensors' h_m); plan_u: the
    same sensors unweighted (apply_weights off), whose transpose is A.
    f: (nz, ny, nx) float32 CUDA tensor.  sensor_xy: (M, 2) float64 array
    (metres), the starting layout.  lr is a step in units of the lateral
    extent X per step (Adam).  movable: optional (M,) bool mask.  Returns
    {"xy": final positions (M, 2) array, "rho": [rho at each step, and at the
    end], "grad_norm": [...]}."""
    import torch
    dev = f.device
    X = plan_w.nx * plan_w.grid[3]
    Y = plan_w.ny * plan_w.grid[4]
    scale = torch.tensor([X, Y], dtype=torch.float64)
    u = torch.as_tensor(np.asarray(sensor_xy, dtype=np.float64)) / scale
    u = u.clone().requires_grad_(True)
    mv = None if movable is None else torch.as_tensor(np.asarray(movable, dtype=bool))
    mk = None if mask is None else torch.as_tensor(np.asarray(mask, dtype=bool), device=dev)
    opt = torch.optim.Adam([u], lr=lr)
    rho_hist: List[float] = []
    gn: List[float] = []
    for k in range(steps + 1):
        opt.zero_grad()
        xy = u * scale
        g = nedner.model(plan_u, f, xy)
        p0 = nedner.reconstruct(plan_w, g, xy)
        rho = corrcoef(p0, f, mk)
        rho_hist.append(float(rho.detach()))
        if k == steps:
            break
        (-rho).backward()
        if mv is not None:
            u.grad[~mv] = 0.0
        gn.append(float(u.grad.norm()))
        opt.step()
        with torch.no_grad():
            u[:, 0].clamp_(-0.5 * margin, 0.5 * margin)
            u[:, 1].clamp_(-0.5 * margin, 0.5 * margin)
    return {"xy": (u.detach() * scale).numpy(), "rho": rho_hist, "grad_norm": gn}


def layout_rho(cfg_grid, Nt: int, dt: float, c: float, xy, h, balls, truth, mask=None, snr_db: Optional[float] = None,
               rng=None) -> float:
    """Correlation coefficient of the reconstruction from analytic N-wave
    data of ``balls`` at the sensors ``xy`` (weights h) with the voxelised
    ``truth`` (over ``mask``).  cfg_grid: (nx, ny, nz, dx, dy, dz)."""
    import torch
    from . import inputs
    g = inputs.nwave_data(xy, balls, Nt, dt, c)
    if snr_db is not None:
        g = inputs.add_noise(g, snr_db, rng if rng is not None else np.random.default_rng(0))
    plan = nedner.Plan(xy, Nt, dt, c, cfg_grid, sensor_w=h)
    try:
        p0 = plan.forward(torch.as_tensor(g, dtype=torch.float32, device="cuda")).cpu().numpy()
    finally:
        plan.close()
    return corrcoef(p0, truth, mask)


def compare_layouts(N: int = 1024, D: float = 18e-3, r0: float = 5e-3, grid=(128, 128, 256), X: float = 20e-3,
                    Nt: int = 512, dt: float = 16.7e-9, c: float = 1500.0, n_balls: int = 20, seed: int = 1510,
                    steps: int = 30, lr: float = 2e-3, snr_db: Optional[float] = 20.0) -> Dict:
    """Correlation coefficient (Eq. corrcoeff, over the upper half depth) of
    reconstructions of synthetic balls around the point of interest from
    three layouts with the same number of sensors: the equi-steradian layout,
    a regular grid, and the equi-steradian layout refined by
    ``optimise_placement`` (sensor weights kept).  Data are the analytic
    N-waves of the balls at each layout (plus noise at ``snr_db``)."""
    import torch
    from . import inputs
    nx, ny, nz = grid
    dx, dy = X / nx, X / ny
    dz = c * Nt * dt / nz
    g3 = (nx, ny, nz, dx, dy, dz)
    rng = np.random.default_rng(seed)
    balls = inputs.random_balls(n_balls, rng, (0.1e-3, 0.5e-3), 0.2 * D, (0.5 * r0, 1.5 * r0), (0.5, 1.0))
    truth = inputs.voxelise(balls, nx, ny, nz, dx, dy, dz)
    mask = upper_half_mask(nz, ny, nx)
    xy_es, h_es = equi_steradian(N, D, r0)
    M = xy_es.shape[0]
    xy_rg, h_rg = regular_grid(M, D)
    out = {"M_equi_steradian": int(M), "M_grid": int(xy_rg.shape[0]), "D": D, "r0": r0,
           "grid": list(grid), "X": X, "Nt": Nt, "dt": dt, "balls": n_balls, "snr_db": snr_db}
    out["rho_equi_steradian"] = layout_rho(g3, Nt, dt, c, xy_es, h_es, balls, truth, mask, snr_db, np.random.default_rng(1))
    out["rho_grid"] = layout_rho(g3, Nt, dt, c, xy_rg, h_rg, balls, truth, mask, snr_db, np.random.default_rng(1))
    plan_w = nedner.Plan(xy_es, Nt, dt, c, g3, sensor_w=h_es)
    plan_u = nedner.Plan(xy_es, Nt, dt, c, g3, apply_weights=False)
    try:
        f = torch.as_tensor(truth, dtype=torch.float32, device="cuda")
        res = optimise_placement(plan_w, plan_u, f, xy_es, steps=steps, lr=lr, mask=mask)
    finally:
        plan_w.close()
        plan_u.close()
    out["model_rho_history"] = [round(v, 5) for v in res["rho"]]
    out["rho_optimised"] = layout_rho(g3, Nt, dt, c, res["xy"], h_es, balls, truth, mask, snr_db, np.random.default_rng(1))
    out["mean_shift_m"] = float(np.sqrt(((res["xy"] - xy_es) ** 2).sum(1)).mean())
    return out


__all__ = ["equi_steradian", "equi_angular", "regular_grid", "corrcoef", "upper_half_mask", "optimise_placement", "layout_rho",
           "compare_layouts"]


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="equi-steradian vs regular grid vs optimised placement")
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--lr", type=float, default=2e-3)
    a = ap.parse_args()
    from . import build
    build.build()
    print(json.dumps(compare_layouts(N=a.N, steps=a.steps, lr=a.lr)))
