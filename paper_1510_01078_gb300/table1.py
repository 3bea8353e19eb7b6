"""The comparison of Sec. 5.1 (Table 1) on synthetic data: the NER-NUFFT
against the FFT with linear interpolation (oversampling sigma = 2 and 1),
each scored by its correlation deficit 100 (1 - rho) in % against the direct
FT (the NER sums evaluated directly), over the 3-D volume and its three
maximum intensity projections, with the reconstruction time of each.

The paper's sphere comes from a k-Wave forward simulation; here the data are
the analytic N-waves of a uniform ball (the closed form of the wave
equation's solution for a uniform ball) sampled at sensors on the output
grid (a regular grid, h = dx dy).  Every reconstruction, the ground truth
included, runs in the library (nedner_opts.ner_interp selects the NER
method); the MIPs and the correlation coefficient as well.
"""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np

from . import inputs, nedner
from .placement import corrcoef

METHODS = [("NER (sigma=2, w=12)", "nufft", 12), ("NER (sigma=2, w=4)", "nufft", 4),
           ("FFT + linear (sigma=2)", "linear2", 12), ("FFT + linear (sigma=1)", "linear1", 12)]


def ball_workload(n: int = 128, nz: int = 256, Nt: int = 512, dx: float = 0.1e-3, dt: float = 20e-9,
                  c: float = 1500.0, R: float = 1.0e-3, depth: Optional[float] = None) -> Dict:
    """Sensors on the n x n output grid, one uniform ball of radius R at the
    centre, at ``depth`` (default a quarter of the periodic depth range)."""
    X = n * dx
    dz = c * Nt * dt / nz
    q = (np.arange(n) - n // 2) * dx
    YY, XX = np.meshgrid(q, q, indexing="ij")
    xy = np.stack([XX.ravel(), YY.ravel()], 1)
    # the grid point -X/2 lies on the boundary of the open aperture (it is the
    # periodic image of +X/2); nudge it inside
    xy = np.clip(xy, -0.5 * X + 1e-12 * X, None)
    h = np.full(n * n, dx * dx)
    depth = 0.25 * nz * dz if depth is None else depth
    balls = inputs.Balls(np.array([[0.0, 0.0, depth]]), np.array([R]), np.array([1.0]))
    g = inputs.nwave_data(xy, balls, Nt, dt, c)
    return dict(name="ball_on_regular_grid", sensor_xy=xy, h=h, Nt=Nt, dt=dt, c=c, nx=n, ny=n, nz=nz,
                dx=dx, dy=dx, dz=dz, g=g, balls=balls)


def _scores(p, ref):
    """Correlation deficits (%) in 3-D and of the MIPs along z (xy), y (xz), x (yz)."""
    out = {"3D": 100.0 * (1.0 - float(corrcoef(p, ref)))}
    for name, axis in (("xy", 0), ("xz", 1), ("yz", 2)):
        out[name] = 100.0 * (1.0 - float(corrcoef(nedner.mip(p, axis), nedner.mip(ref, axis))))
    return out


def _timed_forward(plan, g, reps: int):
    import torch
    out = plan.forward(g)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record()
        plan.forward(g, out=out)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return out, float(np.median(ts))


def run(cfg: Optional[Dict] = None, reps: int = 10) -> Dict:
    import torch
    cfg = ball_workload() if cfg is None else cfg
    g = torch.as_tensor(np.asarray(cfg["g"], dtype=np.float32), device="cuda")
    res = {"workload": "%s: %d sensors on the %dx%d output grid, Nt=%d at dt=%.3g s, %dx%dx%d voxels, ball "
                       "radius %.3g m" % (cfg["name"], cfg["sensor_xy"].shape[0], cfg["nx"], cfg["ny"], cfg["Nt"],
                                          cfg["dt"], cfg["nx"], cfg["ny"], cfg["nz"], float(cfg["balls"].radii[0])),
           "rows": []}
    plan = nedner.plan_from_config(cfg, ner_mode="direct")
    ref, t_ref = _timed_forward(plan, g, max(1, reps // 5))
    plan.close()
    res["direct_ms"] = t_ref
    for label, mode, w in METHODS:
        plan = nedner.plan_from_config(cfg, ner_mode=mode, window=("kb", w))
        p, t = _timed_forward(plan, g, reps)
        plan.close()
        res["rows"].append(dict(method=label, ms=round(t, 4), deficit_pct={k: float("%.4g" % v) for k, v in
                                                                           _scores(p, ref).items()}))
    return res


if __name__ == "__main__":
    import json
    from . import build
    build.build()
    print(json.dumps(run()))
