"""Model-based reconstruction and sensor placement on top of the NEDNER
operators (the differentiation workload).

The paper reconstructs with the inversion formula alone (Sec. 2-3).  Because
that map R and its transpose R^T are linear and available as a
differentiable pair (``nedner.reconstruct`` / ``nedner.model``), two uses
follow directly:

* ``fit_p0``: least-squares fit  min_f || A f - g ||^2  with A = R^T of an
  unweighted plan (the physical forward model: plane-wave expansion of the
  wave equation's solution sampled at the sensors), by conjugate gradients on
  the normal equations or by Adam on the loss through autograd;
* ``placement_step``: one gradient step on the movable sensor positions for a
  reconstruction loss L(R(x) g), the question of Sec. 6 (where to put a
  limited number of sensors) posed as an optimisation.

All operator applications run in the CUDA library; torch only does the
vector updates.
"""
from __future__ import annotations

from typing import Dict, List, Optional

import numpy as np

from . import nedner


def fit_p0(plan_unweighted: "nedner.Plan", g, iters: int = 50, method: str = "cg", lr: float = 1e-2,
           f0=None) -> Dict:
    """Least-squares fit of the initial pressure to data g.

    plan_unweighted: a plan built with apply_weights=False (A = its adjoint).
    Returns {"f": tensor, "residual": [||A f_k - g||, k = 0..iters]}.
    """
    import torch
    dev = g.device
    shape = (plan_unweighted.nz, plan_unweighted.ny, plan_unweighted.nx)
    f = torch.zeros(shape, dtype=torch.float32, device=dev) if f0 is None else f0.clone()
    res: List[float] = []
    if method == "cg":
        # CG on A^T A f = A^T g (CGNR)
        r = g - plan_unweighted.adjoint(f)
        s = plan_unweighted.forward(r)
        p = s.clone()
        gamma = float((s.double() * s.double()).sum())
        res.append(float(r.double().norm()))
        for _ in range(iters):
            q = plan_unweighted.adjoint(p)
            qq = float((q.double() * q.double()).sum())
            if qq == 0.0 or gamma == 0.0:
                res.append(res[-1])
                continue
            alpha = gamma / qq
            f = f + alpha * p
            r = r - alpha * q
            s = plan_unweighted.forward(r)
            gamma_new = float((s.double() * s.double()).sum())
            p = s + (gamma_new / gamma) * p
            gamma = gamma_new
            res.append(float(r.double().norm()))
    elif method == "adam":
        f = f.requires_grad_(True)
        opt = torch.optim.Adam([f], lr=lr)
        for k in range(iters + 1):
            opt.zero_grad()
            resid = nedner.model(plan_unweighted, f) - g
            loss = 0.5 * (resid * resid).sum()
            res.append(float(resid.detach().double().norm()))
            if k == iters:
                break
            loss.backward()
            opt.step()
        f = f.detach()
    else:
        raise ValueError(method)
    return {"f": f, "residual": res}


def placement_step(plan: "nedner.Plan", g, target, sensor_xy, movable, lr: float) -> Dict:
    """One gradient step on the movable sensors for L = ||R(x) g - target||^2 / 2.

    sensor_xy: (M, 2) float64 tensor (metres); movable: (M,) bool mask.
    Returns {"loss": float, "grad": (M, 2) tensor, "xy": new positions}.
    """
    import torch
    xy = sensor_xy.detach().clone().requires_grad_(True)
    p0 = nedner.reconstruct(plan, g, xy)
    loss = 0.5 * ((p0 - target) ** 2).sum()
    loss.backward()
    grad = xy.grad * movable[:, None].to(xy.grad.dtype)
    X = plan.nx * plan.grid[3]
    Y = plan.ny * plan.grid[4]
    new = (xy.detach() - lr * grad).clone()
    new[:, 0] = new[:, 0].clamp(-0.5 * X * 0.999, 0.5 * X * 0.999)
    new[:, 1] = new[:, 1].clamp(-0.5 * Y * 0.999, 0.5 * Y * 0.999)
    return {"loss": float(loss.detach()), "grad": grad, "xy": new}


__all__ = ["fit_p0", "placement_step"]
