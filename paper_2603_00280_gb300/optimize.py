"""Inverse rendering of a GPSS object: fits the mean, variance, albedo and length
scale of a single-object scene to a target image with Adam, through the
differentiable renderer (``gpss.render_differentiable``: the forward render and
the path-replay adjoint of the C-ABI library).  PyTorch holds the parameters and
runs the optimiser; every render and gradient is the library's.

Parameterisation: the mean grid and the albedo grid directly (the albedo clamped
to [0, 1] after each step), the variance through its logarithm (it must stay
positive and spans two orders of magnitude), the length scale through its
logarithm.  Loss: the mean squared difference to the target image.
"""
from __future__ import annotations

import math
import time

from . import gpss


def fit(start: dict, target, camera: dict, opts: dict, steps: int = 30, lr_mean: float = 2e-3,
        lr_log_var: float = 0.05, lr_albedo: float = 0.02, lr_log_l: float = 0.02, seed0: int = 1, callback=None):
    """Runs `steps` Adam iterations from the single-object scene `start` (a scene
    dictionary of workloads.py) toward the (H, W, 3) CUDA tensor `target`.  Each
    iteration renders with its own seed (seed0 + i).  Returns a dict with the
    per-iteration losses, the final parameter tensors and the milliseconds per
    iteration (over the iterations after the first, whose time -- the library's and
    PyTorch's first-use set-up -- is returned apart as first_iteration_ms); callback(i,
    loss, params) is called after each step."""
    import torch

    obj = start["objects"][0]
    S = gpss.Scene(start)
    mean = torch.tensor(obj["mean"], device="cuda", dtype=torch.float32, requires_grad=True)
    log_var = torch.tensor(obj["var"], device="cuda", dtype=torch.float32).log().requires_grad_(True)
    albedo = torch.tensor(obj["albedo"], device="cuda", dtype=torch.float32, requires_grad=True)
    log_l = torch.tensor(math.log(obj["length_scale"]), device="cuda", dtype=torch.float32, requires_grad=True)
    opt = torch.optim.Adam([{"params": [mean], "lr": lr_mean}, {"params": [log_var], "lr": lr_log_var},
                            {"params": [albedo], "lr": lr_albedo}, {"params": [log_l], "lr": lr_log_l}])
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t1 = t0
    for i in range(steps):
        if i == 1:
            torch.cuda.synchronize()
            t1 = time.perf_counter()
        opt.zero_grad(set_to_none=True)
        img = gpss.render_differentiable(S, obj, mean, log_var.exp(), albedo, log_l.exp(), camera,
                                         dict(opts, seed=seed0 + i))
        loss = ((img - target) ** 2).mean()
        loss.backward()
        opt.step()
        with torch.no_grad():
            albedo.clamp_(0.0, 1.0)
        losses.append(float(loss))
        if callback is not None:
            with torch.no_grad():
                callback(i, losses[-1], {"mean": mean.detach(), "var": log_var.detach().exp(), "albedo": albedo.detach(),
                                         "l": log_l.detach().exp()})
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ms = 1e3 * (t2 - t1) / max(steps - 1, 1) if steps > 1 else 1e3 * (t2 - t0)
    S.close()
    return {"losses": losses, "mean": mean.detach(), "var": log_var.detach().exp(), "albedo": albedo.detach(),
            "length_scale": float(log_l.detach().exp()), "ms_per_iteration": ms,
            "first_iteration_ms": 1e3 * (t1 - t0) if steps > 1 else ms}
