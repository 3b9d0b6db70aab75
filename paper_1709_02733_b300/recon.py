"""Accelerated reconstruction with the matched pair H, H^T.

The paper's outlook (Sec. 8; Sec. 3 on iterative methods that need H and H^T
repeatedly) is penalised least-squares reconstruction with proximal first-order
methods.  ``fista_nn`` minimises 1/2 ||H p - y||^2 subject to p >= 0 with
FISTA (Beck and Teboulle): a projected gradient step at an extrapolated point,

    x_k = max(0, z_k - H^T (H z_k - y) / L),
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
    z_{k+1} = x_k + (t_k - 1) / t_{k+1} (x_k - x_{k-1}),

with L >= ||H||^2.  Each iteration costs one forward and one adjoint solve
(the CUDA kernels behind pact_forward / pact_adjoint); the projection and
the extrapolation are elementwise updates of the image on the device.
Projected gradient descent (``autograd.reconstruct_gd``) is the same step
without the extrapolation.  ``fista_tv`` adds a total-variation penalty
lam TV(p): its proximal step (with p >= 0) is the CUDA fast gradient
projection behind pact_tv_prox_nn.

    python -m paper_1709_02733_b300.recon [iters] [tv_weight]

runs the differentiable-reconstruction workload (skull-192, SNR 30 dB data)
with projected GD, FISTA and FISTA-TV (lam = tv_weight x L, default 1e-5; 20
dual iterations) from
the same start and step size and prints one JSON line per iteration and a
summary.
"""
from __future__ import annotations

import math
from typing import Callable, Optional

import torch

from .pact import Grid


def fista_nn(grid: Grid, rec, nsteps: int, y: torch.Tensor, L: float, iters: int = 50,
             p_init: Optional[torch.Tensor] = None,
             callback: Optional[Callable[[int, torch.Tensor, float], None]] = None) -> torch.Tensor:
    """FISTA with the non-negativity projection; callback(k, x_k, 1/2||H z_k - y||^2)."""
    x_prev = torch.zeros(grid.shape, device="cuda") if p_init is None else p_init.detach().clone().float()
    z = x_prev.clone()
    t = 1.0
    for k in range(iters):
        r = grid.forward(z.contiguous(), rec, nsteps) - y
        loss = 0.5 * float((r.double() ** 2).sum())
        grad = grid.adjoint(r.contiguous(), rec)
        x = (z - grad / L).clamp_(min=0.0)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev, t = x, t_next
        if callback is not None:
            callback(k, x, loss)
    return x_prev


def fista_tv(grid: Grid, rec, nsteps: int, y: torch.Tensor, L: float, lam: float, iters: int = 50, inner: int = 20,
             p_init: Optional[torch.Tensor] = None,
             callback: Optional[Callable[[int, torch.Tensor, float], None]] = None) -> torch.Tensor:
    """FISTA on 1/2 ||H p - y||^2 + lam TV(p) subject to p >= 0: the projection
    of fista_nn becomes the proximal step of (lam / L) TV + (p >= 0), computed
    by pact_tv_prox_nn with `inner` dual iterations."""
    from .pact import pact_tv_prox_nn
    x_prev = torch.zeros(grid.shape, device="cuda") if p_init is None else p_init.detach().clone().float()
    z = x_prev.clone()
    work = torch.empty(6 * z.numel(), device="cuda")
    t = 1.0
    for k in range(iters):
        r = grid.forward(z.contiguous(), rec, nsteps) - y
        loss = 0.5 * float((r.double() ** 2).sum())
        grad = grid.adjoint(r.contiguous(), rec)
        x = pact_tv_prox_nn((z - grad / L).contiguous(), lam / L, inner, work=work)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev, t = x, t_next
        if callback is not None:
            callback(k, x, loss)
    return x_prev


def main():  # pragma: no cover - example runner
    import json
    import sys
    import time

    from . import build, synth
    from .autograd import operator_norm_sq, reconstruct_gd
    build.build()
    iters = int(sys.argv[1]) if len(sys.argv) > 1 else 50
    tv_weight = float(sys.argv[2]) if len(sys.argv) > 2 else 1e-5
    w = synth.skull_192()
    grid = Grid(w.desc)
    grid.set_medium(*[torch.from_numpy(m).cuda() for m in w.medium])
    p_true = torch.from_numpy(w.p0).cuda()
    y0 = grid.forward(p_true, w.rec, w.nsteps)
    sigma = float(y0.pow(2).mean().sqrt()) * 10 ** (-1.5)
    y = y0 + sigma * torch.randn(y0.shape, generator=torch.Generator().manual_seed(4)).cuda()
    lam = operator_norm_sq(grid, w.rec, w.nsteps, iters=10)
    L = 1.05 * lam
    pn = float(p_true.norm())
    runs = {}
    for name in ("gd", "fista", "fista_tv"):
        errs, losses = [], []

        def cb(k, p, loss, name=name, errs=errs, losses=losses):
            errs.append(float((p.detach() - p_true).norm()) / pn)
            losses.append(loss)
            print(json.dumps({"method": name, "iter": k, "loss": loss, "rel_err": errs[-1]}), flush=True)

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if name == "gd":
            reconstruct_gd(grid, w.rec, w.nsteps, y, iters=iters, eta=1.0 / L, callback=cb)
        elif name == "fista":
            fista_nn(grid, w.rec, w.nsteps, y, L, iters=iters, callback=cb)
        else:
            fista_tv(grid, w.rec, w.nsteps, y, L, tv_weight * L, iters=iters, inner=20, callback=cb)
        torch.cuda.synchronize()
        runs[name] = {"wall_s": time.perf_counter() - t0, "rel_err": errs, "loss": losses}
    grid.close()
    summary = {"workload": "skull-192: 192^3, 1500 steps, 256 receivers, SNR 30 dB", "iters": iters,
               "L": L, "power_iteration_lambda": lam, "tv_lambda": tv_weight * L}
    for name, r in runs.items():
        summary[name] = {"wall_s": r["wall_s"], "s_per_iter": r["wall_s"] / iters, "final_rel_err": r["rel_err"][-1],
                         "first_loss": r["loss"][0], "last_loss": r["loss"][-1]}
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":  # pragma: no cover
    main()
