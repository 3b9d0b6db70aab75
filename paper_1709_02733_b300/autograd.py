"""Differentiable forward operator: torch.autograd.Function around H.

forward(p0) = H p0 through pact_forward; backward(g) = H^T g through
pact_adjoint.  H is linear in p0, so the backward pass needs no stored
wavefield (no checkpointing): the adjoint recursion of Sec. 4 (Eq. (Adjup))
recomputes everything from the incoming trace gradient.  The medium and the
receivers are constants (not differentiated).

Least-squares reconstruction (Sec. 2.3: H and H^T inside an iterative method
that minimises a data-fidelity functional; Sec. 8 names penalised least
squares as the intended use) is in ``reconstruct_gd``: projected gradient
descent p <- max(0, p - eta grad) on 1/2 ||H p - y||^2 with eta = 1 / ||H||^2,
||H||^2 from power iteration on H^T H.
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional

import torch

from .pact import Grid


class PactForward(torch.autograd.Function):
    """traces = H p0 with d(traces)/d(p0) applied as H^T."""

    @staticmethod
    def forward(ctx, p0: torch.Tensor, grid: Grid, rec, nsteps: int) -> torch.Tensor:
        ctx.grid = grid
        ctx.rec = rec
        return grid.forward(p0.detach().contiguous(), rec, int(nsteps))

    @staticmethod
    def backward(ctx, grad_traces: torch.Tensor):
        img = ctx.grid.adjoint(grad_traces.detach().contiguous().float(), ctx.rec)
        return img, None, None, None


def pact_forward_op(p0: torch.Tensor, grid: Grid, rec, nsteps: int) -> torch.Tensor:
    """Differentiable H p0 (float32 CUDA tensor of the grid's shape)."""
    return PactForward.apply(p0, grid, rec, nsteps)


def operator_norm_sq(grid: Grid, rec, nsteps: int, iters: int = 10, seed: int = 0) -> float:
    """||H||^2 = largest eigenvalue of H^T H by power iteration."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.randn(grid.shape, generator=g).cuda()
    v /= v.norm()
    lam = 0.0
    for _ in range(iters):
        w = grid.adjoint(grid.forward(v, rec, nsteps), rec)
        lam = float(torch.dot(v.flatten().double(), w.flatten().double()))
        v = w / w.norm()
    return lam


def reconstruct_gd(grid: Grid, rec, nsteps: int, y: torch.Tensor, iters: int = 50, eta: Optional[float] = None,
                   p_init: Optional[torch.Tensor] = None, nonneg: bool = True,
                   callback: Optional[Callable[[int, torch.Tensor, float], None]] = None) -> torch.Tensor:
    """Projected gradient descent on 1/2 ||H p - y||^2 with gradients from autograd."""
    if eta is None:
        eta = 1.0 / operator_norm_sq(grid, rec, nsteps)
    p = torch.zeros(grid.shape, device="cuda") if p_init is None else p_init.clone()
    for it in range(iters):
        p.requires_grad_(True)
        r = pact_forward_op(p, grid, rec, nsteps) - y
        loss = 0.5 * (r.double() ** 2).sum()
        loss.backward()
        with torch.no_grad():
            p = p - eta * p.grad
            if nonneg:
                p.clamp_(min=0.0)
        if callback is not None:
            callback(it, p, float(loss))
    return p.detach()


def main():  # pragma: no cover - example runner
    """Differentiable-reconstruction workload: 192^3 skull-like medium, 1500
    steps, 256 receivers, data at SNR 30 dB, 50 projected GD iterations."""
    import json
    import sys

    from . import build, synth
    build.build()
    w = synth.skull_192()
    iters = int(sys.argv[1]) if len(sys.argv) > 1 else 50
    grid = Grid(w.desc)
    grid.set_medium(*[torch.from_numpy(m).cuda() for m in w.medium])
    p_true = torch.from_numpy(w.p0).cuda()
    y0 = grid.forward(p_true, w.rec, w.nsteps)
    sigma = float(y0.pow(2).mean().sqrt()) * 10 ** (-1.5)
    y = y0 + sigma * torch.randn(y0.shape, generator=torch.Generator().manual_seed(4)).cuda()
    errs: List[float] = []
    pn = float(p_true.norm())

    def cb(it, p, loss):
        errs.append(float((p - p_true).norm()) / pn)
        print(json.dumps({"iter": it, "loss": loss, "rel_err": errs[-1]}), flush=True)

    reconstruct_gd(grid, w.rec, w.nsteps, y, iters=iters, callback=cb)
    grid.close()
    print(json.dumps({"final_rel_err": errs[-1] if errs else math.nan}))


if __name__ == "__main__":  # pragma: no cover
    main()
