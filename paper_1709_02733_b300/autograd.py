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
            callback(it, p, float(loss.detach()))
    return p.detach()


def _smooth3(v: torch.Tensor, sigma: float) -> torch.Tensor:
    """Separable Gaussian smoothing of a 3-D tensor (zero padding)."""
    r = int(3 * sigma + 0.5)
    t = torch.arange(-r, r + 1, device=v.device, dtype=v.dtype)
    k = torch.exp(-0.5 * (t / sigma) ** 2)
    k = (k / k.sum()).view(1, 1, -1)
    out = v
    for axis in range(3):
        x = out.movedim(axis, -1)
        shp = x.shape
        x = torch.nn.functional.conv1d(x.reshape(-1, 1, shp[-1]), k, padding=r).reshape(shp)
        out = x.movedim(-1, axis)
    return out.contiguous()


def fd_check(grid: Grid, rec, nsteps: int, p: torch.Tensor, y: torch.Tensor, ndir: int = 16,
             seed: int = 4, sigma: float = 2.0):
    """Compare <grad L, d> (autograd, i.e. H^T) with the central difference
    (L(p + d) - L(p - d)) / 2 of L = 1/2 ||H p - y||^2 on ndir seeded random
    directions d (white noise smoothed over sigma cells, the scale of the
    image's features, and scaled to ||p||).  L is quadratic, so the central
    difference is exact up to the round-off of the FP32 forward solves.
    Returns per direction (|fd - an| / |fd|, |fd - an| / (||grad|| ||d||))."""
    def loss_of(q):
        r = grid.forward(q.contiguous(), rec, nsteps).double() - y.double()
        return 0.5 * float((r ** 2).sum())

    q = p.detach().clone().requires_grad_(True)
    r = pact_forward_op(q, grid, rec, nsteps) - y
    (0.5 * (r.double() ** 2).sum()).backward()
    grad = q.grad.detach()
    gnorm = float(grad.double().norm())
    gen = torch.Generator().manual_seed(seed)
    rel, nrm = [], []
    for _ in range(ndir):
        d = _smooth3(torch.randn(p.shape, generator=gen).cuda(), sigma)
        d *= float(p.norm()) / float(d.norm())
        fd = 0.5 * (loss_of(p + d) - loss_of(p - d))
        an = float(torch.dot(grad.flatten().double(), d.flatten().double()))
        rel.append(abs(fd - an) / max(abs(fd), 1e-300))
        nrm.append(abs(fd - an) / max(gnorm * float(d.double().norm()), 1e-300))
    return rel, nrm


def main():  # pragma: no cover - example runner
    """Differentiable-reconstruction workload: 192^3 skull-like medium, 1500
    steps, 256 receivers, data at SNR 30 dB; finite-difference check of the
    autograd gradient on 16 random directions, then 50 projected GD
    iterations with eta = 1 / ||H||^2.  Prints one JSON line per iteration and a summary line."""
    import json
    import sys
    import time

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
    fd, fdn = fd_check(grid, w.rec, w.nsteps, 0.5 * p_true, y)
    print(json.dumps({"fd_directions": len(fd), "fd_max_rel_diff": max(fd), "fd_max_normalised_diff": max(fdn)}),
          flush=True)
    errs: List[float] = []
    losses: List[float] = []
    pn = float(p_true.norm())

    def cb(it, p, loss):
        errs.append(float((p.detach() - p_true).norm()) / pn)
        losses.append(loss)
        print(json.dumps({"iter": it, "loss": loss, "rel_err": errs[-1]}), flush=True)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reconstruct_gd(grid, w.rec, w.nsteps, y, iters=iters, callback=cb)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    grid.close()
    print(json.dumps({"workload": "skull-192: 192^3, 1500 steps, 256 receivers, SNR 30 dB", "iters": iters,
                      "fd_max_rel_diff": max(fd), "fd_max_normalised_diff": max(fdn), "loss_first": losses[0] if losses else math.nan,
                      "loss_last": losses[-1] if losses else math.nan,
                      "rel_err_first": errs[0] if errs else math.nan, "final_rel_err": errs[-1] if errs else math.nan,
                      "gd_wall_s": wall}))


if __name__ == "__main__":  # pragma: no cover
    main()
