"""Non-inverse-crime reconstruction: data from a finer discretisation.

The paper's simulation study (Sec. 6.2) avoids the inverse crime by simulating
the data on a finer grid than the one the operator pair reconstructs on, and by
adding noise.  This module does the same with the seeded skull-like stand-ins:

- a coarse grid (spacing dx) and a fine grid (spacing 3/4 dx) cover the same
  physical box, with the same physical layer depth, skull geometry and
  receiver positions; the fine medium and the initial pressure are rasterised
  from the same analytic skull and seeded vessel geometry at the fine
  resolution;
- the fine forward operator records the traces, one sample per fine step;
- the traces are resampled in time to the coarse operator's samples
  (``pact_resample_traces``; sample k of an operator with step dt stands for
  the time (k + 1/2) dt, so coarse sample k sits at fine sample
  (k + 1/2) dt_c / dt_f - 1/2), and white noise of 5 % of the maximum trace
  amplitude is added;
- the coarse pair reconstructs: the adjoint image H^T y and FISTA with
  non-negativity.

The result is compared with the same reconstructions from inverse-crime data
(simulated with the coarse operator itself, same noise level).

    python -m paper_1709_02733_b300.pipeline [n_coarse] [fista_iters]
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import synth
from .pact import Grid, pact_resample_traces


@dataclass
class Study:
    coarse: synth.Workload      # the reconstruction grid (its p0 is the fine p0 resampled to it)
    fine: synth.Workload        # the data grid
    y: torch.Tensor             # noisy traces on the coarse time axis (device)
    y_crime: torch.Tensor       # noisy traces simulated on the coarse grid itself (device)
    noise_sigma: float


def resample_volume(v: np.ndarray, n_out: int) -> np.ndarray:
    """Trilinear resampling of a cubic volume onto another grid over the same
    box (node-centred: node i of n sits at i / (n - 1) of the box)."""
    from scipy.ndimage import map_coordinates
    n_in = v.shape[0]
    s = np.arange(n_out) * (n_in - 1) / (n_out - 1)
    zz, yy, xx = np.meshgrid(s, s, s, indexing="ij")
    return map_coordinates(v.astype(np.float64), [zz, yy, xx], order=1).astype(np.float32)


def make_study(n_coarse: int = 96, dx: float = 0.8e-3, npml: int = 6, nsteps: int = 600, L: int = 256,
               seed: int = 7, noise_frac: float = 0.05) -> Study:
    """Coarse grid n_coarse^3 at dx; fine grid at 3/4 dx over the same box
    (n_coarse must be a multiple of 4 and npml of 3)."""
    if n_coarse % 4 or npml % 3:
        raise ValueError("n_coarse must be a multiple of 4 and npml of 3 (fine grid 4/3 finer)")
    n_f, dx_f, npml_f = n_coarse * 4 // 3, dx * 0.75, npml * 4 // 3
    coarse = synth.skull(n_coarse, dx, npml, nsteps, L, seed, name=f"coarse-{n_coarse}")
    fine0 = synth.skull(n_f, dx_f, npml_f, 1, L, seed, name=f"fine-{n_f}")
    dt_c, dt_f = coarse.desc.dt, fine0.desc.dt
    T = (nsteps + 0.5) * dt_c                             # last coarse sample time
    nsteps_f = int(math.ceil(T / dt_f)) + 1
    fine = synth.Workload(fine0.name, fine0.desc, nsteps_f, fine0.rho, fine0.lam, fine0.mu, fine0.alpha, fine0.p0,
                          fine0.rec)
    # the truth is the fine initial pressure; the coarse grid's p0 is its resampling
    coarse.p0 = resample_volume(fine.p0, n_coarse)
    # fine data
    g_f = Grid(fine.desc)
    g_f.set_medium(*[torch.from_numpy(m).cuda() for m in fine.medium])
    tr_f = g_f.forward(torch.from_numpy(fine.p0).cuda(), fine.rec, nsteps_f)
    torch.cuda.synchronize()
    g_f.close()
    ratio = dt_c / dt_f
    y0 = pact_resample_traces(tr_f, nsteps + 1, 0.5 * ratio - 0.5, ratio)
    sigma = noise_frac * float(y0.abs().max())
    gen = torch.Generator().manual_seed(seed + 100)
    y = y0 + sigma * torch.randn(y0.shape, generator=gen).cuda()
    # inverse-crime data on the coarse grid, same noise level
    g_c = Grid(coarse.desc)
    g_c.set_medium(*[torch.from_numpy(m).cuda() for m in coarse.medium])
    yc0 = g_c.forward(torch.from_numpy(coarse.p0).cuda(), coarse.rec, nsteps)
    y_crime = yc0 + sigma * torch.randn(yc0.shape, generator=gen).cuda()
    torch.cuda.synchronize()
    g_c.close()
    return Study(coarse, fine, y, y_crime, sigma)


def main():  # pragma: no cover - example runner
    import json
    import sys
    import time

    from . import build
    from .autograd import operator_norm_sq
    from .recon import fista_nn
    build.build()
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 96
    iters = int(sys.argv[2]) if len(sys.argv) > 2 else 20
    t0 = time.perf_counter()
    st = make_study(n_coarse=n)
    t_data = time.perf_counter() - t0
    c = st.coarse
    g = Grid(c.desc)
    g.set_medium(*[torch.from_numpy(m).cuda() for m in c.medium])
    p_true = torch.from_numpy(c.p0).cuda()
    pn = float(p_true.norm())
    L = 1.05 * operator_norm_sq(g, c.rec, c.nsteps, iters=10)
    out = {"coarse": f"{n}^3, dx {c.desc.dx * 1e3:.3g} mm, {c.nsteps} steps",
           "fine": f"{st.fine.desc.nx}^3, dx {st.fine.desc.dx * 1e3:.3g} mm, {st.fine.nsteps} steps",
           "receivers": int(c.rec.shape[0]), "noise_sigma": st.noise_sigma, "data_seconds": t_data}
    for name, y in (("fine_data", st.y), ("inverse_crime", st.y_crime)):
        img = g.adjoint(y, c.rec)
        a = float(torch.dot(img.flatten().double(), p_true.flatten().double()))
        scale = a / float(img.double().pow(2).sum())
        err_adj = float((scale * img - p_true).norm()) / pn
        corr = a / (float(img.double().norm()) * pn)
        t1 = time.perf_counter()
        x = fista_nn(g, c.rec, c.nsteps, y, L, iters=iters)
        torch.cuda.synchronize()
        out[name] = {"adjoint_corr": corr, "adjoint_scaled_rel_err": err_adj,
                     "fista_rel_err": float((x - p_true).norm()) / pn,
                     "fista_residual": float((g.forward(x, c.rec, c.nsteps) - y).norm()) / float(y.norm()),
                     "fista_seconds": time.perf_counter() - t1}
    g.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":  # pragma: no cover
    main()
