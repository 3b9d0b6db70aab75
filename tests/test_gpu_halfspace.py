"""Validation of H against the exact solution of Sec. 5: a line source in water
over a lossless elastic solid, pressure at a receiver in the water.

The exact trace is oracle/halfspace.py (Cagniard-de Hoop, pinned in
tests/test_halfspace_pins.py); the FDTD run is the y-invariant 3-D problem on
the paper's x-z box (58.2 mm, dx 0.15 mm, 4.5 mm C-PML) with a y extent long
enough that the ends of the line source cannot reach the receiver within the
window (c_p t_end below the distance to the end of the line), sampled at
40 MHz (every second step; sample m of the operator stands for (m + 1/2) dt).

    python tests/test_gpu_halfspace.py [ny] [refine]

runs the comparison at a chosen y extent (2312 = the paper's 346.8 mm) and
grid refinement (2 = dx / 2 on a correspondingly larger grid) and prints one
JSON line; at refine 1 a second line holds the inner-product test of H and
H^T on the same grid.
"""
import json
import math
import os
import sys
import time

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import halfspace as hs  # noqa: E402
from paper_1709_02733_b300 import synth  # noqa: E402


def fdtd_trace(case):
    import torch
    from paper_1709_02733_b300 import pact
    d = case.desc
    g = pact.Grid(d)

    def ex(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()[:, None, :].expand(d.nz, d.ny, d.nx).contiguous()

    g.set_medium(ex(case.rho), ex(case.lam), ex(case.mu), ex(case.alpha))
    p0 = torch.zeros(d.shape, device="cuda")
    j0, j1 = case.p0_y
    p0[:, j0:j1, :] = torch.from_numpy(case.p0).cuda()[:, None, :]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr = g.forward(p0, case.rec, case.nsteps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = tr.cpu().numpy()[:, 0].astype(np.float64)
    g.close()
    del p0
    torch.cuda.empty_cache()
    return out, wall


_EXACT = {}


def exact_trace(case, every):
    """Exact pressure at the times the kept samples stand for, (m + 1/2) dt:
    these differ between grid refinements, so the cache is keyed on them."""
    p = case.params
    t = (np.arange(0, case.nsteps + 1, every) + 0.5) * case.desc.dt
    key = (tuple(sorted(p.items())), t.tobytes())
    if key not in _EXACT:
        m = hs.HalfSpace.from_lame(p["rho_f"], p["lam_f"], p["rho_s"], p["lam_s"], p["mu_s"])
        src = hs.LineSource(0.0, p["h_t"], p["sigma"], p["taper"])
        _EXACT[key] = (t, hs.pressure_trace(t, p["d"], p["h_r"], src, m))
    return _EXACT[key]


def compare(ny=544, refine=1, t_end=10e-6):
    case = synth.halfspace(ny=ny * refine, n_xz=388 * refine, dx=0.15e-3 / refine, npml=30 * refine,
                           dt=12.5e-9 / refine, t_end=t_end)
    # the ends of the line stay out of the receiver's domain of dependence
    c_p = math.sqrt((case.params["lam_s"] + 2 * case.params["mu_s"]) / case.params["rho_s"])
    reach = (case.rec[0, 1] - case.p0_y[0]) * case.desc.dx
    assert c_p * t_end < reach, (c_p * t_end, reach)
    every = 2 * refine                                  # 40 MHz samples
    t, exact = exact_trace(case, every)
    fd, wall = fdtd_trace(case)
    fd = fd[::every]
    err = fd - exact
    peak = np.abs(exact).max()
    d = case.desc
    return {"grid": [d.nx, d.ny, d.nz], "dx_mm": d.dx * 1e3, "dt_ns": d.dt * 1e9, "nsteps": case.nsteps,
            "samples_40MHz": int(t.size), "rel_l2": float(np.linalg.norm(err) / np.linalg.norm(exact)),
            "max_err_over_peak": float(np.abs(err).max() / peak), "peak": float(peak),
            "updates_per_s": d.N * case.nsteps / wall, "fdtd_wall_s": wall,
            "t_us": (t[::20] * 1e6).tolist(), "exact": exact[::20].tolist(), "fdtd": fd[::20].tolist()}


def inner_product(ny=544, L=64, seed=5):
    """Sec. 5's adjoint check on the validation problem: <H f, g> against
    <f, H^T g> with f the validation p0 and g = H f + 10 % white noise (so
    that <H f, g> is not small), L seeded receivers in the water; both sums in
    FP64 on the host."""
    import torch
    from paper_1709_02733_b300 import pact
    case = synth.halfspace(ny=ny)
    d = case.desc
    rng = np.random.default_rng(seed)
    lo, hi = d.npml + 2, d.nx - d.npml - 3
    rec = np.stack([rng.uniform(lo, hi, L), rng.uniform(lo, d.ny - d.npml - 3, L),
                    rng.uniform(case.k0 + 1, hi, L)], axis=1).astype(np.float32)
    g = pact.Grid(d)

    def ex(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()[:, None, :].expand(d.nz, d.ny, d.nx).contiguous()

    g.set_medium(ex(case.rho), ex(case.lam), ex(case.mu), ex(case.alpha))
    p0 = torch.zeros(d.shape, device="cuda")
    j0, j1 = case.p0_y
    p0[:, j0:j1, :] = torch.from_numpy(case.p0).cuda()[:, None, :]
    tr = g.forward(p0, rec, case.nsteps).cpu().numpy().astype(np.float64)
    y = (tr + 0.1 * np.sqrt(np.mean(tr ** 2)) * rng.standard_normal(tr.shape)).astype(np.float32)
    img = g.adjoint(torch.from_numpy(y).cuda(), rec)
    # <f, H^T g> over the grid in FP64 on the device, summed per plane on the host
    rhs = float(sum(torch.sum(p0[k].double() * img[k].double()).item() for k in range(d.nz)))
    lhs = float(np.sum(tr * y.astype(np.float64)))
    g.close()
    del p0, img
    torch.cuda.empty_cache()
    return {"grid": [d.nx, d.ny, d.nz], "receivers": L, "nsteps": case.nsteps, "lhs": lhs, "rhs": rhs,
            "rel_diff": abs(lhs - rhs) / abs(lhs)}


_RESULTS = {}


def _run(refine):
    if refine not in _RESULTS:
        from paper_1709_02733_b300 import build
        build.build()
        _RESULTS[refine] = compare(ny=544, refine=refine)
    return _RESULTS[refine]


@pytest.mark.gpu
def test_halfspace_matches_cagniard_de_hoop():
    """At the paper's dx (0.15 mm, 6.7 cells per sigma) the trace matches the
    exact one to 0.29 % (relative L2) and 0.32 % of the peak (measured on a
    B300); the bound leaves a factor of two for the FP32 rounding order of a
    different launch configuration.  The error is discretisation error: it
    falls under refinement (next test)."""
    r = _run(1)
    assert r["rel_l2"] < 0.006, r
    assert r["max_err_over_peak"] < 0.006, r


@pytest.mark.gpu
def test_halfspace_error_falls_under_refinement():
    """dx / 2 (776 x 1088 x 776, 1600 steps): the error drops by more than 2x
    (measured 2.7x in L2, 3.5x in the maximum)."""
    r1, r2 = _run(1), _run(2)
    assert r2["rel_l2"] < r1["rel_l2"] / 2, (r1["rel_l2"], r2["rel_l2"])
    assert r2["max_err_over_peak"] < r1["max_err_over_peak"] / 2, (r1["max_err_over_peak"], r2["max_err_over_peak"])


@pytest.mark.gpu
def test_halfspace_inner_product():
    """The paper reports agreement to 6 digits; FP32 on the validation grid
    (388 x 544 x 388, 800 steps, 64 receivers) is held to 1e-5, the bound of
    the other FP32 inner-product tests."""
    from paper_1709_02733_b300 import build
    build.build()
    r = inner_product(ny=544)
    assert r["rel_diff"] <= 1e-5, r


if __name__ == "__main__":
    from paper_1709_02733_b300 import build
    build.build()
    ny = int(sys.argv[1]) if len(sys.argv) > 1 else 2312
    refine = int(sys.argv[2]) if len(sys.argv) > 2 else 1
    print(json.dumps(compare(ny=ny, refine=refine)), flush=True)
    if refine == 1:
        print(json.dumps(inner_product(ny=ny)), flush=True)
