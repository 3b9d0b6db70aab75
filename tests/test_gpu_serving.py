"""Serving on the GPU: solves advanced together by pact_advance (small grids
on the persistent multi-instance kernels, large ones on their own step
graphs) give the same results as the same solves alone and as the FP64
oracle's H and H^T (Appendix A.3, Eqs. (HPML) and (AdjupPML)), and a queued
stream served with continuous batching completes with correct results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_02733_b300 import pact, synth  # noqa: E402
from paper_1709_02733_b300.serving import InputCache, make_stream, run_continuous, run_one_at_a_time  # noqa: E402
from paper_1709_02733_b300.synth import GridDesc  # noqa: E402

TOL_MIX = 1e-6
TOL_ORACLE = 1e-4  # FP32 kernels against the FP64 oracle, relative L2


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1709_02733_b300 import build
    build.build()


def _random(shape, npml, seed, L):
    rho, lam, mu, al, vmax = synth.random_medium(shape, seed)
    nz, ny, nx = shape
    d = GridDesc(nx, ny, nz, 1e-3, 0.3e-3 / vmax, npml=npml, pml_vmax=vmax)
    rng = np.random.default_rng(seed)
    return d, (rho, lam, mu, al), rng.standard_normal(shape).astype(np.float32), synth.random_receivers(L, shape, seed)


def _mix_cases():
    w = synth.skull(48, 1.2e-3, 6, 60, 40, seed=21)
    cases = [("fwd", w.desc, w.medium, w.p0, w.rec, 60)]
    d, med, p0, rec = _random((36, 44, 40), 3, 22, 17)
    cases.append(("fwd", d, med, p0, rec, 45))
    d, med, p0, rec = _random((48, 56, 64), 4, 23, 21)
    cases.append(("adj", d, med, p0, rec, 38))
    wp = synth.plain_fluid_64(npml=3, nsteps=50)
    cases.append(("adj", wp.desc, wp.medium, wp.p0, wp.rec, 50))
    # grids with interior, z-slab, edge and corner work items
    d, med, p0, rec = _random((40, 44, 104), 4, 24, 19)
    cases.append(("fwd", d, med, p0, rec, 41))
    d, med, p0, rec = _random((52, 37, 100), 5, 25, 23)
    cases.append(("adj", d, med, p0, rec, 47))
    return cases


def _serve_mix(cases, k=7):
    """Begin every case on its own handle, advance them all together with
    pact_advance (k steps per call) and return, per case, the input, the
    served result and the same solve run alone."""
    grids, out = [], []
    rng = np.random.default_rng(3)
    for kind, d, med, p0, rec, ns in cases:
        g = pact.Grid(d)
        g.set_medium(*[cuda(m) for m in med])
        if kind == "fwd":
            inp = cuda(p0)
            ref = g.forward(inp, rec, ns).cpu().numpy()
            res = torch.full((ns + 1, rec.shape[0]), float("nan"), device="cuda")
        else:
            inp = cuda(rng.standard_normal((ns + 1, rec.shape[0])))
            ref = g.adjoint(inp, rec).cpu().numpy()
            res = torch.full(d.shape, float("nan"), device="cuda")
        g.begin(kind == "adj", inp, rec, ns, res)
        grids.append(g)
        out.append((inp, res, ref))
    for _ in range(100):
        if all(g.poll() >= c[5] for g, c in zip(grids, cases)):
            break
        pact.pact_advance(grids, k)
    torch.cuda.synchronize()
    served = [(inp.cpu().numpy(), res.cpu().numpy(), ref) for inp, res, ref in out]
    for g in grids:
        g.close()
    return served


# pact_advance steps grids of at least PACT_SERVE_SOLO_POINTS points on their
# own step kernels and the rest on the multi-instance kernels: "150000" sends
# four of the six cases to their own kernels and two to the multi-instance
# ones, "-1" all to the multi-instance kernels
SPLITS = [None, "150000", "-1"]


@pytest.mark.parametrize("split", SPLITS)
def test_mixed_solves_match_solo(split, monkeypatch):
    if split is not None:
        monkeypatch.setenv("PACT_SERVE_SOLO_POINTS", split)
    cases = _mix_cases()
    for (kind, *_rest), (_inp, got, ref) in zip(cases, _serve_mix(cases)):
        assert np.all(np.isfinite(got)), kind
        assert rel_l2(got, ref) <= TOL_MIX, kind


@pytest.mark.parametrize("split", SPLITS[1:])
def test_served_results_match_oracle(split, monkeypatch):
    """Every solve of a served mix (forward and adjoint instances, on grids
    holding interior, z-slab, edge and corner work items) against the FP64
    oracle's H p0 / H^T y on the same inputs: this covers the persistent
    multi-instance step kernels and the multi-instance receiver kernel
    (sampling, and injection weighted by 3 lambda + 2 mu in the adjoint's
    variables)."""
    from oracle import Oracle
    monkeypatch.setenv("PACT_SERVE_SOLO_POINTS", split)
    cases = _mix_cases()
    kinds = {c[0] for c in cases}
    assert kinds == {"fwd", "adj"}
    for (kind, d, med, p0, rec, ns), (inp, got, _ref) in zip(cases, _serve_mix(cases, k=5)):
        o = Oracle(d.as_dict(), *med)
        want = o.forward(p0, rec, ns) if kind == "fwd" else o.adjoint(inp, rec)
        assert np.all(np.isfinite(got)), kind
        assert np.linalg.norm(want) > 0, kind
        assert rel_l2(got, want) <= TOL_ORACLE, (kind, d.shape, rel_l2(got, want))


def test_continuous_batching_stream():
    """A small seeded stream under a budget that admits only part of it at a
    time: every request completes and equals its one-at-a-time result."""
    kw = dict(rate=200.0, seed=7, n_range=(96, 128), n_step=16, steps_range=(60, 160), L_range=(32, 96))
    reqs = make_stream(10, **kw)
    reqs2 = make_stream(10, **kw)
    cache = InputCache()
    from paper_1709_02733_b300.serving import request_bytes
    budget = 3 * max(request_bytes(r, cache) for r in reqs)
    st = run_continuous(reqs, budget, ksteps=8, max_slots=8, cache=cache, realtime=False)
    assert st["requests"] == 10
    base = run_one_at_a_time(reqs2, cache=cache, realtime=False)
    assert base["requests"] == 10
    by = {r.rid: r for r in reqs2}
    for r in reqs:
        a = r.result.cpu().numpy().astype(np.float64)
        b = by[r.rid].result.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a)) and np.linalg.norm(b) > 0, r.rid
        assert np.linalg.norm(a - b) <= TOL_MIX * np.linalg.norm(b), r.rid
        assert r.done >= r.arrival


@pytest.mark.parametrize("split", [None, "-1"])
def test_deep_items_served(split, monkeypatch):
    """A medium with deep fluid items (sigma^11 written alone far from the
    solid) served by pact_advance, on the step graphs and on the
    multi-instance kernels: the multi-instance receiver kernel reads 3 sigma^11
    at deep corners and the read-out follows the fill of sigma^22, sigma^33."""
    if split is not None:
        monkeypatch.setenv("PACT_SERVE_SOLO_POINTS", split)
    nz, ny, nx = 64, 64, 192
    rng = np.random.default_rng(41)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = ((x - 0.85 * nx) / 12.0) ** 2 + ((y - ny / 2) / 9.0) ** 2 + ((z - nz / 2) / 12.0) ** 2 <= 1.0
    cp = np.where(inside, 2900.0, 1480.0)
    cs = np.where(inside, 1400.0, 0.0)
    rho = np.where(inside, 1850.0, 1000.0)
    lam, mu = synth.lame_from_speeds(cp, cs, rho)
    med = tuple(np.ascontiguousarray(a, dtype=np.float32) for a in (rho, lam, mu, np.zeros_like(rho)))
    d = GridDesc(nx, ny, nz, 0.4e-3, 0.3 * 0.4e-3 / 2900.0, npml=4, pml_vmax=2900.0)
    p0 = np.zeros((nz, ny, nx), np.float32)
    p0[8:-8, 8:-8, 8:-8] = rng.standard_normal((nz - 16, ny - 16, nx - 16))
    rec = synth.random_receivers(19, (nz, ny, nx), 42)
    rec[:6] = [[40.0 + 8 * k, 30.0, 20.0 + 3 * k] for k in range(6)]  # deep in the water
    cases = [("fwd", d, med, p0, rec, 33), ("adj", d, med, p0, rec, 29)]
    g = pact.Grid(d)
    g.set_medium(*[cuda(m) for m in med])
    assert g.deep_points() > 0
    g.close()
    for (kind, *_rest), (_inp, got, ref) in zip(cases, _serve_mix(cases, k=6)):
        assert np.all(np.isfinite(got)), kind
        assert rel_l2(got, ref) <= TOL_MIX, kind
