"""GPU: the z-slab decomposition (pact_create_slab + half steps + halo exchange).

R slab handles on one device advance in lockstep with LoopbackExchange (plain
device copies between the slabs' halo planes; DistExchange runs the same
pattern between processes).  Checked against the whole-grid handle (1e-6
relative L2: the same kernels, with the medium-adaptive split made
conservative beside the cuts) and the FP64 oracle (1e-4), forward and
adjoint, with receivers on both sides of the cuts, on a cut plane, and a slab
that samples no receiver.  The inner-product test across slabs checks that
the pieces assemble H and H^T of one operator.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from paper_1709_02733_b300 import pact, slabs, synth  # noqa: E402
from paper_1709_02733_b300.synth import GridDesc  # noqa: E402

TOL = 1e-4
TOL_WHOLE = 1e-6
DOT_TOL = 1e-5


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
    assert torch.cuda.is_available()


def _inclusion_case(shape=(60, 40, 104), npml=4, seed=41, L=15):
    """Water with an absorbing solid ellipsoid that crosses the cut planes."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = ((x - 0.7 * nx) / 14.0) ** 2 + ((y - ny / 2) / 9.0) ** 2 + ((z - nz / 2) / 16.0) ** 2 <= 1.0
    cp = np.where(inside, 2900.0, 1480.0) * (1 + 0.05 * inside * rng.uniform(-1, 1, shape))
    cs = np.where(inside, 1400.0, 0.0)
    rho = np.where(inside, 1850.0, 1000.0) * (1 + 0.05 * inside * rng.uniform(-1, 1, shape))
    lam, mu = synth.lame_from_speeds(cp, cs, rho)
    al = np.where(inside, 1e5, 0.0)
    med = tuple(np.ascontiguousarray(a, dtype=np.float32) for a in (rho, lam, mu, al))
    dx = 0.4e-3
    vmax = float(cp.max())
    d = GridDesc(nx, ny, nz, dx, 0.3 * dx / vmax, npml=npml, pml_vmax=vmax)
    p0 = np.zeros(shape, np.float32)
    m = npml + 3
    p0[m:nz - m, m:ny - m, m:nx - m] = rng.standard_normal((nz - 2 * m, ny - 2 * m, nx - 2 * m))
    rec = synth.random_receivers(L, shape, seed + 1)
    # straddling the cuts of 2 slabs (30) and of 3 slabs (20, 40), and on a cut
    rec[0, 2], rec[1, 2], rec[2, 2], rec[3, 2] = 29.5, 19.25, 39.75, 30.0
    return d, med, p0, rec


def _slabs(d, med, rec, R):
    parts = slabs.partition(d.nz, R, d.npml)
    out = []
    for r in range(R):
        s = slabs.make_slab(d, parts, r, rec)
        s.grid.set_medium(*[cuda(m[s.zl:s.zh]) for m in med])
        out.append(s)
    return out


def _slab_solves(d, med, p0, rec, y, nsteps, R):
    sl = _slabs(d, med, rec, R)
    ex = slabs.LoopbackExchange()
    tr = slabs.forward(sl, [cuda(p0[s.zl:s.zh]) for s in sl], nsteps, ex)
    traces = slabs.gather_traces(sl, tr, len(rec)).cpu().numpy()
    yt = torch.from_numpy(y)
    img = slabs.adjoint(sl, [yt[:, torch.as_tensor(s.inj_idx, dtype=torch.long)].cuda() for s in sl], nsteps, ex)
    image = slabs.assemble_image(sl, img).cpu().numpy()
    return sl, traces, image


@pytest.mark.parametrize("R", [2, 3])
def test_slabs_match_whole_grid_and_oracle(R):
    d, med, p0, rec = _inclusion_case()
    nsteps = 61
    y = np.random.default_rng(9).standard_normal((nsteps + 1, len(rec))).astype(np.float32)
    sl, traces, image = _slab_solves(d, med, p0, rec, y, nsteps, R)
    # the receivers beside the cuts are injected by two slabs
    assert sum(len(s.inj_idx) for s in sl) > len(rec)
    g = pact.Grid(d)
    g.set_medium(*[cuda(m) for m in med])
    tr_w = g.forward(cuda(p0), rec, nsteps).cpu().numpy()
    img_w = g.adjoint(cuda(y), rec).cpu().numpy()
    assert rel_l2(traces, tr_w) <= TOL_WHOLE
    assert rel_l2(image, img_w) <= TOL_WHOLE
    o = Oracle(d.as_dict(), *med)
    assert rel_l2(traces, o.forward(p0, rec, nsteps)) <= TOL
    assert rel_l2(image, o.adjoint(y, rec)) <= TOL


def test_slab_without_receivers():
    """All receivers in the lower slab: the upper one runs with L = 0."""
    d, med, p0, rec = _inclusion_case(seed=43)
    rec[:, 2] = np.clip(rec[:, 2] * 0.4, 0, 26)
    nsteps = 40
    y = np.random.default_rng(10).standard_normal((nsteps + 1, len(rec))).astype(np.float32)
    sl, traces, image = _slab_solves(d, med, p0, rec, y, nsteps, 2)
    assert len(sl[1].rec_idx) == 0 and len(sl[1].inj_idx) == 0
    g = pact.Grid(d)
    g.set_medium(*[cuda(m) for m in med])
    assert rel_l2(traces, g.forward(cuda(p0), rec, nsteps).cpu().numpy()) <= TOL_WHOLE
    assert rel_l2(image, g.adjoint(cuda(y), rec).cpu().numpy()) <= TOL_WHOLE


def test_slabs_inner_product_skull():
    """Skull medium (fluid and solid beside the cuts, hemisphere receivers
    across them), 4 slabs: <H p, y> = <p, H^T y> summed over the slabs."""
    w = synth.skull(96, 0.4e-3, 10, 300, 128, seed=3)
    d = w.desc
    sl = _slabs(d, w.medium, w.rec, 4)
    ex = slabs.LoopbackExchange()
    tr = slabs.forward(sl, [cuda(w.p0[s.zl:s.zh]) for s in sl], w.nsteps, ex)
    traces = slabs.gather_traces(sl, tr, len(w.rec)).cpu().numpy()
    rng = np.random.default_rng(1)
    y = traces + 0.1 * float(traces.std()) * rng.standard_normal(traces.shape).astype(np.float32)
    yt = torch.from_numpy(y)
    img = slabs.adjoint(sl, [yt[:, torch.as_tensor(s.inj_idx, dtype=torch.long)].cuda() for s in sl],
                        w.nsteps, ex)
    image = slabs.assemble_image(sl, img).cpu().numpy()
    lhs = float(np.dot(traces.astype(np.float64).ravel(), y.astype(np.float64).ravel()))
    rhs = float(np.dot(w.p0.astype(np.float64).ravel(), image.astype(np.float64).ravel()))
    assert abs(lhs - rhs) / abs(lhs) <= DOT_TOL
    g = pact.Grid(d)
    g.set_medium(*[cuda(m) for m in w.medium])
    assert rel_l2(traces, g.forward(cuda(w.p0), w.rec, w.nsteps).cpu().numpy()) <= TOL_WHOLE


def test_create_slab_rejects():
    d = GridDesc(64, 32, 40, 0.4e-3, 5e-8, npml=4)
    for lo, hi in ((-1, 10), (0, 41), (10, 14)):
        with pytest.raises(pact.PactError):
            pact.Grid(d, slab=(lo, hi))


def test_slabs_with_deep_items():
    """Slabs cut through a medium with deep fluid items (sigma^11 written
    alone): the planes a slab exchanges are never deep, so the slabs match the
    whole grid."""
    d, med, p0, rec = _inclusion_case(shape=(64, 64, 192), npml=4, seed=45, L=17)
    g = pact.Grid(d)
    g.set_medium(*[cuda(m) for m in med])
    assert g.deep_points() > 0
    nsteps = 41
    y = np.random.default_rng(11).standard_normal((nsteps + 1, len(rec))).astype(np.float32)
    tr_w = g.forward(cuda(p0), rec, nsteps).cpu().numpy()
    img_w = g.adjoint(cuda(y), rec).cpu().numpy()
    for R in (2, 3):
        sl, traces, image = _slab_solves(d, med, p0, rec, y, nsteps, R)
        assert sum(s.grid.deep_points() for s in sl) > 0
        assert rel_l2(traces, tr_w) <= TOL_WHOLE
        assert rel_l2(image, img_w) <= TOL_WHOLE
