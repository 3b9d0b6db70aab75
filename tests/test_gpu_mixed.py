"""GPU: the medium-adaptive interior (fluid work items on the acoustic kernels).

Where mu = 0 at every integer node of a work item's reach, the elastic update
of Eq. (it) keeps sigma^11 = sigma^22 = sigma^33 and the shear stresses at
zero, so the acoustic update computes the same operator there (the paper's
acoustic ablation, Sec. 7, as a sub-domain of the elastic problem).  These
tests run media holding both fluid and solid interior work items and check:

- the forward traces and adjoint images against the FP64 oracle (1e-4);
- against the elastic kernels everywhere (PACT_ACOUSTIC=0): the two paths
  agree to 1e-6 relative L2 on traces, images and wavefields;
- the FP32 inner-product test (1e-5);
- the structure the switch relies on: in the fluid, the three normal stresses
  are bitwise equal and the shear stresses exactly zero.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from paper_1709_02733_b300 import pact, synth  # noqa: E402
from paper_1709_02733_b300.synth import GridDesc  # noqa: E402

TOL = 1e-4
TOL_PATHS = 1e-6
DOT_TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def make_grid(desc, medium):
    g = pact.Grid(desc)
    g.set_medium(*[cuda(m) for m in medium])
    return g


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1709_02733_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _inclusion_case(shape=(60, 40, 104), npml=4, seed=31, L=15, cx=0.8, rx=12.0):
    """Water with a solid ellipsoid (absorbing, +-5 % noise) off-centre in x:
    the tiles on one side see only fluid, those on the other side the solid
    (with cx near 1 the solid reaches into the x layer, so that elastic and
    fluid C-PML work items neighbour each other)."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = ((x - cx * nx) / rx) ** 2 + ((y - ny / 2) / 9.0) ** 2 + ((z - nz / 2) / 12.0) ** 2 <= 1.0
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
    p0[npml + 3:nz - npml - 3, npml + 3:ny - npml - 3, npml + 3:nx - npml - 3] = rng.standard_normal(
        (nz - 2 * npml - 6, ny - 2 * npml - 6, nx - 2 * npml - 6))
    rec = synth.random_receivers(L, shape, seed + 1)
    return d, med, p0, rec


def _paths(d, med, monkeypatch):
    g_m = make_grid(d, med)
    monkeypatch.setenv("PACT_ACOUSTIC", "0")
    g_e = make_grid(d, med)
    monkeypatch.delenv("PACT_ACOUSTIC")
    n_ac = g_m.role_points("fwd_ac_vel")[0]
    assert g_e.role_points("fwd_ac_vel")[0] == 0
    return g_m, g_e, n_ac


@pytest.mark.parametrize("cx,rx", [(0.8, 12.0), (0.95, 10.0)])
def test_mixed_against_oracle_and_elastic_path(cx, rx, monkeypatch):
    d, med, p0, rec = _inclusion_case(cx=cx, rx=rx)
    g_m, g_e, n_ac = _paths(d, med, monkeypatch)
    # fluid and solid interior work items both present
    assert 0 < n_ac < d.N
    assert g_m.role_points("fwd_velocity")[0] + n_ac == d.N
    nsteps = 57
    o = Oracle(d.as_dict(), *med)
    tr = g_m.forward(cuda(p0), rec, nsteps).cpu().numpy()
    assert rel_l2(tr, o.forward(p0, rec, nsteps)) <= TOL
    tr_e = g_e.forward(cuda(p0), rec, nsteps).cpu().numpy()
    assert rel_l2(tr, tr_e) <= TOL_PATHS
    assert rel_l2(g_m.get_wavefield(), g_e.get_wavefield()) <= TOL_PATHS
    y = np.random.default_rng(5).standard_normal(tr.shape).astype(np.float32)
    img = g_m.adjoint(cuda(y), rec).cpu().numpy()
    assert rel_l2(img, o.adjoint(y, rec)) <= TOL
    img_e = g_e.adjoint(cuda(y), rec).cpu().numpy()
    assert rel_l2(img, img_e) <= TOL_PATHS
    assert rel_l2(g_m.get_wavefield(), g_e.get_wavefield()) <= TOL_PATHS


def test_mixed_fluid_structure(monkeypatch):
    """After forward steps the fluid part of the mixed path holds equal normal
    stresses and zero shear (bitwise), as the elastic update does there."""
    d, med, p0, rec = _inclusion_case(seed=33)
    g_m, _g_e, n_ac = _paths(d, med, monkeypatch)
    assert n_ac > 0
    g_m.forward(cuda(p0), rec, 40)
    wf = g_m.get_wavefield()
    mu = med[2]
    from scipy.ndimage import maximum_filter
    fluid = maximum_filter((mu > 0).astype(np.uint8), size=7) == 0
    m = d.npml + 3  # off the C-PML layers and their reach
    core = np.zeros_like(fluid)
    core[m:-m, m:-m, m:-m] = True
    fluid &= core
    assert fluid.sum() > 1000
    s11, s22, s33, s23, s13, s12 = wf[3:9]
    assert np.array_equal(s11[fluid], s22[fluid]) and np.array_equal(s11[fluid], s33[fluid])
    assert not np.any(s23[fluid]) and not np.any(s13[fluid]) and not np.any(s12[fluid])
    assert np.abs(s11[fluid]).max() > 0


def test_mixed_inner_product_skull():
    w = synth.skull(96, 0.4e-3, 10, 300, 128, seed=3)
    g = make_grid(w.desc, w.medium)
    n_ac = g.role_points("fwd_ac_vel")[0]
    assert 0 < n_ac < w.desc.N
    tr = g.forward(cuda(w.p0), w.rec, w.nsteps)
    rng = np.random.default_rng(1)
    y = tr.cpu().numpy() + 0.1 * float(tr.std()) * rng.standard_normal(tr.shape).astype(np.float32)
    img = g.adjoint(cuda(y), w.rec).cpu().numpy()
    lhs = float(np.dot(tr.cpu().numpy().astype(np.float64).ravel(), y.astype(np.float64).ravel()))
    rhs = float(np.dot(w.p0.astype(np.float64).ravel(), img.astype(np.float64).ravel()))
    assert abs(lhs - rhs) / abs(lhs) <= DOT_TOL


def test_mixed_skull_512_split():
    """On the bench medium most of the interior runs the acoustic kernels."""
    w = synth.skull_512()
    g = make_grid(w.desc, w.medium)
    n_ac = g.role_points("fwd_ac_vel")[0]
    assert 0.5 * w.desc.N < n_ac < 0.7 * w.desc.N
    assert g.role_points("fwd_velocity")[0] + n_ac == w.desc.N
    # most of the water writes sigma^11 alone (no solid within a tile)
    assert 0.4 * w.desc.N < g.deep_points() < n_ac + 0.3 * w.desc.N
    g.close()


def test_deep_items_write_sigma11_only_and_change_nothing(monkeypatch):
    """Fluid no-layer items with no elastic item within a tile and three planes
    write sigma^11 alone; the sampler reads 3 sigma^11 there and the three
    normal stresses are filled in before the image read-out and the wavefield
    copy.  Fluid items that read no absorbing node (ITEM_NOALPHA) load no
    alpha box.  Traces, images and wavefields are bitwise those of the path
    without either (PACT_AC_DEEP=0, PACT_NOALPHA=0), and match the FP64
    oracle."""
    d, med, p0, rec = _inclusion_case(shape=(64, 64, 192), npml=4, seed=37, L=23, cx=0.85, rx=12.0)
    # receivers also deep inside the water, away from the inclusion
    rec[:8, 0] = np.linspace(36.0, 90.0, 8)
    rec[:8, 1] = np.linspace(20.0, 40.0, 8)
    rec[:8, 2] = np.linspace(20.0, 44.0, 8)
    g_d = make_grid(d, med)
    monkeypatch.setenv("PACT_AC_DEEP", "0")
    monkeypatch.setenv("PACT_NOALPHA", "0")
    g_a = make_grid(d, med)
    monkeypatch.delenv("PACT_AC_DEEP")
    monkeypatch.delenv("PACT_NOALPHA")
    assert g_d.deep_points() > 0 and g_a.deep_points() == 0
    assert g_d.noalpha_points() > 0 and g_a.noalpha_points() == 0
    nsteps = 45
    tr_d = g_d.forward(cuda(p0), rec, nsteps)
    # inside the solve sigma^22 is stale on the deep items (raw device views)
    raw11, raw22 = g_d.field_view(3), g_d.field_view(4)
    assert not torch.equal(raw11, raw22)
    tr_a = g_a.forward(cuda(p0), rec, nsteps)
    assert torch.equal(tr_d, tr_a)
    wf_d, wf_a = g_d.get_wavefield(), g_a.get_wavefield()
    assert np.array_equal(wf_d, wf_a)
    y = torch.from_numpy(np.random.default_rng(8).standard_normal(tuple(tr_d.shape)).astype(np.float32)).cuda()
    img_d = g_d.adjoint(y, rec)
    img_a = g_a.adjoint(y, rec)
    assert torch.equal(img_d, img_a)
    assert np.array_equal(g_d.get_wavefield(), g_a.get_wavefield())
    o = Oracle(d.as_dict(), *med)
    assert rel_l2(tr_d.cpu().numpy(), o.forward(p0, rec, nsteps)) <= TOL
    assert rel_l2(img_d.cpu().numpy(), o.adjoint(y.cpu().numpy(), rec)) <= TOL
