"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (written in each test): relative L2 error <= 1e-4 on receiver traces and
adjoint images; inner-product test <= 1e-5 in FP32.  Sizes are small enough
for the oracle to finish in seconds yet span several thread blocks and ragged
tails (odd, non-cubic grids); full-size checks use properties that hold at any
size or samples the oracle can compute one by one on a crop of the grid.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from paper_1709_02733_b300 import synth  # noqa: E402
from paper_1709_02733_b300 import pact  # noqa: E402
from paper_1709_02733_b300.synth import GridDesc  # noqa: E402

TOL = 1e-4
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


def _random_case(shape, npml, seed, L=9, absorb=True):
    rho, lam, mu, al, vmax = synth.random_medium(shape, seed, absorb=absorb)
    nz, ny, nx = shape
    dx = 1e-3
    d = GridDesc(nx, ny, nz, dx, 0.3 * dx / vmax, npml=npml, pml_vmax=vmax)
    rng = np.random.default_rng(seed + 1)
    p0 = rng.standard_normal(shape).astype(np.float32)
    rec = synth.random_receivers(L, shape, seed + 2)
    return d, (rho, lam, mu, al), p0, rec


@pytest.mark.parametrize("shape,npml,nsteps", [((29, 41, 37), 4, 60), ((20, 18, 35), 0, 40), ((16, 16, 16), 3, 30)])
def test_forward_adjoint_random_medium(shape, npml, nsteps):
    """Random heterogeneous medium (fluid and solid nodes, absorption), odd grid."""
    d, med, p0, rec = _random_case(shape, npml, 100 + npml)
    o = Oracle(d.as_dict(), *med)
    g = make_grid(d, med)
    tr = g.forward(cuda(p0), rec, nsteps).cpu().numpy()
    ref = o.forward(p0, rec, nsteps)
    assert rel_l2(tr, ref) <= TOL
    y = np.random.default_rng(5).standard_normal(ref.shape).astype(np.float32)
    img = g.adjoint(cuda(y), rec).cpu().numpy()
    ref_img = o.adjoint(y, rec)
    assert rel_l2(img, ref_img) <= TOL


def test_skull_like_48():
    """Skull-like 48^3 workload (shell, tissue, tubes, hemisphere receivers, 6-cell C-PML)."""
    w = synth.skull(48, 1.2e-3, 6, 150, 64, seed=9)
    o = Oracle(w.desc.as_dict(), *w.medium)
    g = make_grid(w.desc, w.medium)
    tr = g.forward(cuda(w.p0), w.rec, w.nsteps).cpu().numpy()
    ref = o.forward(w.p0, w.rec, w.nsteps)
    assert rel_l2(tr, ref) <= TOL
    img = g.adjoint(cuda(ref.astype(np.float32)), w.rec).cpu().numpy()
    assert rel_l2(img, o.adjoint(ref.astype(np.float32), w.rec)) <= TOL


def test_plain_fluid_64_full():
    """The plain 64^3 workload in full: 400 steps, 128 receivers, 3-cell C-PML."""
    w = synth.plain_fluid_64(npml=3, nsteps=400)
    o = Oracle(w.desc.as_dict(), *w.medium)
    g = make_grid(w.desc, w.medium)
    tr = g.forward(cuda(w.p0), w.rec, w.nsteps).cpu().numpy()
    ref = o.forward(w.p0, w.rec, w.nsteps)
    assert rel_l2(tr, ref) <= TOL
    rng = np.random.default_rng(1)
    y = (ref + 0.1 * np.sqrt(np.mean(ref ** 2)) * rng.standard_normal(ref.shape)).astype(np.float32)
    img = g.adjoint(cuda(y), w.rec).cpu().numpy()
    assert rel_l2(img, o.adjoint(y, w.rec)) <= TOL


def _dot_test(g, p0, rec, nsteps, seed=1):
    tr = g.forward(cuda(p0), rec, nsteps).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(seed)
    y = tr + 0.1 * np.sqrt(np.mean(tr ** 2)) * rng.standard_normal(tr.shape)
    img = g.adjoint(cuda(y), rec).cpu().numpy().astype(np.float64)
    lhs = float(np.sum(tr * y.astype(np.float32).astype(np.float64)))
    rhs = float(np.sum(p0.astype(np.float64) * img))
    return abs(lhs - rhs) / abs(lhs)


def test_inner_product_fp32_skull():
    w = synth.skull(96, 0.4e-3, 10, 300, 128, seed=3)
    g = make_grid(w.desc, w.medium)
    assert _dot_test(g, w.p0, w.rec, w.nsteps) <= DOT_TOL


def test_first_sample_and_zero_steps():
    """nsteps = 0: traces are p_hat_0 = trilinear interpolation of p0; receivers
    on the grid edges (0 and n-2) are accepted."""
    from scipy.ndimage import map_coordinates
    d, med, p0, rec = _random_case((13, 12, 11), 2, 7, L=6)
    rec[0] = [0, 0, 0]
    rec[1] = [d.nx - 2, d.ny - 2, d.nz - 2]
    g = make_grid(d, med)
    tr = g.forward(cuda(p0), rec, 0).cpu().numpy()
    assert tr.shape == (1, 6)
    ref = map_coordinates(p0.astype(np.float64), [rec[:, 2], rec[:, 1], rec[:, 0]], order=1)
    np.testing.assert_allclose(tr[0], ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())


def test_single_receiver_and_determinism():
    d, med, p0, rec = _random_case((24, 23, 22), 3, 11, L=1)
    g = make_grid(d, med)
    a = g.forward(cuda(p0), rec, 25).cpu().numpy()
    b = g.forward(cuda(p0), rec, 25).cpu().numpy()
    assert np.array_equal(a, b)
    y = cuda(np.random.default_rng(2).standard_normal(a.shape))
    i1 = g.adjoint(y, rec).cpu().numpy()
    i2 = g.adjoint(y, rec).cpu().numpy()
    assert np.array_equal(i1, i2)
    o = Oracle(d.as_dict(), *med)
    assert rel_l2(a, o.forward(p0, rec, 25)) <= TOL


def test_host_pointer_calls_match_device_calls():
    d, med, p0, rec = _random_case((20, 21, 22), 3, 13)
    g = make_grid(d, med)
    a = g.forward(cuda(p0), rec, 15).cpu().numpy()
    b = g.forward_host(p0, rec, 15)
    assert np.array_equal(a, b)
    i1 = g.adjoint(cuda(a), rec).cpu().numpy()
    i2 = g.adjoint_host(a, rec)
    assert np.array_equal(i1, i2)


def test_error_paths():
    d, med, p0, rec = _random_case((16, 16, 16), 2, 17)
    g = pact.Grid(d)
    with pytest.raises(pact.PactError) as e:
        g.forward(cuda(p0), rec, 3)
    assert e.value.code == pact.PACT_ESTATE
    g.set_medium(*[cuda(m) for m in med])
    bad = rec.copy()
    bad[0, 0] = d.nx - 1.5  # beyond n-2
    with pytest.raises(pact.PactError) as e:
        g.forward(cuda(p0), bad, 3)
    assert e.value.code == pact.PACT_EINVAL
    rho = med[0].copy()
    rho[3, 3, 3] = 0.0
    with pytest.raises(pact.PactError) as e:
        g.set_medium(cuda(rho), *[cuda(m) for m in med[1:]])
    assert e.value.code == pact.PACT_EINVAL
    fast = GridDesc(d.nx, d.ny, d.nz, d.dx, d.dt * 2.0, npml=2, pml_vmax=d.pml_vmax)  # CFL 0.6
    g2 = pact.Grid(fast)
    with pytest.raises(pact.PactError) as e:
        g2.set_medium(*[cuda(m) for m in med])
    assert e.value.code == pact.PACT_ECFL


def _crop_check(w, g, nsteps, centers):
    """Oracle on a crop around each sample point: after k steps a point depends on
    the data within 4k cells, so a crop of half-width 4k+2 with no C-PML (the
    samples are deep in the interior) reproduces the full-grid values there."""
    fields = g.get_wavefield()  # u1 u2 u3 s11 s22 s33 s23 s13 s12
    hw = 4 * nsteps + 2
    errs = []
    for (x, y, z) in centers:
        sl = (slice(z - hw, z + hw + 1), slice(y - hw, y + hw + 1), slice(x - hw, x + hw + 1))
        n = 2 * hw + 1
        dd = dict(nx=n, ny=n, nz=n, dx=w.desc.dx, dt=w.desc.dt, npml=0, pml_vmax=w.desc.pml_vmax)
        o = Oracle(dd, *[np.ascontiguousarray(m[sl]) for m in w.medium])
        st = o.run_state(np.ascontiguousarray(w.p0[sl]), nsteps)
        v = Oracle.views(st)
        ref = np.concatenate([v["u"][:, hw, hw, hw], v["sigma"][:, hw, hw, hw]])
        got = fields[:, z, y, x].astype(np.float64)
        errs.append(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30))
    return max(errs)


def _layer_crop_check(w, p0, fields, nsteps, m, high, points):
    """Oracle on the m^3 corner crop at the grid's low (or high) corner, with
    the grid's C-PML: a layer's profile depends only on the depth into it, so
    the crop's layers on the grid's own faces are the grid's.  A point after k
    steps depends on the data within 4k cells; the points must keep that reach
    clear of the crop's other three faces and their (artificial) layers."""
    d = w.desc
    P, reach = d.npml, 4 * nsteps
    lo = [d.nz - m, d.ny - m, d.nx - m] if high else [0, 0, 0]
    for (x, y, z) in points:
        for c, l in zip((z, y, x), lo):
            assert (c - reach >= l + P + 1) if high else (c + reach + 2 <= m - P - 1), (x, y, z)
    sl = tuple(slice(l, l + m) for l in lo)
    dd = dict(nx=m, ny=m, nz=m, dx=d.dx, dt=d.dt, npml=P, pml_R0=d.pml_R0, pml_f0=d.pml_f0, pml_vmax=d.pml_vmax)
    o = Oracle(dd, *[np.ascontiguousarray(a[sl]) for a in w.medium])
    v = Oracle.views(o.run_state(np.ascontiguousarray(p0[sl]), nsteps))
    errs = []
    for (x, y, z) in points:
        cz, cy, cx = z - lo[0], y - lo[1], x - lo[2]
        ref = np.concatenate([v["u"][:, cz, cy, cx], v["sigma"][:, cz, cy, cx]])
        got = fields[:, z, y, x].astype(np.float64)
        errs.append(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30))
    return max(errs)


def test_full_size_512_sampled():
    """The 512^3 skull workload in the launch configuration the bench times:
    (a) p_hat_0 equals the trilinear interpolation of p0 at every receiver;
    (b) the wavefield after 2 steps matches the oracle at sampled interior
        points (oracle on a crop);
    (c) inner-product test over 12 steps at full size, with a seeded random p0
        over the whole grid so that the receivers see it from the first sample;
    (d) the C-PML frame kernels at full size against oracle corner crops."""
    from scipy.ndimage import map_coordinates
    w = synth.skull_512()
    g = make_grid(w.desc, w.medium)
    tr0 = g.forward(cuda(w.p0), w.rec, 0).cpu().numpy()
    ref0 = map_coordinates(w.p0.astype(np.float64), [w.rec[:, 2], w.rec[:, 1], w.rec[:, 0]], order=1)
    assert np.abs(tr0[0] - ref0).max() <= 1e-5 * max(np.abs(ref0).max(), 1e-6) + 1e-7
    g.forward(cuda(w.p0), w.rec, 2)
    idx = np.argwhere(w.p0 > 0.3 * w.p0.max())
    rng = np.random.default_rng(0)
    pick = idx[rng.choice(len(idx), 6, replace=False)]
    centers = [(int(c[2]), int(c[1]), int(c[0])) for c in pick]
    # plus points in the skull shell (solid, absorbing)
    shell = np.argwhere(w.mu[::7, ::7, ::7] > 0) * 7
    for c in shell[rng.choice(len(shell), 4, replace=False)]:
        centers.append((int(c[2]), int(c[1]), int(c[0])))
    assert _crop_check(w, g, 2, centers) <= 1e-4
    pr = np.random.default_rng(11).standard_normal(w.p0.shape).astype(np.float32)
    # (d) the C-PML frame at full size (corner, edge and z-slab tiles, both
    #     ends of every axis) after 2 steps of a p0 that fills the grid, against
    #     the oracle on 64^3 corner crops that carry the grid's own layers
    g.forward(cuda(pr), w.rec, 2)
    fields = g.get_wavefield()
    n = w.desc.nx
    # corner tiles, x-edge tiles (layer and non-layer points), interior tiles on a z slab and next to the y layer
    low = [(10, 10, 10), (3, 30, 30), (30, 12, 30), (30, 30, 19), (21, 30, 30), (19, 19, 30), (40, 40, 10),
           (36, 25, 41)]
    high = [(n - 1 - x, n - 1 - y, n - 1 - z) for (x, y, z) in low]
    assert _layer_crop_check(w, pr, fields, 2, 72, False, low) <= 1e-4
    assert _layer_crop_check(w, pr, fields, 2, 72, True, high) <= 1e-4
    del fields
    assert _dot_test(g, pr, w.rec, 12) <= DOT_TOL


# ---------------------------------------------------------------------------
# TMA-staged kernels (used when nx % 4 == 0): ragged tiles on every axis
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,npml,nsteps", [((23, 19, 36), 3, 40), ((40, 44, 68), 5, 60), ((17, 33, 64), 0, 30),
                                               ((70, 12, 8), 2, 25), ((30, 34, 132), 0, 30)])
def test_tiled_random_medium(shape, npml, nsteps):
    d, med, p0, rec = _random_case(shape, npml, 300 + npml)
    assert d.nx % 4 == 0
    o = Oracle(d.as_dict(), *med)
    g = make_grid(d, med)
    tr = g.forward(cuda(p0), rec, nsteps).cpu().numpy()
    ref = o.forward(p0, rec, nsteps)
    assert rel_l2(tr, ref) <= TOL
    y = np.random.default_rng(6).standard_normal(ref.shape).astype(np.float32)
    img = g.adjoint(cuda(y), rec).cpu().numpy()
    assert rel_l2(img, o.adjoint(y, rec)) <= TOL


# Grids with every region kind of the TMA-staged kernels: interior tiles off
# and on the z slabs, x-layer and y-layer edge tiles and corner tiles (the
# interior needs nx >= 72 and ny >= 24 at a 4-cell layer); ragged tiles too.
@pytest.mark.parametrize("shape,npml,nsteps", [((40, 44, 104), 4, 40), ((52, 37, 100), 5, 45)])
def test_tiled_all_region_kinds(shape, npml, nsteps, monkeypatch):
    d, med, p0, rec = _random_case(shape, npml, 500 + npml, L=13)
    o = Oracle(d.as_dict(), *med)
    g = make_grid(d, med)
    tr = g.forward(cuda(p0), rec, nsteps).cpu().numpy()
    assert rel_l2(tr, o.forward(p0, rec, nsteps)) <= TOL
    y = np.random.default_rng(8).standard_normal(tr.shape).astype(np.float32)
    img = g.adjoint(cuda(y), rec).cpu().numpy()
    assert rel_l2(img, o.adjoint(y, rec)) <= TOL
    # and the one-thread-per-point kernels agree to FP32 rounding
    monkeypatch.setenv("PACT_KERNELS", "direct")
    g_d = make_grid(d, med)
    monkeypatch.delenv("PACT_KERNELS")
    assert rel_l2(tr, g_d.forward(cuda(p0), rec, nsteps).cpu().numpy()) <= 1e-5
    assert rel_l2(img, g_d.adjoint(cuda(y), rec).cpu().numpy()) <= 1e-5


def test_tiled_matches_direct(monkeypatch):
    """Both kernel families compute the same operator (agreement to FP32 rounding)."""
    d, med, p0, rec = _random_case((30, 27, 44), 4, 400)
    g_t = make_grid(d, med)
    monkeypatch.setenv("PACT_KERNELS", "direct")
    g_d = make_grid(d, med)
    monkeypatch.delenv("PACT_KERNELS")
    a = g_t.forward(cuda(p0), rec, 50).cpu().numpy()
    b = g_d.forward(cuda(p0), rec, 50).cpu().numpy()
    assert rel_l2(a, b) <= 1e-5
    fa, fb = g_t.get_wavefield(), g_d.get_wavefield()
    assert rel_l2(fa, fb) <= 1e-5
    y = cuda(np.random.default_rng(7).standard_normal(a.shape))
    ia = g_t.adjoint(y, rec).cpu().numpy()
    ib = g_d.adjoint(y, rec).cpu().numpy()
    assert rel_l2(ia, ib) <= 1e-5


# ---------------------------------------------------------------------------
# Single-pass interior kernel (PACT_FUSED=1: two wavefield buffers) against the
# in-place two-pass kernels: fused regions with and without a layer, of one tile and of
# several, beside ragged edge tiles.  Every grid point must be written by
# exactly one launch per half step; a point left out would keep the value of
# two steps before and show up here.  The two paths differ only by FP32
# rounding (contraction order).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,npml,nsteps", [((40, 44, 104), 4, 41), ((33, 30, 72), 3, 30), ((48, 50, 132), 0, 35),
                                               ((60, 61, 100), 6, 52)])
def test_fused_matches_two_pass(shape, npml, nsteps, monkeypatch):
    d, med, p0, rec = _random_case(shape, npml, 700 + npml, L=11)
    g_2 = make_grid(d, med)
    monkeypatch.setenv("PACT_FUSED", "1")
    g_f = make_grid(d, med)
    monkeypatch.delenv("PACT_FUSED")
    nf = g_f.role_points("fwd_fused")[0]
    assert nf > 0 and g_2.role_points("fwd_fused")[0] == 0
    assert g_f.role_points("fwd_velocity")[0] + nf == d.N == g_f.role_points("fwd_stress")[0] + nf
    a = g_f.forward(cuda(p0), rec, nsteps).cpu().numpy()
    b = g_2.forward(cuda(p0), rec, nsteps).cpu().numpy()
    assert rel_l2(a, b) <= 1e-6
    assert rel_l2(g_f.get_wavefield(), g_2.get_wavefield()) <= 1e-6
    y = cuda(np.random.default_rng(9).standard_normal(a.shape))
    ia = g_f.adjoint(y, rec).cpu().numpy()
    ib = g_2.adjoint(y, rec).cpu().numpy()
    assert rel_l2(ia, ib) <= 1e-6
    assert rel_l2(g_f.get_wavefield(), g_2.get_wavefield()) <= 1e-6


def test_fused_odd_and_even_step_counts(monkeypatch):
    """The state ends in either buffer: forward/adjoint results and the
    wavefield read-back are right after an odd and an even number of steps,
    and a solve after another one starts from zero."""
    d, med, p0, rec = _random_case((36, 30, 72), 3, 801, L=7)
    o = Oracle(d.as_dict(), *med)
    monkeypatch.setenv("PACT_FUSED", "1")
    g = make_grid(d, med)
    monkeypatch.delenv("PACT_FUSED")
    assert g.role_points("adj_fused")[0] > 0
    for nsteps in (13, 14):
        tr = g.forward(cuda(p0), rec, nsteps).cpu().numpy()
        assert rel_l2(tr, o.forward(p0, rec, nsteps)) <= TOL
        st = o.run_state(p0, nsteps)
        v = Oracle.views(st)
        ref = np.concatenate([v["u"], v["sigma"]])
        assert rel_l2(g.get_wavefield(), ref) <= TOL
        y = np.random.default_rng(nsteps).standard_normal(tr.shape).astype(np.float32)
        img = g.adjoint(cuda(y), rec).cpu().numpy()
        assert rel_l2(img, o.adjoint(y, rec)) <= TOL


def test_fused_inner_product_and_oracle(monkeypatch):
    """The single-pass path: FP32 inner-product test on a skull-like grid with
    a fused region, and oracle parity on a random medium."""
    monkeypatch.setenv("PACT_FUSED", "1")
    w = synth.skull(96, 0.4e-3, 10, 300, 128, seed=3)
    g = make_grid(w.desc, w.medium)
    assert g.role_points("fwd_fused")[0] > 0
    assert _dot_test(g, w.p0, w.rec, w.nsteps) <= DOT_TOL
    d, med, p0, rec = _random_case((40, 44, 104), 4, 904, L=13)
    g = make_grid(d, med)
    monkeypatch.delenv("PACT_FUSED")
    assert g.role_points("adj_fused")[0] > 0
    o = Oracle(d.as_dict(), *med)
    tr = g.forward(cuda(p0), rec, 37).cpu().numpy()
    assert rel_l2(tr, o.forward(p0, rec, 37)) <= TOL
    y = np.random.default_rng(10).standard_normal(tr.shape).astype(np.float32)
    assert rel_l2(g.adjoint(cuda(y), rec).cpu().numpy(), o.adjoint(y, rec)) <= TOL


def _band_count(p0, band):
    nz, ny, nx = p0.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dmin = np.minimum.reduce([x, nx - 1 - x, y, ny - 1 - y, z, nz - 1 - z])
    return int(np.count_nonzero((p0 != 0) & (dmin < band)))


@pytest.mark.parametrize("shape,npml", [((40, 44, 52), 4), ((21, 19, 35), 3)])
def test_p0_support_warning_counts(shape, npml):
    """The source pass counts the nonzero p0 entries within npml + 2 nodes of a
    face (the paper's support rule, a warning only): exact against numpy for a
    dense p0, 0 for a p0 kept clear of the band, and reset by every solve."""
    d, med, p0, rec = _random_case(shape, npml, 13, L=4)
    g = make_grid(d, med)
    band = npml + 2
    g.forward(cuda(p0), rec, 3)
    assert g.support_warning() == _band_count(p0, band) > 0
    inner = np.zeros_like(p0)
    inner[band:-band, band:-band, band:-band] = p0[band:-band, band:-band, band:-band]
    g.forward(cuda(inner), rec, 3)
    assert g.support_warning() == 0
    # single points at distance band - 1 (counted) and band (not counted) from each face
    pts = np.zeros_like(p0)
    nz, ny, nx = shape
    cz, cy, cx = nz // 2, ny // 2, nx // 2
    for dist, val in ((band - 1, 1.0), (band, 2.0)):
        pts[cz, cy, dist] = pts[cz, cy, nx - 1 - dist] = val
        pts[cz, dist, cx] = pts[cz, ny - 1 - dist, cx] = val
        pts[dist, cy, cx] = pts[nz - 1 - dist, cy, cx] = val
    g.forward(cuda(pts), rec, 0)
    assert g.support_warning() == 6 == _band_count(pts, band)
    g.close()


def test_p0_support_warning_without_layer():
    d, med, p0, rec = _random_case((20, 18, 36), 0, 14, L=4)
    g = make_grid(d, med)
    g.forward(cuda(p0), rec, 2)
    assert g.support_warning() == 0
    g.close()


def test_degenerate_inputs_and_rejected_calls():
    """Zero p0 gives exactly zero traces and zero traces exactly zero image; the
    raw ABI rejects L = 0, nsteps < 0 and NULL data pointers with PACT_EINVAL
    and the handle then solves exactly as a fresh one."""
    import ctypes
    d, med, p0, rec = _random_case((18, 17, 20), 2, 21, L=5)
    g = make_grid(d, med)
    assert g.support_warning() == 0                      # no forward solve yet
    zero = torch.zeros(d.shape, device="cuda")
    tr = g.forward(zero, rec, 7)
    assert torch.count_nonzero(tr).item() == 0
    assert torch.count_nonzero(g.adjoint(torch.zeros_like(tr), rec)).item() == 0
    vp = ctypes.c_void_p
    r = np.ascontiguousarray(rec, np.float32)
    out = torch.empty((8, 5), device="cuda")
    img = torch.empty(d.shape, device="cuda")
    lib = g.lib
    assert lib.pact_forward(g._h, vp(zero.data_ptr()), r.ctypes.data_as(vp), 0, 7, vp(out.data_ptr())) == pact.PACT_EINVAL
    assert lib.pact_forward(g._h, vp(zero.data_ptr()), r.ctypes.data_as(vp), 5, -1, vp(out.data_ptr())) == pact.PACT_EINVAL
    assert lib.pact_forward(g._h, None, r.ctypes.data_as(vp), 5, 7, vp(out.data_ptr())) == pact.PACT_EINVAL
    assert lib.pact_forward(g._h, vp(zero.data_ptr()), None, 5, 7, vp(out.data_ptr())) == pact.PACT_EINVAL
    assert lib.pact_adjoint(g._h, vp(out.data_ptr()), r.ctypes.data_as(vp), 5, 7, None) == pact.PACT_EINVAL
    assert lib.pact_adjoint(g._h, None, r.ctypes.data_as(vp), 5, 7, vp(img.data_ptr())) == pact.PACT_EINVAL
    assert lib.pact_last_error(g._h)
    a = g.forward(cuda(p0), rec, 7).cpu().numpy()
    b = make_grid(d, med).forward(cuda(p0), rec, 7).cpu().numpy()
    assert np.array_equal(a, b)
