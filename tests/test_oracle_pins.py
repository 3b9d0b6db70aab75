"""Pins of the FP64 oracle against facts that do not come from the oracle.

Every oracle function is checked here against something independent of its
own formulas:

  stencil, staggering, Voigt order, velocity / stress updates
      -> exactness on degree-4 polynomials (the 4th-order staggered difference of
         Sec. 2.2, Eq. (derivative), differentiates quartics exactly)
  medium averaging (rho, alpha arithmetic; mu harmonic)
      -> linear fields are averaged exactly; alternating mu gives 2ab/(a+b)
  source tau' and sampler Theta' (Eqs. (initialp0), (interpgrid))
      -> p_hat_0 equals scipy's trilinear interpolation of p0
  adjoint (Sec. 4, Eq. (Adjup); Appendix A.3, Eq. (AdjupPML))
      -> dense brute-force transposes of H and of every sub-update
      -> inner-product test (Sec. 5) to 1e-12
  leapfrog + materials + zero-padded boundary
      -> exact energy conservation with alpha = 0 and no PML
  the physics
      -> closed-form N-wave / smooth-bump solution of the homogeneous fluid and
         its convergence order
  C-PML (Appendix A.1-A.3)
      -> profile properties and continuous normal-incidence reflection = R0
      -> reflection off the layer vs a larger grid with no layer
  structure
      -> fluid: shear stresses vanish, normal stresses equal; linearity;
         x <-> y axis permutation equivariance
  FISTA with the non-negativity projection (oracle/fista.py)
      -> converges to scipy.optimize.nnls's solution on a dense problem
  total-variation proximal step with non-negativity (oracle/fista.py)
      -> equals a direct QP solve (scipy SLSQP on the split formulation) in 1-D,
         and reduces to that 1-D solution when the 3-D input varies along one
         axis only; the difference pair is an exact adjoint pair
"""
import math

import numpy as np
import pytest

from oracle import Oracle, pml_profile
from paper_1709_02733_b300 import synth


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def _desc(shape, dx, dt, npml=0, vmax=1500.0):
    nz, ny, nx = shape
    return dict(nx=nx, ny=ny, nz=nz, dx=dx, dt=dt, npml=npml, pml_R0=1e-4, pml_f0=1e6, pml_vmax=vmax)


# staggered offsets (x, y, z) in cells of every field
U_OFF = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
S_OFF = [(0, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]  # Voigt 11 22 33 23 13 12
VOIGT = [[0, 5, 4], [5, 1, 3], [4, 3, 2]]


class Poly:
    """Random polynomial of total degree <= 4 in (X, Y, Z) with its gradient."""

    def __init__(self, rng):
        self.terms = []
        for a in range(5):
            for b in range(5 - a):
                for c in range(5 - a - b):
                    self.terms.append((a, b, c, rng.uniform(-1, 1)))

    def __call__(self, X, Y, Z):
        return sum(k * X ** a * Y ** b * Z ** c for a, b, c, k in self.terms)

    def d(self, axis, X, Y, Z):
        out = 0.0
        for a, b, c, k in self.terms:
            e = [a, b, c]
            if e[axis] == 0:
                continue
            f = k * e[axis]
            e[axis] -= 1
            out = out + f * X ** e[0] * Y ** e[1] * Z ** e[2]
        return out


def _coords(shape, off, dx):
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (X + off[0]) * dx, (Y + off[1]) * dx, (Z + off[2]) * dx


def _interior(shape, m=2):
    nz, ny, nx = shape
    return (slice(m, nz - m - 1), slice(m, ny - m - 1), slice(m, nx - m - 1))


# ---------------------------------------------------------------------------
# stencil / staggering / update formulas
# ---------------------------------------------------------------------------
def test_velocity_update_exact_on_quartics():
    """S2 with polynomial stresses: u^i += dt/rho_i * sum_j d_j sigma^{ij}, exactly,
    with rho and alpha linear in space (so their arithmetic mean at the velocity
    node is their value there)."""
    rng = np.random.default_rng(11)
    shape, dx, dt = (10, 11, 12), 0.5, 0.1
    desc = _desc(shape, dx, dt)
    X, Y, Z = _coords(shape, (0, 0, 0), 1.0)
    rho = 2.0 + 0.05 * X + 0.03 * Y + 0.02 * Z
    alpha = 0.3 + 0.01 * X + 0.02 * Y + 0.04 * Z
    lam = np.full(shape, 3.0)
    mu = np.full(shape, 1.0)
    o = Oracle(desc, rho, lam, mu, alpha)
    polys = [Poly(rng) for _ in range(6)]
    st = o.new_state()
    v = Oracle.views(st)
    for s in range(6):
        v["sigma"][s] = polys[s](*_coords(shape, S_OFF[s], dx))
    u0 = rng.standard_normal((3,) + shape)
    v["u"][:] = u0
    o.substep(2, st)
    I = _interior(shape)
    for i in range(3):
        Xc, Yc, Zc = _coords(shape, U_OFF[i], dx)
        div = sum(polys[VOIGT[i][j]].d(j, Xc, Yc, Zc) for j in range(3))
        Xi, Yi, Zi = _coords(shape, U_OFF[i], 1.0)
        rho_i = 2.0 + 0.05 * Xi + 0.03 * Yi + 0.02 * Zi
        alpha_i = 0.3 + 0.01 * Xi + 0.02 * Yi + 0.04 * Zi
        expect = (1.0 - dt * alpha_i) * u0[i] + dt / rho_i * div
        np.testing.assert_allclose(v["u"][i][I], expect[I], rtol=1e-9, atol=1e-9 * np.abs(expect[I]).max())


@pytest.mark.parametrize("mu0", [0.0, 1.7])
def test_stress_update_exact_on_quartics(mu0):
    """S4 with polynomial velocities: sigma^ii += dt (lambda div u + 2 mu d_i u^i),
    sigma^ij += dt mu (d_i u^j + d_j u^i), exactly (fluid and solid)."""
    rng = np.random.default_rng(12 + int(mu0 > 0))
    shape, dx, dt = (11, 10, 12), 0.25, 0.05
    desc = _desc(shape, dx, dt)
    lam0 = 3.0
    o = Oracle(desc, np.full(shape, 2.0), np.full(shape, lam0), np.full(shape, mu0), np.zeros(shape))
    polys = [Poly(rng) for _ in range(3)]
    st = o.new_state()
    v = Oracle.views(st)
    for i in range(3):
        v["u"][i] = polys[i](*_coords(shape, U_OFF[i], dx))
    s0 = rng.standard_normal((6,) + shape)
    v["sigma"][:] = s0
    o.substep(4, st)
    I = _interior(shape)
    for s in range(6):
        C = _coords(shape, S_OFF[s], dx)
        if s < 3:
            div = sum(polys[k].d(k, *C) for k in range(3))
            expect = s0[s] + dt * (lam0 * div + 2 * mu0 * polys[s].d(s, *C))
        else:
            i, j = [(1, 2), (0, 2), (0, 1)][s - 3]
            expect = s0[s] + dt * mu0 * (polys[j].d(i, *C) + polys[i].d(j, *C))
        np.testing.assert_allclose(v["sigma"][s][I], expect[I], rtol=1e-9, atol=1e-9 * np.abs(expect[I]).max())


def test_medium_averaging():
    """rho, alpha: arithmetic mean at velocity nodes (exact for linear fields);
    mu at shear nodes: harmonic mean of 4 nodes (alternating a, b -> 2ab/(a+b)),
    zero next to any fluid node."""
    shape = (6, 7, 8)
    X, Y, Z = _coords(shape, (0, 0, 0), 1.0)
    rho = 1000 + 10 * X + 20 * Y + 30 * Z
    alpha = 5 + X - Y + 2 * Z
    a, b = 1.0, 3.0
    mu = np.where(X % 2 == 0, a, b)
    mu[3, 3, 3] = 0.0
    o = Oracle(_desc(shape, 1.0, 0.1), rho, np.ones(shape), mu, alpha)
    rho_u, alpha_u, mu_s = o.stagger()
    for i in range(3):
        Xi, Yi, Zi = _coords(shape, U_OFF[i], 1.0)
        sl = [slice(None)] * 3
        sl[2 - i] = slice(0, shape[2 - i] - 1)  # last index is clamped, excluded
        sl = tuple(sl)
        np.testing.assert_allclose(rho_u[i][sl], (1000 + 10 * Xi + 20 * Yi + 30 * Zi)[sl], rtol=1e-14)
        np.testing.assert_allclose(alpha_u[i][sl], (5 + Xi - Yi + 2 * Zi)[sl], rtol=1e-13)
    hm = 2 * a * b / (a + b)
    # sigma12 and sigma13 straddle two x values -> harmonic of (a, b); sigma23 does not
    m12, m13, m23 = mu_s[2], mu_s[1], mu_s[0]
    ok = np.ones(shape, bool)
    ok[2:4, 2:4, 2:4] = False  # squares touching the fluid node
    inner = (slice(0, 5), slice(0, 6), slice(0, 7))
    np.testing.assert_allclose(m12[inner][ok[inner]], hm, rtol=1e-14)
    np.testing.assert_allclose(m13[inner][ok[inner]], hm, rtol=1e-14)
    np.testing.assert_allclose(m23[inner][ok[inner]], mu[inner][ok[inner]], rtol=1e-14)
    # every shear node whose square contains (3,3,3) is zero
    assert m12[3, 3, 3] == 0 and m12[3, 2, 2] == 0 and m12[3, 2, 3] == 0 and m12[3, 3, 2] == 0
    assert m13[3, 3, 3] == 0 and m13[2, 3, 2] == 0 and m23[2, 2, 3] == 0 and m23[3, 3, 3] == 0


# ---------------------------------------------------------------------------
# source and sampler
# ---------------------------------------------------------------------------
def test_first_sample_is_trilinear_interpolation_of_p0():
    """tau' loads sigma^ii = -p0/3 and Theta' reads -R(sigma11+sigma22+sigma33),
    so p_hat_0 = R p0: compare with scipy's order-1 interpolation."""
    from scipy.ndimage import map_coordinates
    shape = (9, 10, 11)
    rng = np.random.default_rng(5)
    p0 = rng.standard_normal(shape)
    rec = synth.random_receivers(40, shape, 6).astype(np.float64)
    rho, lam, mu, al, vmax = synth.random_medium(shape, 7)
    o = Oracle(_desc(shape, 1e-3, 1e-7, npml=2, vmax=vmax), rho, lam, mu, al)
    tr = o.forward(p0, rec, 0)
    ref = map_coordinates(p0, [rec[:, 2], rec[:, 1], rec[:, 0]], order=1)
    np.testing.assert_allclose(tr[0], ref, rtol=1e-13, atol=1e-13)


def test_readout_of_injection():
    """tau'^T tau' = (1/3) I: readout(inject(p0)) = p0 / 3."""
    shape = (5, 6, 7)
    p0 = np.random.default_rng(1).standard_normal(shape)
    o = Oracle(_desc(shape, 1.0, 0.1), *synth.fluid_medium(shape))
    np.testing.assert_allclose(o.readout(o.inject(p0)), p0 / 3.0, rtol=1e-15)


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
def _small_case(shape=(9, 8, 7), npml=2, seed=21):
    rho, lam, mu, al, vmax = synth.random_medium(shape, seed)
    dx = 1e-3
    dt = 0.3 * dx / vmax
    return Oracle(_desc(shape, dx, dt, npml=npml, vmax=vmax), rho, lam, mu, al)


def test_dense_transpose_of_H():
    """Brute force on a 7x8x9 grid: H^T assembled from L*M adjoint solves equals
    the transpose of H assembled from N forward solves (random heterogeneous
    medium with fluid nodes, absorption, 2-cell C-PML, 5 receivers, M = 12)."""
    o = _small_case()
    shape, N = o.shape, o.N
    rec = synth.random_receivers(5, shape, 22)
    nsteps = 11
    H = np.zeros((nsteps + 1, 5, N))
    e = np.zeros(N)
    for n in range(N):
        e[:] = 0
        e[n] = 1
        H[:, :, n] = o.forward(e.reshape(shape), rec, nsteps)
    H = H.reshape(-1, N)
    HT = np.zeros((N, H.shape[0]))
    g = np.zeros(H.shape[0])
    for q in range(H.shape[0]):
        g[:] = 0
        g[q] = 1
        HT[:, q] = o.adjoint(g.reshape(nsteps + 1, 5), rec).reshape(-1)
    scale = np.abs(H).max()
    assert scale > 0
    assert np.abs(HT - H.T).max() <= 1e-13 * scale


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_dense_transpose_of_each_substep(k):
    """Each scatter-form sub-update S_k^T is the transpose of S_k (27N x 27N,
    4x5x6 grid, 1-cell C-PML on every side, random medium)."""
    o = _small_case(shape=(6, 5, 4), npml=1, seed=31)
    n = 27 * o.N
    A = np.zeros((n, n))
    AT = np.zeros((n, n))
    for c in range(n):
        st = np.zeros((27,) + o.shape)
        st.reshape(-1)[c] = 1.0
        o.substep(k, st)
        A[:, c] = st.reshape(-1)
        st = np.zeros((27,) + o.shape)
        st.reshape(-1)[c] = 1.0
        o.substep(k, st, transpose=True)
        AT[:, c] = st.reshape(-1)
    assert np.abs(A).max() > 0
    assert np.abs(AT - A.T).max() <= 1e-14 * np.abs(A).max()


def test_inner_product_test_48():
    """<H p0, y> = <p0, H^T y> to 1e-12 with y = H p0 + noise (Sec. 5), skull-like
    48^3 medium with a 6-cell C-PML."""
    w = synth.skull(48, 1.2e-3, 6, 120, 64, seed=9)
    o = Oracle(w.desc.as_dict(), *w.medium)
    tr = o.forward(w.p0, w.rec, w.nsteps)
    rng = np.random.default_rng(1)
    y = tr + 0.1 * np.sqrt(np.mean(tr ** 2)) * rng.standard_normal(tr.shape)
    img = o.adjoint(y, w.rec)
    lhs = float(np.sum(tr * y))
    rhs = float(np.sum(w.p0.astype(np.float64) * img))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------------------
# energy conservation
# ---------------------------------------------------------------------------
def _energy(o, st_prev, st_next, lam, mu):
    """E_m = 1/2 sum_i <Q_i u_{m+1/2}, u_{m-1/2}> + 1/2 <sigma_m, C^+ sigma_m>."""
    rho_u, _, mu_s = o.stagger()
    vp, vn = Oracle.views(st_prev), Oracle.views(st_next)
    kin = 0.5 * np.sum(rho_u * vn["u"] * vp["u"])
    s = vp["sigma"]
    tr = s[0] + s[1] + s[2]
    solid = mu > 0
    # solid: C^-1 = (1/2mu) (I - lambda/(3 lambda + 2 mu) 1 1^T); fluid: 1 1^T / (9 lambda)
    ss = s[0] ** 2 + s[1] ** 2 + s[2] ** 2
    mu_safe = np.where(solid, mu, 1.0)
    e_sol = (ss - lam / (3 * lam + 2 * mu_safe) * tr ** 2) / (2 * mu_safe)
    e_flu = tr ** 2 / (9 * lam)
    pot = 0.5 * np.sum(np.where(solid, e_sol, e_flu))
    for q in range(3):
        m = mu_s[q]
        sh = s[3 + q]
        assert np.all(sh[m == 0] == 0)
        pot += 0.5 * np.sum(np.where(m > 0, sh ** 2 / np.where(m > 0, m, 1.0), 0.0))
    return kin + pot


def test_energy_conservation_heterogeneous():
    """alpha = 0, no PML, zero padding: the leapfrog energy is conserved to
    round-off over 200 steps in a random medium with fluid and solid nodes."""
    shape = (20, 22, 24)
    rho, lam, mu, _, vmax = synth.random_medium(shape, 41, fluid_fraction=0.4, absorb=False)
    dx = 1e-3
    o = Oracle(_desc(shape, dx, 0.3 * dx / vmax, npml=0, vmax=vmax), rho, lam, mu, np.zeros(shape))
    p0 = synth.bump_p0(shape, 6.0).astype(np.float64)
    st = o.inject(p0)
    lam64, mu64 = lam.astype(np.float64), mu.astype(np.float64)
    E = []
    for m in range(200):
        nxt = st.copy()
        o.step(nxt)
        E.append(_energy(o, st, nxt, lam64, mu64))
        st = nxt
    E = np.array(E)
    assert E[0] > 0
    assert np.abs(E - E[0]).max() <= 1e-12 * E[0]


def test_energy_decays_with_absorption():
    """With alpha > 0 (and no PML) the same energy is non-increasing."""
    shape = (16, 16, 16)
    rho, lam, mu, al, vmax = synth.random_medium(shape, 43, fluid_fraction=0.4, absorb=True)
    dx = 1e-3
    o = Oracle(_desc(shape, dx, 0.3 * dx / vmax, npml=0, vmax=vmax), rho, lam, mu, al * 50)
    st = o.inject(synth.bump_p0(shape, 5.0))
    E = []
    for m in range(80):
        nxt = st.copy()
        o.step(nxt)
        E.append(_energy(o, st, nxt, lam.astype(np.float64), mu.astype(np.float64)))
        st = nxt
    E = np.array(E)
    assert E[-1] < 0.95 * E[0]


# ---------------------------------------------------------------------------
# closed-form physics
# ---------------------------------------------------------------------------
def _radial_solution(f, R, r, ct):
    """Exact solution of the 3-D wave equation with radial initial value f(s)
    (support s < R) and zero initial rate: [(r-ct) f(|r-ct|) + (r+ct) f(r+ct)] / (2r)."""
    def fe(s):
        s = np.abs(s)
        return np.where(s < R, f(s), 0.0)
    return ((r - ct) * fe(r - ct) + (r + ct) * fe(r + ct)) / (2 * r)


def _bump_run(k, time_shift):
    """cos^2 bump of radius 2k cells seen by 24 receivers at radius 4.5k cells in a
    (16k)^3 water grid of fixed physical size; returns (relative L2 error, traces)."""
    n, R_cells, r_cells = 16 * k, 2.0 * k, 4.5 * k
    c, dx = 1500.0, 1e-3 * 32 / n
    dt = 0.3 * dx / c
    shape = (n, n, n)
    o = Oracle(_desc(shape, dx, dt), *synth.fluid_medium(shape, cp=c))
    ctr = (n - 1) / 2.0
    p0 = synth.bump_p0(shape, R_cells)
    rec = synth.fibonacci_sphere(24, r_cells, (ctr, ctr, ctr))
    nsteps = int(round((r_cells + R_cells) / 0.3))
    tr = o.forward(p0, rec, nsteps)
    rr = np.linalg.norm(rec.astype(np.float64) - ctr, axis=1) * dx
    t = (np.arange(nsteps + 1) + time_shift) * dt
    f = lambda s: np.cos(np.pi * s / (2 * R_cells * dx)) ** 2
    ref = _radial_solution(f, R_cells * dx, rr[None, :], c * t[:, None])
    return np.linalg.norm(tr - ref) / np.linalg.norm(ref)


def test_smooth_bump_closed_form_and_convergence():
    """Homogeneous fluid, cos^2 bump: the receiver traces converge to the exact
    radial solution at 2nd order under (dx, dt) -> 3/4 (dx, dt).

    The discrete initial state of Sec. 3 (Eq. (Propagate)) starts the velocity at
    zero at t = -dt/2 instead of t = 0.  For the pressure this is the same as an
    initial rate (dt/2) c^2 Lap p0, i.e. the discrete solution tracks the exact one
    at t + dt/2: compared at t the convergence is first order, compared at
    t + dt/2 it is second order.  Both facts are checked."""
    e3, e4 = _bump_run(3, 0.5), _bump_run(4, 0.5)
    order = math.log(e3 / e4) / math.log(4.0 / 3.0)
    assert e4 < 0.03, e4
    assert order >= 1.8, (e3, e4, order)
    u3, u4 = _bump_run(3, 0.0), _bump_run(4, 0.0)
    order0 = math.log(u3 / u4) / math.log(4.0 / 3.0)
    assert 0.8 <= order0 <= 1.3, (u3, u4, order0)


def test_uniform_ball_n_wave():
    """Uniform ball of radius 5 cells in water (the plain 64^3 workload without
    a PML): the receiver signal is the N-wave P (r - ct) / (2r).  The stair-cased
    ball is a step in space, so the discrete traces ring at the two jumps of the
    N-wave and their window L2 error is discretisation-limited (0.33 measured;
    bound 0.4).  The zero crossing of the N-wave is sharp: it must sit at
    t = r / c - dt / 2 (the half-step shift of the discrete initial state, see the
    smooth-bump test) to within half a step."""
    w = synth.plain_fluid_64(npml=0, nsteps=0)
    n, dx, dt, c = 64, w.desc.dx, w.desc.dt, 1500.0
    o = Oracle(w.desc.as_dict(), *w.medium)
    ctr = (n - 1) / 2.0
    r_cells = 20.0
    rec = synth.fibonacci_sphere(16, r_cells, (ctr, ctr, ctr))
    nsteps = int((r_cells + 8) / 0.3)
    tr = o.forward(w.p0, rec, nsteps)
    # radius of the sphere with the ball's volume (number of nodes inside)
    Reff = (3 * float(w.p0.sum()) / (4 * np.pi)) ** (1 / 3) * dx
    rr = np.linalg.norm(rec.astype(np.float64) - ctr, axis=1) * dx
    t = (np.arange(nsteps + 1) + 0.5) * dt
    ref = _radial_solution(lambda s: np.ones_like(s), Reff, rr[None, :], c * t[:, None])
    err = np.linalg.norm(tr - ref) / np.linalg.norm(ref)
    assert err < 0.4, err
    mean = tr.mean(axis=1)
    k = np.argmax(mean)  # positive lobe first
    kz = k + np.argmax(mean[k:] < 0)
    t0 = (kz - mean[kz] / (mean[kz] - mean[kz - 1])) * dt  # linear crossing
    assert abs(t0 - (rr.mean() / c - 0.5 * dt)) <= 0.5 * dt


# ---------------------------------------------------------------------------
# C-PML
# ---------------------------------------------------------------------------
def test_pml_profile_properties():
    n, npml, dx, dt, vmax, R0 = 60, 10, 1e-3, 1e-7, 3000.0, 1e-4
    for half in (False, True):
        d, beta, a, b, chi = pml_profile(n, npml, dx, dt, vmax, R0, 1e6, half)
        pos = np.arange(n) + (0.5 if half else 0.0)
        inside = (pos < npml) | (pos > n - 1 - npml)
        assert np.all(a[~inside] == 0) and np.all(b[~inside] == 1) and np.all(chi[~inside] == 0)
        assert np.all(chi[inside] == 1) and np.all((b[inside] > 0) & (b[inside] < 1)) and np.all(a[inside] < 0)
        left = pos < npml
        assert np.all(np.diff(d[left]) < 0)  # deeper into the layer -> larger d
    # continuous normal-incidence reflection exp(-2/c int d) equals R0 (midpoint rule)
    d_half, *_ = pml_profile(n, npml, dx, dt, vmax, R0, 1e6, True)
    integral = d_half[:npml].sum() * dx
    R = math.exp(-2.0 * integral / vmax)
    assert abs(math.log(R) / math.log(R0) - 1.0) < 0.01


def test_pml_reflection_small():
    """A smooth pulse leaving a 32^3 grid through an 8-cell C-PML: traces agree
    with the same pulse in a 64^3 grid with no layer (before that grid's own
    boundary echo arrives) to 1 % of the peak (0.39 % measured); without the
    layer the echo is large.  f0 (the CFS frequency shift) is set near the
    pulse's band, as the layer's design intends."""
    c, dx = 1500.0, 1e-3
    dt = 0.3 * dx / c
    def run(n, npml, off):
        shape = (n, n, n)
        d = _desc(shape, dx, dt, npml=npml, vmax=c)
        d["pml_f0"] = 3e5
        o = Oracle(d, *synth.fluid_medium(shape, cp=c))
        ctr = 15.5 + off
        p0 = synth.bump_p0(shape, 3.0, (ctr, ctr, ctr))
        rec = synth.fibonacci_sphere(12, 8.0, (ctr, ctr, ctr))
        return o.forward(p0, rec, 160)
    small = run(32, 8, 0)
    bare = run(32, 0, 0)
    big = run(64, 0, 16)
    peak = np.abs(big).max()
    err_pml = np.abs(small - big).max() / peak
    err_bare = np.abs(bare - big).max() / peak
    assert err_pml < 0.01, err_pml
    assert err_bare > 0.1, err_bare


# ---------------------------------------------------------------------------
# structure
# ---------------------------------------------------------------------------
def test_fluid_structure():
    """Homogeneous fluid (with C-PML): shear stresses stay exactly zero and the
    three normal stresses stay exactly equal."""
    shape = (14, 15, 16)
    o = Oracle(_desc(shape, 1e-3, 2e-7, npml=3), *synth.fluid_medium(shape))
    p0 = np.random.default_rng(3).standard_normal(shape) * (synth.ball_p0(shape, 4.0) > 0)
    st = o.run_state(p0, 25)
    s = Oracle.views(st)["sigma"]
    assert np.all(s[3:] == 0)
    assert np.array_equal(s[0], s[1]) and np.array_equal(s[1], s[2])
    assert np.abs(s[0]).max() > 0


def test_linearity():
    o = _small_case(shape=(10, 9, 8), npml=2, seed=51)
    rng = np.random.default_rng(52)
    p, q = rng.standard_normal((2,) + o.shape)
    rec = synth.random_receivers(7, o.shape, 53)
    Hp, Hq = o.forward(p, rec, 20), o.forward(q, rec, 20)
    Hpq = o.forward(2 * p - 3 * q, rec, 20)
    assert np.abs(Hpq - (2 * Hp - 3 * Hq)).max() <= 1e-12 * np.abs(Hpq).max()


def test_axis_permutation_equivariance():
    """Swapping x and y of the medium, p0 and receivers permutes the results."""
    shape = (10, 9, 8)
    rho, lam, mu, al, vmax = synth.random_medium(shape, 61)
    dx = 1e-3
    dt = 0.3 * dx / vmax
    rng = np.random.default_rng(62)
    p0 = rng.standard_normal(shape)
    rec = synth.random_receivers(6, shape, 63)
    o1 = Oracle(_desc(shape, dx, dt, 2, vmax), rho, lam, mu, al)
    sw = lambda a: np.ascontiguousarray(np.swapaxes(a, 1, 2))
    shape2 = (10, 8, 9)
    o2 = Oracle(_desc(shape2, dx, dt, 2, vmax), sw(rho), sw(lam), sw(mu), sw(al))
    rec2 = rec[:, [1, 0, 2]]
    t1, t2 = o1.forward(p0, rec, 15), o2.forward(sw(p0), rec2, 15)
    assert np.abs(t1 - t2).max() <= 1e-12 * np.abs(t1).max()
    y = rng.standard_normal(t1.shape)
    a1, a2 = o1.adjoint(y, rec), o2.adjoint(y, rec2)
    assert np.abs(sw(a1) - a2).max() <= 1e-12 * np.abs(a1).max()


# ---------------------------------------------------------------------------
# FISTA reference (oracle/fista.py) against an active-set NNLS solver
# ---------------------------------------------------------------------------
def test_fista_nn_reaches_nnls():
    """On a dense, well-posed problem with active constraints, the FISTA
    iterates of the oracle reach the non-negative least-squares solution that
    scipy.optimize.nnls (Lawson-Hanson active set) computes; a dropped
    projection, a wrong momentum or a sign error in the gradient fails this."""
    from scipy.optimize import nnls

    from oracle.fista import fista_nn
    rng = np.random.default_rng(21)
    m, n = 60, 30
    A = rng.standard_normal((m, n))
    x_true = np.maximum(0.0, rng.standard_normal(n))       # about half the entries at zero
    y = A @ x_true + 0.3 * rng.standard_normal(m)
    ref, _ = nnls(A, y)
    assert (ref == 0).sum() >= 5                           # the constraint is active somewhere
    L = np.linalg.norm(A, 2) ** 2
    it = fista_nn(lambda v: A @ v, lambda r: A.T @ r, y, np.zeros(n), L, 3000)
    assert np.linalg.norm(it[-1] - ref) / np.linalg.norm(ref) <= 1e-9
    # the accelerated method is ahead of plain projected gradient after 100 steps
    x = np.zeros(n)
    for _ in range(100):
        x = np.maximum(0.0, x - A.T @ (A @ x - y) / L)
    f = lambda v: 0.5 * np.sum((A @ v - y) ** 2)  # noqa: E731
    assert f(it[99]) - f(ref) <= f(x) - f(ref)


def _tv1d_qp(b, tau):
    """argmin_{x >= 0} 1/2 ||x - b||^2 + tau sum |x_{i+1} - x_i| as the QP in
    (x, t) with -t <= D x <= t, solved by SLSQP."""
    from scipy.optimize import minimize
    n = b.size
    D = np.zeros((n - 1, n))
    for i in range(n - 1):
        D[i, i], D[i, i + 1] = -1.0, 1.0
    f = lambda v: 0.5 * np.sum((v[:n] - b) ** 2) + tau * np.sum(v[n:])  # noqa: E731
    g = lambda v: np.concatenate([v[:n] - b, tau * np.ones(n - 1)])  # noqa: E731
    cons = [{"type": "ineq", "fun": lambda v: v[n:] - D @ v[:n], "jac": lambda v: np.hstack([-D, np.eye(n - 1)])},
            {"type": "ineq", "fun": lambda v: v[n:] + D @ v[:n], "jac": lambda v: np.hstack([D, np.eye(n - 1)])}]
    v0 = np.concatenate([np.maximum(b, 0), np.abs(D @ np.maximum(b, 0))])
    res = minimize(f, v0, jac=g, constraints=cons, bounds=[(0, None)] * n + [(None, None)] * (n - 1),
                   method="SLSQP", options={"ftol": 1e-13, "maxiter": 5000})
    return res.x[:n]


def test_tv_prox_matches_qp_1d():
    from oracle.fista import tv_prox_nn
    rng = np.random.default_rng(3)
    b = np.cumsum(rng.standard_normal(16)) * 0.6 + rng.standard_normal(16) * 0.4 + 1.3
    x = tv_prox_nn(b, 0.5, 20000)
    ref = _tv1d_qp(b, 0.5)
    assert (x == 0).sum() >= 2 and len(np.unique(np.round(x, 6))) >= 4   # active bound and plateaus
    assert np.abs(x - ref).max() <= 1e-6


def test_tv_prox_3d_reduces_to_1d():
    """An input that varies along one axis only: every line is the same 1-D
    problem, so the 3-D solution is the 1-D one broadcast (each axis in turn)."""
    from oracle.fista import tv_prox_nn
    rng = np.random.default_rng(5)
    f = np.cumsum(rng.standard_normal(12)) * 0.5 + 0.2
    ref = _tv1d_qp(f, 0.4)
    for axis in range(3):
        shape = [3, 4, 5]
        shape[axis] = 12
        b = np.broadcast_to(f.reshape([12 if a == axis else 1 for a in range(3)]), shape).copy()
        x = tv_prox_nn(b, 0.4, 20000)
        want = np.broadcast_to(ref.reshape([12 if a == axis else 1 for a in range(3)]), shape)
        assert np.abs(x - want).max() <= 1e-6


def test_difference_pair_is_adjoint():
    from oracle.fista import div3, grad3
    rng = np.random.default_rng(7)
    x = rng.standard_normal((5, 6, 7))
    p = rng.standard_normal((3, 5, 6, 7))
    assert abs(np.sum(grad3(x) * p) + np.sum(x * div3(p))) <= 1e-12 * np.sum(np.abs(x)) * np.sum(np.abs(p))
