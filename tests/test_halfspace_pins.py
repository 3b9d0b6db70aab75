"""Pins of the half-space validation oracle (oracle/halfspace.py) against
results fixed independently of its Cagniard-path quadrature."""
import math

import numpy as np
import pytest

from oracle import halfspace as hs

M = hs.PAPER_MEDIUM


def test_paper_medium_speeds():
    # Sec. 5 Lame parameters: c_f = 1500, c_p = sqrt(14.184e9 / 1200), c_s = sqrt(2.352e9 / 1200) = 1400 m/s
    assert M.c_f == pytest.approx(1500.0, rel=1e-12)
    assert M.c_p == pytest.approx(math.sqrt(14.184e9 / 1200.0), rel=1e-12)
    assert M.c_s == pytest.approx(1400.0, rel=1e-12)


def test_reflection_normal_incidence():
    R0 = complex(hs.reflection_coefficient(0.0, M))
    Zf, Zs = M.rho_f * M.c_f, M.rho_s * M.c_p
    assert abs(R0 - (Zs - Zf) / (Zs + Zf)) < 1e-13


@pytest.mark.parametrize("q", [0.0, 2e-4, 1e-3, 1j * 1e-4, 1j * 2.5e-4])
def test_reflection_fluid_fluid_limit(q):
    # a solid with vanishing shear speed is a fluid: R -> (rho2 g1 - rho1 g2) / (rho2 g1 + rho1 g2)
    m = hs.HalfSpace(1000.0, 1500.0, 1300.0, 2500.0, 1e-4)
    g1 = hs.vertical_slowness(q, m.c_f)
    g2 = hs.vertical_slowness(q, m.c_p)
    ref = (m.rho_s * g1 - m.rho_f * g2) / (m.rho_s * g1 + m.rho_f * g2)
    assert abs(complex(hs.reflection_coefficient(q, m)) - complex(ref)) < 1e-7


@pytest.mark.parametrize("theta", [0.25, 0.6, 1.1])        # theta_c = 0.452: one sub-, two supercritical
@pytest.mark.parametrize("sr_over_c", [0.7, 2.5])
def test_cagniard_path_matches_plane_wave_integral(theta, sr_over_c):
    """The Laplace transform of the Cagniard-path Green's function (hyperbolic
    branch plus head-wave loop) equals the plane-wave integral over real q,
    where nothing is deformed: checks the path, the side of the branch cut and
    the sign and extent of the head-wave term."""
    r = 4.7e-3
    s = sr_over_c * M.c_f / r
    a = hs.reflected_green_laplace_cagniard(s, r, theta, M)
    b = hs.reflected_green_laplace_plane_waves(s, r, theta, M)
    assert abs(a - b) <= 1e-8 * abs(b), (a, b)
    if theta > hs.critical_angle(M):
        # the head-wave loop carries a share of the transform far above the tolerance
        c = hs.reflected_green_laplace_cagniard(s, r, theta, M, head=False)
        assert abs(c - b) > 1e-4 * abs(b), (c, b)


def test_direct_term_matches_hankel_solution():
    src = hs.LineSource(x_s=0.0, h_t=12e-3, sigma=1e-3, taper=0.75e-3)      # taper irrelevant 12 sigma away
    x_r, h_r = 2.1e-3, 12e-3
    times = np.array([0.0, 0.4e-6, 1.4e-6, 2.5e-6, 4.0e-6])
    p = hs.pressure_trace(times, x_r, h_r, src, M, reflected=False)
    ref = np.array([hs.gaussian_free_space(2.1e-3, t, 1e-3, M.c_f) for t in times])
    assert np.max(np.abs(p - ref)) < 1e-7, (p, ref)


def test_rigid_solid_is_an_image_source():
    rigid = hs.HalfSpace(1000.0, 1500.0, 1e15, 3438.0, 1400.0)
    assert abs(complex(hs.reflection_coefficient(1j * 5e-4, rigid)) - 1.0) < 1e-9
    h = 8e-3
    src = hs.LineSource(x_s=0.0, h_t=h, sigma=1e-3, taper=0.75e-3)
    x_r, h_r = 2.1e-3, h
    r_img = math.hypot(2.1e-3, 2 * h)
    times = np.array([9.5e-6, 10.8e-6, 11.5e-6, 12.5e-6])
    p = hs.pressure_trace(times, x_r, h_r, src, rigid)
    ref = np.array([hs.gaussian_free_space(2.1e-3, t, 1e-3, 1500.0) + hs.gaussian_free_space(r_img, t, 1e-3, 1500.0)
                    for t in times])
    assert np.max(np.abs(p - ref)) < 1e-6, (p, ref)


def test_synth_halfspace_rasterises_the_same_source():
    """The input generator's p0 and geometry agree with the oracle's continuous
    definition (two independent writings of the same set-up)."""
    from paper_1709_02733_b300 import synth
    c = synth.halfspace(ny=96)
    d, p = c.desc, c.params
    src = hs.LineSource(0.0, p["h_t"], p["sigma"], p["taper"])
    x = (np.arange(d.nx) - c.x_src) * d.dx
    z = (np.arange(d.nz) - c.k0 + 0.5) * d.dx                 # height above the interface
    ref, _, _ = src.value_and_grad(x[None, :], z[:, None])
    np.testing.assert_allclose(c.p0, ref, rtol=2e-7, atol=1e-30)
    assert not c.p0[:c.k0].any()                               # nothing in the solid
    m = hs.HalfSpace.from_lame(p["rho_f"], p["lam_f"], p["rho_s"], p["lam_s"], p["mu_s"])
    assert m == hs.PAPER_MEDIUM
    assert np.all(c.mu[c.k0:] == 0) and np.all(c.mu[:c.k0] == np.float32(p["mu_s"]))
    # receiver at (d, h_R) from the source line, on the centre y plane
    assert c.rec[0, 0] * d.dx == pytest.approx(c.x_src * d.dx + p["d"], rel=1e-6)
    assert (c.rec[0, 2] - (c.k0 - 0.5)) * d.dx == pytest.approx(p["h_r"], rel=1e-6)
    j0, j1 = c.p0_y
    assert j0 == d.npml + 2 and d.ny - j1 == d.npml + 2         # p0 planes 2 nodes clear of the y layers
    assert m.c_p * d.dt / d.dx < 6 / (7 * math.sqrt(3))


def test_reflected_trace_laplace_transform():
    """The Laplace transform of the oracle's reflected trace (Cagniard path,
    head-wave loop, source integral in image-polar coordinates, time derivative
    moved onto p0) equals the plane-wave integral over real q, where the
    Gaussian's x-integral is exact and nothing is deformed.  At s = 1.2 /us the
    head-wave term carries 9 % of the transform; the bound is 2e-4 (the
    reduced quadrature used here agrees to 2e-5)."""
    src = hs.LineSource(0.0, 2.1e-3, 1e-3, 0.75e-3)
    kw = dict(n_phi_direct=64, n_phi_image=512, n_beta=128, n_w=32)
    s = 1.2e6
    a = hs.laplace_of_trace(lambda t: hs.pressure_trace(t, 2.1e-3, 2.1e-3, src, M, direct=False, **kw), s,
                            40.0 / s, panels=34, nodes=12)
    b = hs.reflected_pressure_laplace(s, 2.1e-3, 2.1e-3, src, M)
    assert abs(a - b) <= 2e-4 * abs(b), (a, b)
