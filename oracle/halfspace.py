"""Exact pressure of the fluid / elastic half-space validation problem -- TEST
INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module; it imports nothing from the product.

The paper validates H (Sec. 5) against the analytic pressure of a lossless
fluid (z > 0) over a linear isotropic solid (z < 0) with a planar interface,
excited by a line source parallel to y at x = 0, z = h_T in the fluid and
observed at x = d, z = h_R, the analytic response being computed with the
Cagniard-de Hoop method.  The FDTD source is an initial pressure whose profile
in the x-z plane is a Gaussian with a standard deviation of 1 mm.  The problem
is invariant along y, so the pressure is that of a 2-D initial-value problem:
p(0) = p0 (supported in the fluid), zero velocity, zero fields in the solid.

Derivation (written out so that each step can be checked):

1. Laplace transform in time (s > 0).  In the fluid the pressure obeys
   (Lap - s^2/c_f^2) P = -(s/c_f^2) p0, so P = (s/c_f^2) int G^(x_R, x') p0(x') dA'
   with G^ the Green's function, (Lap - s^2/c_f^2) G^ = -delta, satisfying the
   interface conditions.  Back in time: p(t) = (1/c_f^2) d/dt int G(t) p0 dA'.
2. Plane waves with horizontal slowness q, vertical slownesses
   gamma_j(q) = sqrt(1/c_j^2 + q^2) (Re >= 0; j = f, p, s):
     G^_direct    = (1/2pi) int exp(-s(gamma_f |z - z'| - i q (x - x'))) / (2 gamma_f) dq
                  = K0(s r / c_f) / (2 pi)  <->  H(t - r/c_f) / (2 pi sqrt(t^2 - r^2/c_f^2)),
     G^_reflected = (1/2pi) int R(q) exp(-s(gamma_f (z + z') - i q (x - x'))) / (2 gamma_f) dq.
3. R(q), the pressure reflection coefficient: with fluid pressure
   A (e^{s gamma_f z} + R e^{-s gamma_f z}) and solid potentials
   B e^{s gamma_p z}, C e^{s gamma_s z}, the conditions at z = 0 (normal
   velocity and normal stress continuous, shear stress zero) give
       R = (W - 1) / (W + 1),
       W = rho_s c_s^4 gamma_f [(2 q^2 + 1/c_s^2)^2 - 4 q^2 gamma_p gamma_s] / (rho_f gamma_p);
   q = 0 gives (Z_s - Z_f)/(Z_s + Z_f) and c_s -> 0 the fluid-fluid coefficient.
4. Cagniard-de Hoop: with the image distance r = |(x - x', z + z')| and the
   angle theta from the normal (sin theta = |x - x'| / r), the exponent
   gamma_f (z + z') - i q |x - x'| equals the real time t on the path
       q(v) = (i sin(theta) cosh v + cos(theta) sinh v) / c_f,  t = r cosh(v) / c_f,
   along which dq/dv = gamma_f, so that
       G_reflected(t) = c_f Re R(q(v)) / (2 pi r sinh v)   for t > r / c_f.
   Beyond the critical angle theta_c = arcsin(c_f / c_p) the path starts above
   the branch point i / c_p of gamma_p; the loop around that cut adds the head
   wave, on q(w) = i sin(theta - w) / c_f (right side of the cut),
   t = r cos(w) / c_f, w in [0, theta - theta_c], with weight -Im R.
5. Quadrature: polar coordinates (rho, phi) about the receiver for the direct
   term and about its mirror image (x_R, -h_R) for the reflected term,
   rho = c_f t cos(beta) on the hyperbolic branch (cosh v = sec beta) and
   rho = c_f t sec(w) on the head-wave segment.  These substitutions remove
   the inverse-square-root wavefront singularities, and the time derivative
   moves onto the source: d/dt [t p0(t/u)] = D = p0 + rho d(p0)/d(rho).
   Altogether
       p(t) = (1/2pi) [ int_0^{2pi} dphi int_0^{pi/2} D(c_f t cos b, phi) cos b db
                      + int_0^pi dphi int_0^{pi/2} Re R(q) D*(c_f t cos b, phi) cos b db
                      + int_0^pi dphi int_0^{theta-theta_c} (-Im R(q)) D*(c_f t sec w, phi) sec^2 w dw ],
   D* about the image point, where theta = theta(phi): sin theta = |cos phi|,
   cos theta = sin phi.

Readings (the paper is silent): the Gaussian is multiplied by a C^2 taper that
vanishes at the interface (initial pressure in the fluid only, as the analytic
solution requires); the y-invariant 3-D FDTD run stands for the 2-D problem.

Parity: pinned by ``tests/test_halfspace_pins.py``: R at normal incidence and
in the fluid-fluid limit; the Cagniard-path Green's function against the
Laplace-domain plane-wave integral of step 2 evaluated on the real q axis
(sub- and supercritical, so that the head-wave loop is checked); the direct
term against the Hankel-transform solution of a Gaussian in free space; a
rigid solid (R = 1) against the same Hankel solution at the image distance;
the Laplace transform of the whole reflected trace (hyperbolic and head-wave
terms, source integral and time derivative) against the plane-wave integral
over real q with the Gaussian's x-integral done exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class HalfSpace:
    """Fluid (z > 0) over an elastic solid (z < 0); SI units."""
    rho_f: float
    c_f: float
    rho_s: float
    c_p: float
    c_s: float

    @staticmethod
    def from_lame(rho_f, lam_f, rho_s, lam_s, mu_s):
        return HalfSpace(rho_f, math.sqrt(lam_f / rho_f), rho_s, math.sqrt((lam_s + 2 * mu_s) / rho_s),
                         math.sqrt(mu_s / rho_s))


# Sec. 5: rho_s 1200 kg/m^3, lambda_s 9.48 GPa, mu_s 2.352 GPa, rho_f 1000 kg/m^3, lambda_f 2.25 GPa.
PAPER_MEDIUM = HalfSpace.from_lame(1000.0, 2.25e9, 1200.0, 9.48e9, 2.352e9)


def vertical_slowness(q, c):
    """gamma = sqrt(1/c^2 + q^2) with Re >= 0; on the imaginary q axis past the
    branch point the value of the right side (Re q -> 0+) of the cut."""
    a = np.asarray(1.0 / (c * c) + np.asarray(q, dtype=np.complex128) ** 2, dtype=np.complex128)
    a = a.real + 1j * np.abs(a.imag)       # right-side limit; a no-op for Re q > 0, Im q >= 0
    return np.sqrt(a)


def reflection_coefficient(q, m: HalfSpace):
    """Pressure reflection coefficient R(q) of the fluid-solid interface (step 3)."""
    q = np.asarray(q, dtype=np.complex128)
    gf = vertical_slowness(q, m.c_f)
    gp = vertical_slowness(q, m.c_p)
    gs = vertical_slowness(q, m.c_s)
    q2 = q * q
    rayleigh = (2.0 * q2 + 1.0 / m.c_s ** 2) ** 2 - 4.0 * q2 * gp * gs
    W = m.rho_s * m.c_s ** 4 * rayleigh * gf / (m.rho_f * gp)
    return (W - 1.0) / (W + 1.0)


def critical_angle(m: HalfSpace) -> float:
    """theta_c = arcsin(c_f / c_p) (no head wave if c_p <= c_f)."""
    return math.asin(m.c_f / m.c_p) if m.c_p > m.c_f else math.pi / 2


def cagniard_q(theta, v, m: HalfSpace):
    """Hyperbolic branch of the Cagniard path, q(v) (step 4)."""
    return (1j * np.sin(theta) * np.cosh(v) + np.cos(theta) * np.sinh(v)) / m.c_f


def head_q(theta, w, m: HalfSpace):
    """Head-wave segment on the imaginary axis, q(w) = i sin(theta - w) / c_f."""
    return 1j * np.sin(theta - w) / m.c_f + 0.0


def reflected_green_laplace_cagniard(s, r, theta, m: HalfSpace, head=True):
    """int_0^inf e^{-st} G_reflected(t) dt computed on the Cagniard path
    (hyperbolic branch plus, beyond theta_c, the head-wave loop): used by the
    pin that checks the contour deformation against the real-axis integral
    (head=False drops the head-wave loop)."""
    from scipy.integrate import quad
    c = m.c_f

    def hyper(v):
        return math.exp(-s * r * math.cosh(v) / c) * float(np.real(reflection_coefficient(cagniard_q(theta, v, m), m)))

    vmax = math.acosh(1.0 + 60.0 * c / (s * r))
    val = quad(hyper, 0.0, vmax, limit=400, epsabs=0, epsrel=1e-11)[0]
    wh = theta - critical_angle(m)
    if head and wh > 0:
        def head_term(w):
            return math.exp(-s * r * math.cos(w) / c) * float(-np.imag(reflection_coefficient(head_q(theta, w, m), m)))
        val += quad(head_term, 0.0, wh, limit=400, epsabs=0, epsrel=1e-11)[0]
    return val / (2.0 * math.pi)


def reflected_green_laplace_plane_waves(s, r, theta, m: HalfSpace):
    """The same transform as the real-q-axis integral of step 2 (R real there)."""
    from scipy.integrate import quad
    x, z = r * math.sin(theta), r * math.cos(theta)

    def f(q):
        gf = math.sqrt(1.0 / m.c_f ** 2 + q * q)
        R = float(np.real(reflection_coefficient(q, m)))
        return R / gf * math.exp(-s * gf * z) * math.cos(s * q * x)

    # decay scale of exp(-s gamma_f z) in q is 1/(s z); integrate to 60 of those
    qmax = 60.0 / (s * z) + 1.0 / m.c_f
    val = quad(f, 0.0, qmax, limit=2000, epsabs=0, epsrel=1e-11)[0]
    return val / (2.0 * math.pi)       # (1/2pi) int_-inf^inf R/(2 gamma) ... = (1/2pi) int_0^inf R/gamma ...


# ---------------------------------------------------------------------------
# the initial pressure
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class LineSource:
    """p0(x, z) = exp(-((x - x_s)^2 + (z - h_t)^2) / (2 sigma^2)) T(z / a), with
    T(u) = u^3 (10 - 15 u + 6 u^2) on [0, 1], 0 below, 1 above (z = height above
    the interface, a = taper width)."""
    x_s: float
    h_t: float
    sigma: float
    taper: float

    def value_and_grad(self, x, z):
        """p0, dp0/dx, dp0/dz at arrays of points."""
        g = np.exp(-((x - self.x_s) ** 2 + (z - self.h_t) ** 2) / (2.0 * self.sigma ** 2))
        if self.taper > 0:
            u = np.clip(z / self.taper, 0.0, 1.0)
            T = u ** 3 * (10.0 - 15.0 * u + 6.0 * u * u)
            dT = np.where((z > 0) & (z < self.taper), 30.0 * u * u * (1.0 - u) ** 2 / self.taper, 0.0)
        else:
            T = (z > 0).astype(np.float64)
            dT = np.zeros_like(z)
        p = g * T
        gx = -(x - self.x_s) / self.sigma ** 2 * p
        gz = -(z - self.h_t) / self.sigma ** 2 * p + g * dT
        return p, gx, gz


def _radial_D(src: LineSource, cx, cz, rho, cosphi, sinphi):
    """D = p0 + rho d(p0)/d(rho) at the points centre + rho (cos phi, sin phi)."""
    x = cx + rho * cosphi
    z = cz + rho * sinphi
    p, gx, gz = src.value_and_grad(x, z)
    return p + rho * (cosphi * gx + sinphi * gz)


def pressure_trace(times, x_r, h_r, src: LineSource, m: HalfSpace, n_phi_direct=256, n_phi_image=2048,
                   n_beta=256, n_w=48, reflected=True, direct=True, head=True):
    """Exact pressure p(x_r, h_r, t) of the 2-D initial-value problem at the given
    times [s] (step 5).  The direct-term phi integral is periodic (trapezoid
    rule); the image-term phi integral runs over (0, pi) with an integrand that
    vanishes at both ends (trapezoid rule); beta and w use Gauss-Legendre, with
    w = w_h (1 - zeta^2) so that the square-root behaviour of R at the branch
    point i/c_p is integrated exactly.  direct / reflected / head select the
    terms (all by default)."""
    times = np.asarray(times, dtype=np.float64)
    c = m.c_f
    xb, wb = np.polynomial.legendre.leggauss(n_beta)
    beta = 0.25 * math.pi * (xb + 1.0)
    wbeta = 0.25 * math.pi * wb * np.cos(beta)                     # includes cos(beta)
    # direct term, polar about the receiver
    phid = 2.0 * math.pi * np.arange(n_phi_direct) / n_phi_direct
    cpd, spd = np.cos(phid)[:, None], np.sin(phid)[:, None]
    # image term, polar about (x_r, -h_r)
    phii = math.pi * (np.arange(n_phi_image) + 0.5) / n_phi_image
    cpi, spi = np.cos(phii)[:, None], np.sin(phii)[:, None]
    theta = np.arcsin(np.clip(np.abs(np.cos(phii)), 0.0, 1.0))[:, None]
    if reflected:
        ReR = np.real(reflection_coefficient(cagniard_q(theta, np.arctanh(np.sin(beta))[None, :], m), m))
        xz, wz = np.polynomial.legendre.leggauss(n_w)
        zeta = 0.5 * (xz + 1.0)
        wh = np.maximum(theta - critical_angle(m), 0.0)               # (n_phi, 1)
        w = wh * (1.0 - zeta[None, :] ** 2)
        ww = wh * 2.0 * zeta[None, :] * 0.5 * wz[None, :]            # dw = 2 w_h zeta dzeta; dzeta = wz/2
        ImR = -np.imag(reflection_coefficient(head_q(theta, w, m), m))
        head_weight = ImR * ww / np.cos(w) ** 2
    out = np.empty(times.shape)
    for i, t in enumerate(times.ravel()):
        rho_b = c * t * np.cos(beta)[None, :]
        val = 0.0
        if direct:
            Dd = _radial_D(src, x_r, h_r, rho_b, cpd, spd)
            val += (Dd * wbeta[None, :]).sum() * (2.0 * math.pi / n_phi_direct)
        if reflected:
            Di = _radial_D(src, x_r, -h_r, rho_b, cpi, spi)
            val += (ReR * Di * wbeta[None, :]).sum() * (math.pi / n_phi_image)
            if head:
                Dh = _radial_D(src, x_r, -h_r, c * t / np.cos(w), cpi, spi)
                val += (head_weight * Dh).sum() * (math.pi / n_phi_image)
        out.ravel()[i] = val / (2.0 * math.pi)
    return out


def reflected_pressure_laplace(s, x_r, h_r, src: LineSource, m: HalfSpace, n_q=1500, n_z=400):
    """Laplace transform of the reflected pressure at (x_r, h_r) computed
    without any contour deformation (step 1 with G^_reflected of step 2):
        P_r(s) = (s/c_f^2) (1/2pi) int R(q)/(2 gamma_f) e^{-s gamma_f h_r}
                 e^{i s q (x_r - x_s)} Fx(q) Fz(q) dq,
    Fx(q) = int e^{-i s q x'} exp(-x'^2/(2 sigma^2)) dx' = sqrt(2pi) sigma exp(-(s q sigma)^2/2)
    (the Gaussian's x-profile, exactly), Fz(q) = int_0^inf T(z'/a)
    exp(-(z'-h_t)^2/(2 sigma^2)) e^{-s gamma_f z'} dz' (Gauss-Legendre).  On
    real q the integrand is real and even, so the integral is twice the one
    over q > 0."""
    c = m.c_f
    qmax = 9.0 / (s * src.sigma)
    xq, wq = np.polynomial.legendre.leggauss(n_q)
    q = 0.5 * qmax * (xq + 1.0)
    wq = 0.5 * qmax * wq
    gf = np.sqrt(1.0 / c ** 2 + q * q)
    R = np.real(reflection_coefficient(q, m))
    zmax = src.h_t + 9.0 * src.sigma
    xz, wz = np.polynomial.legendre.leggauss(n_z)
    z = 0.5 * zmax * (xz + 1.0)
    wz = 0.5 * zmax * wz
    prof, _, _ = src.value_and_grad(np.full_like(z, src.x_s), z)          # T(z/a) exp(-(z-h_t)^2 / 2 sigma^2)
    Fz = (np.exp(-s * gf[:, None] * z[None, :]) * prof[None, :] * wz[None, :]).sum(axis=1)
    Fx = math.sqrt(2.0 * math.pi) * src.sigma * np.exp(-0.5 * (s * q * src.sigma) ** 2)
    integrand = R / (2.0 * gf) * np.exp(-s * gf * h_r) * np.cos(s * q * (x_r - src.x_s)) * Fx * Fz
    return (s / c ** 2) * (2.0 * (integrand * wq).sum()) / (2.0 * math.pi)


def laplace_of_trace(f, s, t_end, panels=40, nodes=16):
    """int_0^t_end e^{-s t} f(t) dt by panel Gauss-Legendre (f vectorised)."""
    x, w = np.polynomial.legendre.leggauss(nodes)
    edges = np.linspace(0.0, t_end, panels + 1)
    t = (0.5 * (edges[1:, None] - edges[:-1, None]) * (x[None, :] + 1.0) + edges[:-1, None]).ravel()
    wt = (0.5 * (edges[1:, None] - edges[:-1, None]) * w[None, :]).ravel()
    return float((np.exp(-s * t) * f(t) * wt).sum())


def gaussian_free_space(r, t, sigma, c):
    """Free-space 2-D pressure of p0 = exp(-r^2 / (2 sigma^2)), zero velocity,
    by the Hankel transform: p(r, t) = sigma^2 int_0^inf k J0(k r)
    exp(-k^2 sigma^2 / 2) cos(c k t) dk (independent of the polar quadrature)."""
    from scipy.integrate import quad
    from scipy.special import j0

    def f(k):
        return k * j0(k * r) * math.exp(-0.5 * (k * sigma) ** 2) * math.cos(c * k * t)

    kmax = 12.0 / sigma
    return sigma ** 2 * quad(f, 0.0, kmax, limit=800, epsabs=1e-13, epsrel=1e-11)[0]
