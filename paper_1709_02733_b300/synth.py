"""Seeded synthetic inputs: media, initial pressures, receivers, traces.

This module is shared by the oracle tests and the CUDA path and therefore
holds none of the method's arithmetic: it only builds inputs.  The paper's own
data (the X-ray CT skull, the vessel phantom, the acrylic-globe measurements)
are not available, so seeded stand-ins with the paper's shapes and material
values take their place (Sec. 6.1: skull rho 1850 kg/m^3, c_l 3.0 mm/us,
c_s 1.5 mm/us, alpha 0.1 /us; background water; vessels a few mm below the
inner skull surface; 11 x 400 transducers on the surrounding surface).

Conventions: arrays are float32, C-order ``(nz, ny, nx)`` (x fastest); SI units
(m, s, kg/m^3, Pa, 1/s); receiver positions are float32 ``(L, 3)`` as
``(x, y, z)`` in grid-index units on the integer lattice.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, field

import numpy as np

# CFL number used for every workload: dt = CFL * dx / c_max.
CFL = 0.3


@dataclass
class GridDesc:
    nx: int
    ny: int
    nz: int
    dx: float
    dt: float
    npml: int = 0
    pml_R0: float = 1e-4
    pml_f0: float = 1e6
    pml_vmax: float = 1500.0

    def as_dict(self):
        return asdict(self)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def N(self):
        return self.nx * self.ny * self.nz


def lame_from_speeds(cp, cs, rho):
    """(lambda, mu) from compressional / shear speed and density (Sec. 2.1)."""
    cp = np.asarray(cp, dtype=np.float64)
    cs = np.asarray(cs, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    mu = rho * cs * cs
    lam = rho * cp * cp - 2.0 * mu
    return lam, mu


def fluid_medium(shape, cp=1500.0, rho=1000.0):
    """Homogeneous fluid: returns (rho, lambda, mu, alpha) float32 arrays."""
    lam = rho * cp * cp
    return (np.full(shape, rho, np.float32), np.full(shape, lam, np.float32),
            np.zeros(shape, np.float32), np.zeros(shape, np.float32))


def _smooth_noise(rng, shape, sigma_cells):
    from scipy.ndimage import gaussian_filter
    n = rng.standard_normal(shape).astype(np.float32)
    n = gaussian_filter(n, sigma=sigma_cells, mode="wrap", truncate=3.0)
    m = np.abs(n).max()
    return n / m if m > 0 else n


def _centered_radius(shape):
    nz, ny, nx = shape
    z = np.arange(nz, dtype=np.float32) - (nz - 1) / 2.0
    y = np.arange(ny, dtype=np.float32) - (ny - 1) / 2.0
    x = np.arange(nx, dtype=np.float32) - (nx - 1) / 2.0
    return np.sqrt(z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2)


@dataclass
class SkullGeometry:
    W: float          # half-width of the PML-free region [m]
    R_outer: float    # outer skull radius [m]
    R_inner: float    # inner skull radius [m]
    R_rec: float      # receiver radius [m]


def skull_geometry(n, dx, npml):
    W = (n / 2.0 - npml) * dx
    Ro = 0.70 * W
    Ri = Ro - 7e-3
    return SkullGeometry(W=W, R_outer=Ro, R_inner=max(Ri, 2 * dx), R_rec=0.9 * W)


SKULL_CP, SKULL_CS, SKULL_RHO, SKULL_ALPHA = 2900.0, 1400.0, 1850.0, 1e5
WATER_CP, WATER_RHO = 1480.0, 1000.0
TISSUE_CP, TISSUE_RHO = 1560.0, 1050.0
SKULL_VMAX = SKULL_CP * 1.05


def skull_medium(n, dx, npml, seed):
    """Skull-like elastic shell in water (cubic grid of side n).

    Water (cp 1480, rho 1000, cs 0, alpha 0) outside a spherical shell 7 mm
    thick centred in the grid, outer radius 0.7 W with W the half-width of the
    region inside the PML; shell cp 2900, cs 1400, rho 1850, each scaled by
    (1 + 0.05 n_k) with n_k seeded white noise (seed + k) Gaussian-smoothed with
    sigma 3 cells and normalised to max |n_k| = 1; shell alpha 1e5 /s; soft
    tissue (cp 1560, rho 1050, cs 0, alpha 0) inside.  The shell mask is
    evaluated at the integer nodes (stair-cased, like a segmentation mask).
    """
    shape = (n, n, n)
    geo = skull_geometry(n, dx, npml)
    r = _centered_radius(shape) * np.float32(dx)
    shell = (r <= geo.R_outer) & (r > geo.R_inner)
    inner = r <= geo.R_inner
    rho = np.full(shape, WATER_RHO, np.float32)
    cp = np.full(shape, WATER_CP, np.float32)
    cs = np.zeros(shape, np.float32)
    alpha = np.zeros(shape, np.float32)
    rho[inner] = TISSUE_RHO
    cp[inner] = TISSUE_CP
    # noise only over the bounding box of the shell
    c = (n - 1) / 2.0
    h = int(math.ceil(geo.R_outer / dx)) + 1
    lo, hi = max(0, int(math.floor(c - h))), min(n, int(math.ceil(c + h)) + 1)
    box = (slice(lo, hi),) * 3
    sub_shell = shell[box]
    vals = []
    for k, base in enumerate((SKULL_CP, SKULL_CS, SKULL_RHO)):
        rng = np.random.default_rng(seed + k)
        noise = _smooth_noise(rng, sub_shell.shape, 3.0)
        vals.append(base * (1.0 + 0.05 * noise))
    cp[box][sub_shell] = vals[0][sub_shell]
    cs[box][sub_shell] = vals[1][sub_shell]
    rho[box][sub_shell] = vals[2][sub_shell]
    alpha[shell] = SKULL_ALPHA
    lam, mu = lame_from_speeds(cp, cs, rho)
    return rho, lam.astype(np.float32), mu.astype(np.float32), alpha


def ball_p0(shape, radius_cells, center=None, amplitude=1.0):
    """Uniform ball: amplitude on integer nodes within radius of the centre."""
    nz, ny, nx = shape
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    z = np.arange(nz)[:, None, None] - center[2]
    y = np.arange(ny)[None, :, None] - center[1]
    x = np.arange(nx)[None, None, :] - center[0]
    r = np.sqrt(x * x + y * y + z * z)
    return np.where(r <= radius_cells, amplitude, 0.0).astype(np.float32)


def bump_p0(shape, radius_cells, center=None, amplitude=1.0):
    """Smooth radial bump amplitude * cos^2(pi r / (2 R)) for r < R."""
    nz, ny, nx = shape
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    z = np.arange(nz)[:, None, None] - center[2]
    y = np.arange(ny)[None, :, None] - center[1]
    x = np.arange(nx)[None, None, :] - center[0]
    r = np.sqrt(x * x + y * y + z * z)
    v = np.where(r < radius_cells, np.cos(np.pi * r / (2.0 * radius_cells)) ** 2, 0.0)
    return (amplitude * v).astype(np.float32)


def tubes_p0(n, dx, npml, seed, ntubes=40):
    """Vessel-like initial pressure: seeded straight tubes inside the skull.

    Each tube is a segment whose end points are uniform in the ball of radius
    R_inner - 3 cells - r_tube, radius r_tube ~ U[1, 3] cells, amplitude
    ~ U[0.5, 1]; tubes are rasterised by distance-to-segment (max-combined),
    Gaussian-smoothed (sigma 1 cell) and cut to zero outside R_inner - 2 cells,
    which keeps the support in the fluid and away from the PML.
    """
    from scipy.ndimage import gaussian_filter
    geo = skull_geometry(n, dx, npml)
    Ri = geo.R_inner / dx
    c = (n - 1) / 2.0
    rng = np.random.default_rng(seed + 10)
    p0 = np.zeros((n, n, n), np.float32)
    for _ in range(ntubes):
        rt = rng.uniform(1.0, 3.0)
        amp = rng.uniform(0.5, 1.0)
        Rb = max(Ri - 3.0 - rt, 1.0)
        ends = []
        for _e in range(2):
            v = rng.standard_normal(3)
            v /= np.linalg.norm(v)
            ends.append(c + v * Rb * rng.uniform(0.0, 1.0) ** (1.0 / 3.0))
        a, b = ends
        lo = np.maximum(np.floor(np.minimum(a, b) - rt - 1), 0).astype(int)
        hi = np.minimum(np.ceil(np.maximum(a, b) + rt + 2), n).astype(int)
        zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]),
                                 indexing="ij")
        P = np.stack([xx, yy, zz], -1).astype(np.float64)
        ab = b - a
        t = np.clip(((P - a) @ ab) / max(ab @ ab, 1e-12), 0.0, 1.0)
        d = np.linalg.norm(P - (a + t[..., None] * ab), axis=-1)
        blk = p0[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        np.maximum(blk, np.where(d <= rt, amp, 0.0).astype(np.float32), out=blk)
    p0 = gaussian_filter(p0, sigma=1.0, mode="constant", truncate=3.0)
    r = _centered_radius(p0.shape)
    p0[r > Ri - 2.0] = 0.0
    return p0.astype(np.float32)


def fibonacci_sphere(L, radius_cells, center):
    """L points of a Fibonacci lattice on a full sphere (golden-angle spiral)."""
    l = np.arange(L, dtype=np.float64)
    cos_t = 1.0 - 2.0 * (l + 0.5) / L
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t ** 2))
    phi = l * math.pi * (3.0 - math.sqrt(5.0))
    pts = np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], -1) * radius_cells
    return (pts + np.asarray(center, dtype=np.float64)).astype(np.float32)


def fibonacci_hemisphere(L, radius_cells, center):
    """L points of a Fibonacci lattice on the upper (+z) hemisphere."""
    l = np.arange(L, dtype=np.float64)
    cos_t = (l + 0.5) / L
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t ** 2))
    phi = l * math.pi * (3.0 - math.sqrt(5.0))
    pts = np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], -1) * radius_cells
    return (pts + np.asarray(center, dtype=np.float64)).astype(np.float32)


def random_medium(shape, seed, fluid_fraction=0.3, absorb=True):
    """Random heterogeneous elastic medium for small parity / adjoint tests.

    Density 900..2000, cp 1400..3000, cs up to 0.5 cp, zeroed (fluid) on a
    random subset of nodes, alpha up to 2e5 /s.  Returns float32 arrays and
    the maximum compressional speed.
    """
    rng = np.random.default_rng(seed)
    rho = rng.uniform(900.0, 2000.0, shape)
    cp = rng.uniform(1400.0, 3000.0, shape)
    cs = cp * rng.uniform(0.1, 0.5, shape)
    cs[rng.random(shape) < fluid_fraction] = 0.0
    alpha = rng.uniform(0.0, 2e5, shape) if absorb else np.zeros(shape)
    lam, mu = lame_from_speeds(cp, cs, rho)
    return (rho.astype(np.float32), lam.astype(np.float32), mu.astype(np.float32),
            alpha.astype(np.float32), float(cp.max()))


def random_receivers(L, shape, seed, margin=0.0):
    """L receivers uniform in the box [margin, n - 2 - margin] per axis."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    hi = np.array([nx - 2, ny - 2, nz - 2], dtype=np.float64) - margin
    return (margin + rng.random((L, 3)) * (hi - margin)).astype(np.float32)


def band_limited_traces(nsteps, L, seed, dt, f_hi=2e6):
    """Seeded random traces (nsteps + 1, L), low-passed below f_hi (FFT mask)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nsteps + 1, L))
    X = np.fft.rfft(x, axis=0)
    f = np.fft.rfftfreq(nsteps + 1, d=dt)
    X[f > f_hi] = 0.0
    y = np.fft.irfft(X, n=nsteps + 1, axis=0)
    s = np.abs(y).max()
    return (y / s if s > 0 else y).astype(np.float32)


# --------------------------------------------------------------------------
# Named workloads (shapes and materials from the paper's studies, Sec. 6.1)
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    desc: GridDesc
    nsteps: int
    rho: np.ndarray = field(repr=False)
    lam: np.ndarray = field(repr=False)
    mu: np.ndarray = field(repr=False)
    alpha: np.ndarray = field(repr=False)
    p0: np.ndarray = field(repr=False)
    rec: np.ndarray = field(repr=False)

    @property
    def medium(self):
        return self.rho, self.lam, self.mu, self.alpha


def plain_fluid_64(npml=3, nsteps=400):
    """64^3 homogeneous fluid, dx 0.5 mm, dt at CFL 0.3 (100 ns), p0 = unit ball
    of radius 5 cells at the centre, 128 full-sphere Fibonacci receivers at
    radius 28 cells."""
    n, dx, cp = 64, 0.5e-3, 1500.0
    d = GridDesc(n, n, n, dx, CFL * dx / cp, npml=npml, pml_vmax=cp)
    rho, lam, mu, alpha = fluid_medium(d.shape, cp=cp)
    c = (n - 1) / 2.0
    p0 = ball_p0(d.shape, 5.0)
    rec = fibonacci_sphere(128, 28.0, (c, c, c))
    return Workload("plain-fluid-64", d, nsteps, rho, lam, mu, alpha, p0, rec)


def skull(n, dx, npml, nsteps, L, seed, name=None):
    """Skull-like workload: skull_medium + tubes_p0 + L hemisphere receivers."""
    d = GridDesc(n, n, n, dx, CFL * dx / SKULL_VMAX, npml=npml, pml_vmax=SKULL_VMAX)
    rho, lam, mu, alpha = skull_medium(n, dx, npml, seed)
    p0 = tubes_p0(n, dx, npml, seed)
    geo = skull_geometry(n, dx, npml)
    c = (n - 1) / 2.0
    rec = fibonacci_hemisphere(L, geo.R_rec / dx, (c, c, c))
    return Workload(name or f"skull-{n}", d, nsteps, rho, lam, mu, alpha, p0, rec)


def skull_256():
    return skull(256, 0.4e-3, 16, 2000, 512, seed=2, name="skull-256")


def skull_192():
    return skull(192, 0.4e-3, 12, 1500, 256, seed=3, name="skull-192")


def skull_512():
    return skull(512, 0.2e-3, 20, 4000, 1024, seed=4, name="skull-512")


@dataclass
class HalfSpaceCase:
    """y-invariant fluid / solid half-space (the validation set-up of Sec. 5).

    The medium and p0 are given as 2-D (nz, nx) profiles; ``p0_y`` is the
    range [j0, j1) of y planes that carry p0 (2 cells clear of the y layers);
    the caller broadcasts them along y (on the device for the full-size grid).
    Node plane k0 - 1 is the last solid plane and k0 the first fluid one, so
    the interface lies at z = k0 - 1/2 (index units); heights above it are
    (k - k0 + 1/2) dx.  The source line is at x index ``x_src``."""
    desc: GridDesc
    nsteps: int
    k0: int
    x_src: int
    rho: np.ndarray = field(repr=False)
    lam: np.ndarray = field(repr=False)
    mu: np.ndarray = field(repr=False)
    alpha: np.ndarray = field(repr=False)
    p0: np.ndarray = field(repr=False)
    p0_y: tuple = (0, 0)
    rec: np.ndarray = field(repr=False, default=None)
    params: dict = field(default_factory=dict)


def halfspace(ny=2312, n_xz=388, dx=0.15e-3, npml=30, dt=12.5e-9, t_end=10e-6, h_t=2.1e-3, h_r=2.1e-3, d=2.1e-3,
              sigma=1e-3, taper=0.75e-3):
    """Sec. 5: water (rho 1000 kg/m^3, lambda 2.25 GPa) over a lossless solid
    (rho 1200 kg/m^3, lambda 9.48 GPa, mu 2.352 GPa); box 58.2 x 346.8 x
    58.2 mm (x, y, z) at dx 0.15 mm with a 4.5 mm C-PML; z normal to the
    interface, y along the line source; line source at height h_t, receiver
    at horizontal offset d and height h_r; p0 a Gaussian of std sigma in the
    x-z plane times the C^2 taper u^3 (10 - 15 u + 6 u^2), u = height / taper
    clipped to [0, 1] (zero at the interface, so p0 lies in the fluid).
    dt 12.5 ns (two steps per 40 MHz sample; CFL 0.29 at c_p 3.44 mm/us)."""
    nz = nx = n_xz
    rho_f, lam_f = 1000.0, 2.25e9
    rho_s, lam_s, mu_s = 1200.0, 9.48e9, 2.352e9
    c_p = math.sqrt((lam_s + 2 * mu_s) / rho_s)
    desc = GridDesc(nx, ny, nz, dx, dt, npml=npml, pml_vmax=c_p)
    k0 = nz // 2
    fluid = (np.arange(nz) >= k0)[:, None] & np.ones((1, nx), bool)
    rho = np.where(fluid, rho_f, rho_s).astype(np.float32)
    lam = np.where(fluid, lam_f, lam_s).astype(np.float32)
    mu = np.where(fluid, 0.0, mu_s).astype(np.float32)
    alpha = np.zeros((nz, nx), np.float32)
    off = int(round(d / dx))
    x_src = nx // 2 - off // 2
    height = (np.arange(nz, dtype=np.float64) - k0 + 0.5) * dx
    xo = (np.arange(nx, dtype=np.float64) - x_src) * dx
    u = np.clip(height / taper, 0.0, 1.0)
    T = u ** 3 * (10.0 - 15.0 * u + 6.0 * u * u)
    g = np.exp(-(xo[None, :] ** 2 + (height[:, None] - h_t) ** 2) / (2.0 * sigma ** 2))
    p0 = (g * T[:, None]).astype(np.float32)
    rec = np.array([[x_src + d / dx, ny // 2, k0 - 0.5 + h_r / dx]], np.float32)
    nsteps = int(round(t_end / dt))
    params = dict(rho_f=rho_f, lam_f=lam_f, rho_s=rho_s, lam_s=lam_s, mu_s=mu_s, h_t=h_t, h_r=h_r, d=d,
                  sigma=sigma, taper=taper)
    return HalfSpaceCase(desc, nsteps, k0, x_src, rho, lam, mu, alpha, p0, (npml + 2, ny - npml - 2), rec, params)
