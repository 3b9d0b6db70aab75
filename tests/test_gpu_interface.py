"""Fluid-solid interface: normal-incidence reflection coefficient.

The paper validates its operator against the analytic response of a fluid
over a solid half-space (Sec. 6.1, Cagniard-de Hoop).  Its simplest exact
special case is a plane pressure wave at normal incidence, which reflects from
the interface with the pressure coefficient R = (Z2 - Z1) / (Z2 + Z1),
Z = rho * c_p, and converts no shear wave.  A laterally uniform Gaussian p0
in water splits into two plane pulses of half amplitude; the down-going one
passes a receiver on the centre column and comes back from a skull-like solid
with amplitude R / 2.  The grid is wide enough that the diffraction from the
lateral edges of the plane source reaches the receiver only after the
reflection has passed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_02733_b300 import pact, synth  # noqa: E402
from paper_1709_02733_b300.synth import GridDesc  # noqa: E402


def test_normal_incidence_reflection_coefficient():
    from paper_1709_02733_b300 import build
    build.build()
    n, nz, dx, P = 192, 192, 0.2e-3, 10
    z0, zs, zr, width = 120, 70, 95, 3.0          # interface, source plane, receiver, pulse sigma [cells]
    rho1, c1 = 1000.0, 1500.0
    rho2, c2, cs2 = 1850.0, 2900.0, 1400.0
    shape = (nz, n, n)
    z = np.arange(nz)[:, None, None]
    fluid = np.broadcast_to(z < z0, shape)
    rho = np.where(fluid, rho1, rho2).astype(np.float32)
    mu = np.where(fluid, 0.0, rho2 * cs2 ** 2).astype(np.float32)
    lam = np.where(fluid, rho1 * c1 ** 2, rho2 * (c2 ** 2 - 2 * cs2 ** 2)).astype(np.float32)
    alpha = np.zeros(shape, np.float32)
    dt = 0.3 * dx / c2
    d = GridDesc(n, n, nz, dx, dt, npml=P, pml_vmax=c2)
    p0 = np.broadcast_to(np.exp(-0.5 * ((z - zs) / width) ** 2), shape).astype(np.float32)
    c = (n - 1) / 2.0
    rec = np.array([[c, c, float(zr)]], np.float32)
    steps_per_cell = dx / (c1 * dt)
    t_inc = (zr - zs) * steps_per_cell
    t_ref = ((z0 - 0.5 - zs) + (z0 - 0.5 - zr)) * steps_per_cell
    nsteps = int(t_ref + 12 * steps_per_cell)
    # diffraction from the lateral edges of the plane source needs (n/2) cells
    assert t_ref + 8 * steps_per_cell < (n / 2 - 2) * steps_per_cell
    g = pact.Grid(d)
    g.set_medium(*[torch.from_numpy(np.ascontiguousarray(m)).cuda() for m in (rho, lam, mu, alpha)])
    tr = g.forward(torch.from_numpy(np.ascontiguousarray(p0)).cuda(), rec, nsteps).cpu().numpy()[:, 0]
    w = int(6 * steps_per_cell)
    inc = tr[int(t_inc) - w:int(t_inc) + w]
    ref = tr[int(t_ref) - w:int(t_ref) + w]
    a_inc = inc[np.argmax(np.abs(inc))]
    a_ref = ref[np.argmax(np.abs(ref))]
    Z1, Z2 = rho1 * c1, rho2 * c2
    R = (Z2 - Z1) / (Z2 + Z1)
    assert abs(a_inc - 0.5) <= 0.01                     # half of the unit pulse goes down
    assert abs(a_ref / a_inc - R) <= 0.01, (a_ref / a_inc, R)
    # the reflection arrives on time (within one cell of travel)
    t_peak = int(t_ref) - w + int(np.argmax(np.abs(ref)))
    assert abs(t_peak - t_ref) <= steps_per_cell
