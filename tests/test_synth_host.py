"""The seeded workloads obey the rules the operator and the paper put on its
inputs (host only): p0 in the fluid and at least 2 nodes clear of the C-PML
(Appendix A.3), admissible media (positive density, positive P and bulk
moduli), the 4th-order CFL limit, and receivers inside [0, n - 2]."""
import math

import numpy as np
import pytest

from paper_1709_02733_b300 import synth


def _band(shape, band):
    nz, ny, nx = shape
    z, y, x = np.ogrid[:nz, :ny, :nx]
    d = np.minimum(np.minimum(np.minimum(x, nx - 1 - x), np.minimum(y, ny - 1 - y)), np.minimum(z, nz - 1 - z))
    return d < band


@pytest.mark.parametrize("make", [synth.skull_192, lambda: synth.skull(96, 0.4e-3, 8, 300, 64, seed=9)])
def test_skull_workload_inputs(make):
    w = make()
    d = w.desc
    rho, lam, mu, alpha = w.medium
    assert np.all(rho > 0) and np.all(mu >= 0) and np.all(lam + 2 * mu > 0) and np.all(3 * lam + 2 * mu > 0)
    cmax = float(np.sqrt((lam + 2 * mu) / rho).max())
    assert cmax * d.dt / d.dx < 6 / (7 * math.sqrt(3))
    assert w.p0.max() > 0
    assert not np.any(w.p0[_band(d.shape, d.npml + 2)])        # 2 nodes clear of the layer
    assert not np.any(w.p0[mu > 0])                             # support in the fluid (inside the skull)
    lim = np.array([d.nx - 2, d.ny - 2, d.nz - 2])
    assert np.all(w.rec >= 0) and np.all(w.rec <= lim)


def test_halfspace_workload_inputs():
    c = synth.halfspace(ny=96)
    d = c.desc
    ny = d.ny
    p0 = np.zeros(d.shape, np.float32)
    j0, j1 = c.p0_y
    p0[:, j0:j1, :] = c.p0[:, None, :]
    assert not np.any(p0[_band(d.shape, d.npml + 2)])
    mu3 = np.broadcast_to(c.mu[:, None, :], d.shape)
    assert not np.any(p0[mu3 > 0])
    assert np.all(c.rec >= 0) and np.all(c.rec <= [d.nx - 2, ny - 2, d.nz - 2])


def test_bench_workload_p0_support():
    """skull-512, the bench workload: p0 zero within npml + 2 nodes of every face
    and at every solid node (about 20 s to generate)."""
    w = synth.skull_512()
    b = w.desc.npml + 2
    p = w.p0
    for sl in ((slice(0, b),), (slice(-b, None),), (slice(None), slice(0, b)), (slice(None), slice(-b, None)),
               (Ellipsis, slice(0, b)), (Ellipsis, slice(-b, None))):
        assert not np.any(p[sl])
    assert not np.any(p[w.mu > 0])
