"""The acoustic operator pair H_{mu=0}, H^T_{mu=0} (mu = 0 at every node, the
paper's ablation): every work item of the medium-adaptive plan is fluid, so the
interior runs the one-stress-field kernels of step_acoustic.cu and the C-PML
frame the fluid C-PML kernels of step_fluid.cu.  Checked against
the FP64 oracle (the elastic operator with mu = 0, 1e-4 relative L2), against
the elastic kernels on the same medium (PACT_ACOUSTIC=0; FP32 rounding), and
by the inner-product test (1e-5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from paper_1709_02733_b300 import pact, synth  # noqa: E402
from paper_1709_02733_b300.synth import GridDesc  # noqa: E402


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


def _fluid_case(shape, npml, seed, L=11):
    rho, lam, mu, al, vmax = synth.random_medium(shape, seed, fluid_fraction=1.0)
    assert not mu.any()
    nz, ny, nx = shape
    dx = 1e-3
    d = GridDesc(nx, ny, nz, dx, 0.3 * dx / vmax, npml=npml, pml_vmax=vmax)
    p0 = np.random.default_rng(seed + 1).standard_normal(shape).astype(np.float32)
    return d, (rho, lam, mu, al), p0, synth.random_receivers(L, shape, seed + 2)


@pytest.mark.parametrize("shape,npml,nsteps", [((40, 44, 104), 4, 41), ((36, 30, 96), 2, 30), ((52, 37, 100), 5, 36)])
def test_acoustic_matches_oracle_and_elastic_kernels(shape, npml, nsteps, monkeypatch):
    d, med, p0, rec = _fluid_case(shape, npml, 1100 + npml)
    g = make_grid(d, med)
    assert g.role_points("fwd_ac_vel")[0] > 0                       # the acoustic kernels run
    monkeypatch.setenv("PACT_ACOUSTIC", "0")
    g_e = make_grid(d, med)
    monkeypatch.delenv("PACT_ACOUSTIC")
    assert g_e.role_points("fwd_ac_vel")[0] == 0
    assert g.role_points("fwd_velocity")[0] + g.role_points("fwd_ac_vel")[0] == d.N
    o = Oracle(d.as_dict(), *med)
    tr = g.forward(cuda(p0), rec, nsteps).cpu().numpy()
    assert rel_l2(tr, o.forward(p0, rec, nsteps)) <= 1e-4
    wf = g.get_wavefield()
    assert rel_l2(tr, g_e.forward(cuda(p0), rec, nsteps).cpu().numpy()) <= 1e-6
    assert rel_l2(wf, g_e.get_wavefield()) <= 1e-6
    assert np.array_equal(wf[3], wf[4]) and np.array_equal(wf[3], wf[5]) and not wf[6:].any()
    y = np.random.default_rng(3).standard_normal(tr.shape).astype(np.float32)
    img = g.adjoint(cuda(y), rec).cpu().numpy()
    assert rel_l2(img, o.adjoint(y, rec)) <= 1e-4
    assert rel_l2(img, g_e.adjoint(cuda(y), rec).cpu().numpy()) <= 1e-6


def test_acoustic_inner_product_fluid_skull():
    """Skull geometry with the shear modulus removed (lambda + 2 mu kept)."""
    w = synth.skull(96, 0.4e-3, 10, 300, 128, seed=3)
    rho, lam, mu, al = w.medium
    med = (rho, (lam + 2.0 * mu).astype(np.float32), np.zeros_like(mu), al)
    g = make_grid(w.desc, med)
    assert g.role_points("adj_ac_a")[0] > 0
    tr = g.forward(cuda(w.p0), w.rec, w.nsteps).cpu().numpy().astype(np.float64)
    y = tr + 0.1 * np.sqrt(np.mean(tr ** 2)) * np.random.default_rng(1).standard_normal(tr.shape)
    img = g.adjoint(cuda(y), w.rec).cpu().numpy().astype(np.float64)
    lhs = float(np.sum(tr * y.astype(np.float32).astype(np.float64)))
    rhs = float(np.sum(w.p0.astype(np.float64) * img))
    assert abs(lhs - rhs) / abs(lhs) <= 1e-5


def test_acoustic_needs_a_layer():
    """Without a C-PML every tile is interior, ragged ones included; those stay
    with the elastic kernels (the acoustic ones assume whole tiles)."""
    d, med, p0, rec = _fluid_case((24, 20, 68), 0, 1200)
    g = make_grid(d, med)
    assert g.role_points("fwd_ac_vel")[0] == 0
    o = Oracle(d.as_dict(), *med)
    assert rel_l2(g.forward(cuda(p0), rec, 20).cpu().numpy(), o.forward(p0, rec, 20)) <= 1e-4
