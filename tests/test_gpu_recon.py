"""FISTA reconstruction with the matched pair (paper_1709_02733_b300.recon)
against the FP64 oracle's FISTA (oracle/fista.py) run with the oracle's own H
and H^T: same data, start and step size; every iterate within 1e-4 relative
L2 (the clamp can only differ where a value is within FP32 rounding of zero).
Plus behaviour: FISTA reduces the data misfit faster than projected gradient
descent with the same step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from oracle.fista import fista_nn as oracle_fista  # noqa: E402
from paper_1709_02733_b300 import pact, synth  # noqa: E402
from paper_1709_02733_b300.autograd import operator_norm_sq, reconstruct_gd  # noqa: E402
from paper_1709_02733_b300.recon import fista_nn  # noqa: E402


@pytest.fixture(scope="module")
def case():
    from paper_1709_02733_b300 import build
    build.build()
    w = synth.skull(32, 1.8e-3, 4, 50, 48, seed=14)
    g = pact.Grid(w.desc)
    g.set_medium(*[torch.from_numpy(m).cuda() for m in w.medium])
    p_true = torch.from_numpy(w.p0).cuda()
    y0 = g.forward(p_true, w.rec, w.nsteps)
    s = float(y0.pow(2).mean().sqrt()) * 10 ** (-1.5)
    y = y0 + s * torch.randn(y0.shape, generator=torch.Generator().manual_seed(6)).cuda()
    L = 1.05 * operator_norm_sq(g, w.rec, w.nsteps, iters=10)
    return w, g, p_true, y, L


def test_fista_iterates_match_oracle(case):
    w, g, p_true, y, L = case
    got = []
    fista_nn(g, w.rec, w.nsteps, y, L, iters=6, callback=lambda k, x, loss: got.append(x.cpu().numpy()))
    o = Oracle(w.desc.as_dict(), *w.medium)
    yn = y.cpu().numpy().astype(np.float64)
    ref = oracle_fista(lambda p: o.forward(p, w.rec, w.nsteps), lambda r: o.adjoint(r, w.rec), yn,
                       np.zeros(w.p0.shape), L, 6)
    for k, (a, b) in enumerate(zip(got, ref)):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-4, k


def test_fista_ahead_of_projected_gd(case):
    w, g, p_true, y, L = case
    lf, lg = [], []
    fista_nn(g, w.rec, w.nsteps, y, L, iters=12, callback=lambda k, x, loss: lf.append(loss))
    reconstruct_gd(g, w.rec, w.nsteps, y, iters=12, eta=1.0 / L, callback=lambda k, x, loss: lg.append(loss))
    assert lf[-1] < lg[-1]
    assert min(x for x in lf) < lf[0]


def test_tv_prox_kernel_matches_oracle():
    """pact_tv_prox_nn (CUDA) against the oracle's fast gradient projection
    (same iteration count) on a ragged 3-D array; tau = 0 is the projection."""
    from oracle.fista import tv_prox_nn as oracle_tv
    rng = np.random.default_rng(8)
    b = (np.cumsum(rng.standard_normal((13, 17, 21)), axis=2) * 0.3 + 0.2).astype(np.float32)
    got = pact.tv_prox_nn(torch.from_numpy(b).cuda(), 0.3, 60).cpu().numpy()
    ref = oracle_tv(b.astype(np.float64), 0.3, 60)
    assert (ref == 0).sum() > 0
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    assert np.array_equal(pact.tv_prox_nn(torch.from_numpy(b).cuda(), 0.0, 5).cpu().numpy(), np.maximum(b, 0))


def test_fista_tv_iterates_match_oracle(case):
    from oracle.fista import fista_tv_nn as oracle_fista_tv

    from paper_1709_02733_b300.recon import fista_tv
    w, g, p_true, y, L = case
    lam = 2e-3 * L
    got = []
    fista_tv(g, w.rec, w.nsteps, y, L, lam, iters=4, inner=30, callback=lambda k, x, loss: got.append(x.cpu().numpy()))
    o = Oracle(w.desc.as_dict(), *w.medium)
    yn = y.cpu().numpy().astype(np.float64)
    ref = oracle_fista_tv(lambda p: o.forward(p, w.rec, w.nsteps), lambda r: o.adjoint(r, w.rec), yn,
                          np.zeros(w.p0.shape), L, lam, 4, 30)
    for k, (a, b) in enumerate(zip(got, ref)):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-4, k
