"""Autograd wrapper: backward = H^T, checked against finite differences (the
loss 1/2 ||H p - y||^2 is quadratic, so central differences are exact up to
round-off) and against the oracle gradient H^T (H p - y) in FP64; plus a short
projected-gradient-descent reconstruction that must reduce loss and error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from paper_1709_02733_b300 import pact, synth  # noqa: E402
from paper_1709_02733_b300.autograd import operator_norm_sq, pact_forward_op, reconstruct_gd  # noqa: E402


@pytest.fixture(scope="module")
def case():
    from paper_1709_02733_b300 import build
    build.build()
    w = synth.skull(48, 1.2e-3, 6, 120, 64, seed=12)
    g = pact.Grid(w.desc)
    g.set_medium(*[torch.from_numpy(m).cuda() for m in w.medium])
    p_true = torch.from_numpy(w.p0).cuda()
    y0 = g.forward(p_true, w.rec, w.nsteps)
    s = float(y0.pow(2).mean().sqrt()) * 10 ** (-1.5)  # SNR 30 dB
    y = y0 + s * torch.randn(y0.shape, generator=torch.Generator().manual_seed(4)).cuda()
    return w, g, p_true, y


def _loss(g, w, p, y):
    r = g.forward(p.contiguous(), w.rec, w.nsteps).double() - y.double()
    return 0.5 * float((r ** 2).sum())


def test_gradient_finite_differences(case):
    """<grad L, d> equals (L(p + e d) - L(p - e d)) / (2e) on 16 random directions."""
    w, g, p_true, y = case
    p = (0.5 * p_true).clone().requires_grad_(True)
    r = pact_forward_op(p, g, w.rec, w.nsteps) - y
    loss = 0.5 * (r.double() ** 2).sum()
    loss.backward()
    grad = p.grad.detach()
    gen = torch.Generator().manual_seed(4)
    for k in range(16):
        d = torch.randn(p.shape, generator=gen).cuda()
        d *= float(p_true.norm()) / float(d.norm())
        eps = 1.0
        fd = (_loss(g, w, p.detach() + eps * d, y) - _loss(g, w, p.detach() - eps * d, y)) / (2 * eps)
        an = float(torch.dot(grad.flatten().double(), d.flatten().double()))
        assert abs(fd - an) <= 1e-4 * max(abs(fd), 1e-3 * float(loss.detach())), (k, fd, an)


def test_gradient_matches_oracle(case):
    w, g, p_true, y = case
    p = (0.3 * p_true).clone().requires_grad_(True)
    r = pact_forward_op(p, g, w.rec, w.nsteps) - y
    (0.5 * (r ** 2).sum()).backward()
    o = Oracle(w.desc.as_dict(), *w.medium)
    pn = p.detach().cpu().numpy().astype(np.float64)
    res = o.forward(pn, w.rec, w.nsteps) - y.cpu().numpy().astype(np.float64)
    ref = o.adjoint(res, w.rec)
    got = p.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4


def test_gd_reconstruction_decreases_loss_and_error(case):
    w, g, p_true, y = case
    lam = operator_norm_sq(g, w.rec, w.nsteps, iters=10)
    assert lam > 0
    losses, errs = [], []
    pn = float(p_true.norm())

    def cb(it, p, loss):
        losses.append(loss)
        errs.append(float((p - p_true).norm()) / pn)

    reconstruct_gd(g, w.rec, w.nsteps, y, iters=8, eta=1.0 / lam, callback=cb)
    assert all(b <= a * (1 + 1e-6) for a, b in zip(losses, losses[1:]))
    assert errs[-1] < errs[0] < 1.0
