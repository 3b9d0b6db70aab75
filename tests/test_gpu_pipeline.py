"""Non-inverse-crime pipeline (paper_1709_02733_b300.pipeline): the trace
resampler against numpy's linear interpolation, and a small study whose
fine-grid data must differ from the coarse operator's own data by more than
the noise (the model mismatch) while describing the same object."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_02733_b300 import pact  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1709_02733_b300 import build
    build.build()


@pytest.mark.parametrize("m_in,m_out,s0,ratio", [(50, 40, 0.3, 1.2), (33, 60, -2.5, 0.6), (10, 5, 0.0, 2.25)])
def test_resample_matches_numpy(m_in, m_out, s0, ratio):
    rng = np.random.default_rng(m_in)
    tr = rng.standard_normal((m_in, 7)).astype(np.float32)
    got = pact.resample_traces(torch.from_numpy(tr).cuda(), m_out, s0, ratio).cpu().numpy()
    s = s0 + ratio * np.arange(m_out)
    ref = np.stack([np.interp(s, np.arange(m_in), tr[:, l].astype(np.float64), left=0.0, right=0.0)
                    for l in range(7)], axis=1)
    inside = (s >= 0) & (s <= m_in - 1)
    ref[~inside] = 0.0
    assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(tr).max())


def test_non_inverse_crime_study_small():
    from paper_1709_02733_b300.pipeline import make_study
    st = make_study(n_coarse=48, dx=1.6e-3, npml=3, nsteps=150, L=64, seed=2)
    c = st.coarse
    assert st.y.shape == st.y_crime.shape == (151, 64)
    assert st.fine.desc.nx == 64 and abs(st.fine.desc.dx - 1.2e-3) < 1e-12
    y, yc = st.y.double(), st.y_crime.double()
    corr = float((y * yc).sum() / (y.norm() * yc.norm()))
    diff = float((y - yc).norm() / yc.norm())
    noise = st.noise_sigma * (y.numel() ** 0.5) / float(yc.norm())
    assert corr > 0.5                       # the same object seen by both discretisations
    assert diff > 1.2 * noise               # more than the two noise draws: the model mismatch
    g = pact.Grid(c.desc)
    g.set_medium(*[torch.from_numpy(m).cuda() for m in c.medium])
    img = g.adjoint(st.y, c.rec)
    p = torch.from_numpy(c.p0).cuda()
    assert float(torch.dot(img.flatten().double(), p.flatten().double())) > 0
