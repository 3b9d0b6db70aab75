"""GPU: pact_forward / pact_adjoint replay CUDA graphs of whole steps.

The graphs' receiver kernels read the step count, the trace buffers and the
receiver table from device memory, so one captured graph serves every solve
of its handle.  Checked: the graph path gives bitwise the traces and images
of direct launches (PACT_GRAPHS=0) over consecutive solves on one handle
with different step counts (graph chunks of 16 plus single-step remainders),
receiver sets of different sizes and a changed medium (which drops the
graphs), forward and adjoint, on a medium-adaptive grid; and the launch
count that pact_profile_read reports is the same on both paths.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_02733_b300 import pact, synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1709_02733_b300 import build
    build.build()
    assert torch.cuda.is_available()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _solves(g, w, med2):
    out = []
    rec_a = w.rec
    rec_b = w.rec[: len(w.rec) // 3]
    for nsteps, rec in ((37, rec_a), (16, rec_b), (1, rec_a), (53, rec_b)):
        tr = g.forward(cuda(w.p0), rec, nsteps)
        out.append(tr.cpu().numpy())
        y = torch.flip(tr, [0]).contiguous()
        out.append(g.adjoint(y, rec).cpu().numpy())
    g.set_medium(*[cuda(m) for m in med2])
    tr = g.forward(cuda(w.p0), rec_a, 40)
    out.append(tr.cpu().numpy())
    out.append(g.adjoint(tr, rec_a).cpu().numpy())
    return out


def test_graph_path_equals_direct_launches(monkeypatch):
    w = synth.skull(96, 0.4e-3, 10, 300, 96, seed=3)
    med2 = (w.medium[0], w.medium[1] * np.float32(0.97), w.medium[2], w.medium[3])
    runs = []
    launches = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("PACT_GRAPHS", graphs)
        g = pact.Grid(w.desc)
        g.set_medium(*[cuda(m) for m in w.medium])
        assert g.role_points("fwd_ac_vel")[0] > 0  # medium-adaptive
        runs.append(_solves(g, w, med2))
        g.close()
        g = pact.Grid(w.desc)
        g.set_medium(*[cuda(m) for m in w.medium])
        g.forward(cuda(w.p0), w.rec, 5)
        g.profile(True)
        g.profile(False)  # counts only: no per-launch events, graphs stay on
        g.forward(cuda(w.p0), w.rec, 40)
        launches.append(g.profile_read()["all"][0])
        g.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    assert launches[0] == launches[1] > 0
