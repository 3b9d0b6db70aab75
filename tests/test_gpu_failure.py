"""Failure detection without a GPU fault: the bounded mbarrier wait of the
TMA-staged kernels, run on a barrier that nothing ever completes, gives up
after its limit; the host sees PACT_ETIMEOUT; the context stays usable (a
solve right after it still matches the oracle)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from paper_1709_02733_b300 import pact, synth  # noqa: E402
from paper_1709_02733_b300.synth import GridDesc  # noqa: E402


def test_bounded_wait_times_out_and_context_survives():
    from paper_1709_02733_b300 import build
    build.build()
    lib = pact.load()
    st = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    rc = lib.pact_check_bounded_wait(50000, st)       # 50 ms
    dt = time.perf_counter() - t0
    assert rc == pact.PACT_ETIMEOUT
    assert dt >= 0.045
    assert lib.pact_check_bounded_wait(0, st) == pact.PACT_EINVAL
    # the context is still usable
    rho, lam, mu, al, vmax = synth.random_medium((16, 16, 20), 5)
    d = GridDesc(20, 16, 16, 1e-3, 0.3e-3 / vmax, npml=2, pml_vmax=vmax)
    g = pact.Grid(d)
    g.set_medium(*[torch.from_numpy(m).cuda() for m in (rho, lam, mu, al)])
    p0 = np.random.default_rng(0).standard_normal((16, 16, 20)).astype(np.float32)
    rec = synth.random_receivers(5, (16, 16, 20), 1)
    tr = g.forward(torch.from_numpy(p0).cuda(), rec, 10).cpu().numpy()
    ref = Oracle(d.as_dict(), rho, lam, mu, al).forward(p0, rec, 10)
    assert np.linalg.norm(tr - ref) / np.linalg.norm(ref) <= 1e-4
