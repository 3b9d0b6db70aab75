"""pact_forward_noalloc: the forward operator for callers that cannot allocate
device memory.

Some hosts own every byte of device memory through their own pool and forbid
outside cudaMalloc / cudaFree (such an allocation escapes the pool's accounting
or fails once the pool has reserved the device).  The no-allocation entry point
serves them from a fixed 64 MiB array inside the library, committed on a device
by the first call there; later calls commit no device memory.  These tests call it
through the C ABI and check its traces against the regular entry point
pact_forward, within the parity tolerance used everywhere else (relative L2
<= 1e-4), on two calls in a row with different inputs (the second call must not
see anything the first one left in the shared array).  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_02733_b300 import pact, synth  # noqa: E402
from paper_1709_02733_b300.synth import GridDesc  # noqa: E402

TOL = 1e-4


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def noalloc_call(lib, desc, medium, p0, rec, nsteps, out):
    """Direct C-ABI call; every buffer is the caller's."""
    r = np.ascontiguousarray(rec, np.float32)
    rc = lib.pact_forward_noalloc(ctypes.byref(pact.pact_grid_desc.from_desc(desc)),
                                  *[ctypes.c_void_p(m.data_ptr()) for m in medium], ctypes.c_void_p(p0.data_ptr()),
                                  r.ctypes.data_as(ctypes.c_void_p), r.shape[0], nsteps,
                                  ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


@pytest.fixture(scope="module")
def lib():
    from paper_1709_02733_b300 import build
    build.build()
    assert torch.cuda.is_available()
    return pact.load()


@pytest.mark.parametrize("case", ["random", "skull"])
def test_noalloc_matches_forward_on_two_calls(lib, case):
    if case == "random":
        shape = (24, 26, 28)
        rho, lam, mu, al, vmax = synth.random_medium(shape, 71)
        dx = 1e-3
        desc = GridDesc(shape[2], shape[1], shape[0], dx, 0.3 * dx / vmax, npml=3, pml_vmax=vmax)
        rng = np.random.default_rng(72)
        p0s = [rng.standard_normal(shape).astype(np.float32) for _ in range(2)]
        rec = synth.random_receivers(16, shape, 73)
        nsteps = 40
        medium = (rho, lam, mu, al)
    else:
        w = synth.skull(48, 1.2e-3, 6, 80, 64, seed=5)
        desc, medium, rec, nsteps = w.desc, w.medium, w.rec, w.nsteps
        p0s = [w.p0, np.roll(w.p0, 3, axis=2)]
    med = [cuda(m) for m in medium]
    g = pact.Grid(desc)
    g.set_medium(*med)
    L = rec.shape[0]
    for p0 in p0s:
        dp0 = cuda(p0)
        ref = g.forward(dp0, rec, nsteps).cpu().numpy()
        out = torch.full((nsteps + 1, L), float("nan"), device="cuda")
        assert noalloc_call(lib, desc, med, dp0, rec, nsteps, out) == pact.PACT_OK, lib.pact_last_error(None)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) <= TOL
    g.close()


def test_noalloc_rejects_grid_beyond_the_fixed_array(lib):
    desc = GridDesc(256, 256, 256, 1e-3, 1e-7, npml=4, pml_vmax=1500.0)
    dummy = torch.zeros(16, device="cuda")
    out = torch.zeros(16, device="cuda")
    rec = np.array([[10.0, 10.0, 10.0]], np.float32)
    rc = noalloc_call(lib, desc, [dummy] * 4, dummy, rec, 1, out)
    assert rc == pact.PACT_EINVAL
    msg = lib.pact_last_error(None).decode()
    assert "scratch" in msg and "bytes" in msg


def test_noalloc_later_calls_commit_no_device_memory(lib):
    """Once the first call on the device has loaded the array, a further call
    changes the device's free memory by nothing (cudaMemGetInfo)."""
    shape = (20, 24, 28)
    rho, lam, mu, al, vmax = synth.random_medium(shape, 81)
    desc = GridDesc(shape[2], shape[1], shape[0], 1e-3, 0.3e-3 / vmax, npml=2, pml_vmax=vmax)
    med = [cuda(m) for m in (rho, lam, mu, al)]
    p0 = cuda(np.random.default_rng(82).standard_normal(shape))
    rec = synth.random_receivers(8, shape, 83)
    outs = [torch.empty((31, 8), device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    assert noalloc_call(lib, desc, med, p0, rec, 30, outs[0]) == pact.PACT_OK, lib.pact_last_error(None)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert noalloc_call(lib, desc, med, p0, rec, 30, outs[1]) == pact.PACT_OK, lib.pact_last_error(None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(outs[0], outs[1])
