"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad grid descriptions without touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_1709_02733_b300 import build as pbuild
from paper_1709_02733_b300 import pact
from paper_1709_02733_b300.synth import GridDesc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pact.load()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pact_[a-z_0-9]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert "pact_forward" in declared and "pact_adjoint" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(pact.EXPORTS) | declared  # binding knows the ABI
    assert set(pact.EXPORTS) <= declared


def test_query_bytes(lib):
    d = GridDesc(64, 64, 64, 0.5e-3, 1e-7, npml=3)
    b = pact.pact_query_bytes(d, L=128, nsteps=400)
    N = 64 ** 3
    assert b >= 13 * N * 4
    b0 = pact.pact_query_bytes(GridDesc(64, 64, 64, 0.5e-3, 1e-7, npml=0), L=128, nsteps=400)
    assert b > b0  # the layer slabs


@pytest.mark.parametrize("bad", [
    dict(nx=3), dict(npml=-1), dict(dx=0.0), dict(dt=-1.0), dict(nx=8, npml=4), dict(pml_R0=0.0),
])
def test_bad_desc_rejected(lib, bad):
    kw = dict(nx=16, ny=16, nz=16, dx=1e-3, dt=1e-7, npml=2)
    kw.update(bad)
    d = GridDesc(**kw)
    with pytest.raises(pact.PactError) as e:
        pact.pact_query_bytes(d, 4, 10)
    assert e.value.code == pact.PACT_EINVAL
    h = ctypes.c_void_p()
    rc = lib.pact_create_grid(ctypes.byref(pact.pact_grid_desc.from_desc(d)), None, ctypes.byref(h))
    assert rc == pact.PACT_EINVAL and not h.value
    assert lib.pact_last_error(None)
