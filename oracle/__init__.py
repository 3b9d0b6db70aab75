"""FP64 CPU oracle for H and H^T -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the cpu_baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library and its binding) never imports it, and it never imports the product.

The arithmetic lives in ``pact_oracle.c`` (plain loops, double precision); this
module compiles it with gcc, loads it with ctypes and wraps it for numpy.
Arrays are C-order ``[z][y][x]`` (x fastest), the lexicographic order of the
paper's field vectors (Sec. 2.2).

Parity status (which tests pin each function) is listed at the top of
``tests/test_oracle_pins.py``; every public function here has at least one pin
that does not re-use the oracle's own formulas.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pact_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``pact_oracle.c`` into ``liboracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class _Desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("npml", ctypes.c_int),
        ("pml_R0", ctypes.c_double), ("pml_f0", ctypes.c_double), ("pml_vmax", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            i = ctypes.c_int
            d = ctypes.c_double
            lib.or_create.restype = vp
            lib.or_create.argtypes = [ctypes.POINTER(_Desc), _D, _D, _D, _D]
            lib.or_free.argtypes = [vp]
            lib.or_get_stagger.argtypes = [vp, _D, _D, _D]
            lib.or_pml_profile.argtypes = [i, i, d, d, d, d, d, i, _D, _D, _D, _D, _D]
            lib.or_substep.argtypes = [vp, i, i, _D]
            lib.or_step.argtypes = [vp, _D]
            lib.or_step_T.argtypes = [vp, _D]
            lib.or_inject.argtypes = [vp, _D, _D]
            lib.or_readout.argtypes = [vp, _D, _D]
            lib.or_sample.argtypes = [vp, _D, i, _D, _D]
            lib.or_sample_T.argtypes = [vp, _D, i, _D, _D]
            lib.or_forward.argtypes = [vp, _D, _D, i, i, _D]
            lib.or_adjoint.argtypes = [vp, _D, _D, i, i, _D]
            lib.or_run_state.argtypes = [vp, _D, i, _D]
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def pml_profile(n, npml, dx, dt, vmax, R0=1e-4, f0=1e6, half=False):
    """C-PML 1-D profile (Appendix A.1, kappa = 1): returns d, beta, a, b, chi."""
    lib = _load()
    out = [np.zeros(n) for _ in range(5)]
    lib.or_pml_profile(n, npml, dx, dt, vmax, R0, f0, int(bool(half)), *[_p(o) for o in out])
    return tuple(out)


class Oracle:
    """One grid + medium.  ``desc`` is a mapping with nx, ny, nz, dx, dt, npml,
    pml_R0, pml_f0, pml_vmax (SI units).  Medium arrays are ``(nz, ny, nx)``:
    density rho [kg/m^3], Lame lambda and mu [Pa], absorption alpha [1/s]."""

    def __init__(self, desc, rho, lam, mu, alpha):
        self.lib = _load()
        self.shape = (int(desc["nz"]), int(desc["ny"]), int(desc["nx"]))
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.desc = _Desc(int(desc["nx"]), int(desc["ny"]), int(desc["nz"]), float(desc["dx"]),
                          float(desc["dt"]), int(desc["npml"]), float(desc.get("pml_R0", 1e-4)),
                          float(desc.get("pml_f0", 1e6)), float(desc.get("pml_vmax", 0.0)))
        arrs = [_f64(a).reshape(self.shape) for a in (rho, lam, mu, alpha)]
        self._ctx = self.lib.or_create(ctypes.byref(self.desc), *[_p(a) for a in arrs])

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx:
            self.lib.or_free(ctx)
            self._ctx = None

    # ---- state helpers -------------------------------------------------
    def new_state(self) -> np.ndarray:
        """Zero state v' = [phi(9), u(3), psi(9), sigma(6)] as (27, nz, ny, nx)."""
        return np.zeros((27,) + self.shape)

    @staticmethod
    def views(st):
        """Named views of a state: phi (3,3,...), u (3,...), psi (3,3,...), sigma (6,...)."""
        return {
            "phi": st[0:9].reshape((3, 3) + st.shape[1:]),
            "u": st[9:12],
            "psi": st[12:21].reshape((3, 3) + st.shape[1:]),
            "sigma": st[21:27],
        }

    def stagger(self):
        """(rho_u, alpha_u, mu_s) each (3, nz, ny, nx); mu_s order 23, 13, 12."""
        out = [np.zeros((3,) + self.shape) for _ in range(3)]
        self.lib.or_get_stagger(self._ctx, *[_p(o) for o in out])
        return tuple(out)

    def substep(self, k: int, st: np.ndarray, transpose: bool = False) -> None:
        assert st.dtype == np.float64 and st.flags.c_contiguous and st.size == 27 * self.N
        self.lib.or_substep(self._ctx, int(k), int(bool(transpose)), _p(st))

    def step(self, st: np.ndarray) -> None:
        assert st.dtype == np.float64 and st.flags.c_contiguous and st.size == 27 * self.N
        self.lib.or_step(self._ctx, _p(st))

    def step_T(self, st: np.ndarray) -> None:
        assert st.dtype == np.float64 and st.flags.c_contiguous and st.size == 27 * self.N
        self.lib.or_step_T(self._ctx, _p(st))

    def inject(self, p0) -> np.ndarray:
        st = self.new_state()
        self.lib.or_inject(self._ctx, _p(_f64(p0).reshape(self.shape)), _p(st))
        return st

    def readout(self, st) -> np.ndarray:
        img = np.zeros(self.shape)
        self.lib.or_readout(self._ctx, _p(st), _p(img))
        return img

    def sample(self, rec, st) -> np.ndarray:
        rec = _f64(rec).reshape(-1, 3)
        out = np.zeros(rec.shape[0])
        self.lib.or_sample(self._ctx, _p(rec), rec.shape[0], _p(st), _p(out))
        return out

    def sample_T(self, rec, ph, st) -> None:
        rec = _f64(rec).reshape(-1, 3)
        ph = _f64(ph).reshape(-1)
        self.lib.or_sample_T(self._ctx, _p(rec), rec.shape[0], _p(ph), _p(st))

    # ---- the operators -------------------------------------------------
    def forward(self, p0, rec, nsteps: int) -> np.ndarray:
        """p_hat = H p0, shape (nsteps + 1, L)."""
        rec = _f64(rec).reshape(-1, 3)
        L = rec.shape[0]
        out = np.zeros((nsteps + 1, L))
        self.lib.or_forward(self._ctx, _p(_f64(p0).reshape(self.shape)), _p(rec), L, int(nsteps), _p(out))
        return out

    def adjoint(self, traces, rec) -> np.ndarray:
        """p_adj = H^T p_hat for traces of shape (nsteps + 1, L)."""
        rec = _f64(rec).reshape(-1, 3)
        tr = _f64(traces)
        L = rec.shape[0]
        assert tr.ndim == 2 and tr.shape[1] == L
        img = np.zeros(self.shape)
        self.lib.or_adjoint(self._ctx, _p(tr), _p(rec), L, tr.shape[0] - 1, _p(img))
        return img

    def run_state(self, p0, nsteps: int) -> np.ndarray:
        st = self.new_state()
        self.lib.or_run_state(self._ctx, _p(_f64(p0).reshape(self.shape)), int(nsteps), _p(st))
        return st
