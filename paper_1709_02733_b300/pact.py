"""Thin ctypes binding of libpact.so (include/pact.h).

Argument marshalling only: every step of H and H^T runs in the library's CUDA
kernels.  PyTorch supplies device memory (``tensor.data_ptr()``) and streams.
There is no CPU fallback: if the library is missing or fails to load, every
call raises.

Function names follow the C ABI (``pact_create_grid`` ... ``pact_destroy``);
``Grid`` wraps one handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from .synth import GridDesc

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "libpact.so")

PACT_OK, PACT_EINVAL, PACT_ECFL, PACT_ENOMEM, PACT_ECUDA, PACT_ETIMEOUT, PACT_ESTATE = range(7)
_NAMES = {1: "EINVAL", 2: "ECFL", 3: "ENOMEM", 4: "ECUDA", 5: "ETIMEOUT", 6: "ESTATE"}

# every symbol include/pact.h declares
EXPORTS = ["pact_create_grid", "pact_set_medium", "pact_forward", "pact_adjoint", "pact_forward_host",
           "pact_adjoint_host", "pact_destroy", "pact_last_error", "pact_query_bytes", "pact_get_wavefield",
           "pact_profile", "pact_profile_read", "pact_role_points", "pact_forward_noalloc", "pact_begin",
           "pact_advance", "pact_poll", "pact_tv_prox_nn", "pact_resample_traces", "pact_check_bounded_wait",
           "pact_support_warning", "pact_create_slab", "pact_step_half", "pact_step_receivers", "pact_field_ptr", "pact_item_points"]

# kernel roles of pact_profile_read (include/pact.h PACT_K_*)
KINDS = ["fwd_velocity", "fwd_stress", "adj_a", "adj_b", "sample", "inject", "source", "readout", "fwd_fused",
         "adj_fused", "fwd_ac_vel", "fwd_ac_str", "adj_ac_a", "adj_ac_b"]


class PactError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pact {_NAMES.get(code, code)}: {msg}")
        self.code = code


class pact_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("npml", ctypes.c_int),
                ("pml_R0", ctypes.c_double), ("pml_f0", ctypes.c_double), ("pml_vmax", ctypes.c_double)]

    @classmethod
    def from_desc(cls, d: GridDesc):
        return cls(int(d.nx), int(d.ny), int(d.nz), float(d.dx), float(d.dt), int(d.npml), float(d.pml_R0),
                   float(d.pml_f0), float(d.pml_vmax))


_lib = None


def load(path: str = SO_PATH):
    """Load libpact.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpact.so not built at {path}: run `python -m paper_1709_02733_b300.build`")
    try:  # share the CUDA runtime torch already loaded
        import torch  # noqa: F401
    except ImportError:
        pass
    lib = ctypes.CDLL(path)
    vp, i, fp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
    D = ctypes.POINTER(pact_grid_desc)
    lib.pact_create_grid.argtypes = [D, vp, ctypes.POINTER(vp)]
    lib.pact_set_medium.argtypes = [vp, fp, fp, fp, fp]
    for name in ("pact_forward", "pact_adjoint", "pact_forward_host", "pact_adjoint_host"):
        getattr(lib, name).argtypes = [vp, fp, fp, i, i, fp]
    lib.pact_destroy.argtypes = [vp]
    lib.pact_last_error.argtypes = [vp]
    lib.pact_last_error.restype = ctypes.c_char_p
    lib.pact_query_bytes.argtypes = [D, i, i, ctypes.POINTER(ctypes.c_size_t)]
    lib.pact_get_wavefield.argtypes = [vp, fp]
    lib.pact_begin.argtypes = [vp, i, fp, fp, i, i, fp]
    lib.pact_advance.argtypes = [ctypes.POINTER(vp), i, i, vp]
    lib.pact_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.pact_support_warning.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.pact_forward_noalloc.argtypes = [D, fp, fp, fp, fp, fp, fp, i, i, fp, vp]
    lib.pact_profile.argtypes = [vp, i]
    lib.pact_profile_read.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]
    lib.pact_role_points.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.pact_tv_prox_nn.argtypes = [fp, fp, i, i, i, ctypes.c_float, i, fp, vp]
    lib.pact_resample_traces.argtypes = [fp, i, fp, i, i, ctypes.c_double, ctypes.c_double, vp]
    lib.pact_check_bounded_wait.argtypes = [ctypes.c_uint, vp]
    lib.pact_create_slab.argtypes = [D, i, i, vp, ctypes.POINTER(vp)]
    lib.pact_step_half.argtypes = [vp, i]
    lib.pact_step_receivers.argtypes = [vp]
    lib.pact_field_ptr.argtypes = [vp, i, ctypes.POINTER(ctypes.c_void_p)]
    lib.pact_item_points.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong)]
    for name in EXPORTS:
        if name != "pact_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc, handle=None):
    if rc != PACT_OK:
        msg = load().pact_last_error(handle).decode(errors="replace")
        raise PactError(rc, msg)


def pact_query_bytes(desc: GridDesc, L: int = 0, nsteps: int = -1) -> int:
    out = ctypes.c_size_t(0)
    _check(load().pact_query_bytes(ctypes.byref(pact_grid_desc.from_desc(desc)), int(L), int(nsteps),
                                   ctypes.byref(out)))
    return int(out.value)


def pact_tv_prox_nn(b, tau: float, iters: int, out=None, work=None, stream=None):
    """x = argmin_{x >= 0} 1/2 ||x - b||^2 + tau TV(x) for a float32 CUDA tensor b
    of shape (nz, ny, nx) (pact_tv_prox_nn; work: 6N floats, allocated if None)."""
    import torch
    if b.dim() != 3:
        raise ValueError("b must be (nz, ny, nx)")
    nz, ny, nx = b.shape
    N = b.numel()
    out = torch.empty_like(b) if out is None else out
    work = torch.empty(6 * N, device=b.device, dtype=torch.float32) if work is None else work
    st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    _check(load().pact_tv_prox_nn(_dev_ptr(b, N), _dev_ptr(out, N), int(nx), int(ny), int(nz), float(tau),
                                  int(iters), _dev_ptr(work, 6 * N), ctypes.c_void_p(st)))
    return out


tv_prox_nn = pact_tv_prox_nn


def pact_resample_traces(traces, m_out: int, s0: float, ratio: float, out=None, stream=None):
    """out[k] = traces(s0 + k * ratio) (linear in time, zero outside) for an
    (m_in, L) float32 CUDA tensor; returns an (m_out, L) tensor."""
    import torch
    m_in, L = traces.shape
    out = torch.empty((m_out, L), device=traces.device, dtype=torch.float32) if out is None else out
    st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    _check(load().pact_resample_traces(_dev_ptr(traces, m_in * L), int(m_in), _dev_ptr(out, m_out * L), int(m_out),
                                       int(L), float(s0), float(ratio), ctypes.c_void_p(st)))
    return out


resample_traces = pact_resample_traces


def pact_advance(grids, ksteps: int, stream=None):
    """Advance the solves prepared on ``grids`` together by up to ksteps steps."""
    import torch
    lib = load()
    arr = (ctypes.c_void_p * max(1, len(grids)))(*[g._h.value for g in grids])
    st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    _check(lib.pact_advance(arr, len(grids), int(ksteps), ctypes.c_void_p(st)))


def pact_forward_noalloc(desc: GridDesc, medium, p0, rec, nsteps: int, out=None, stream=None):
    """traces = H p0 through pact_forward_noalloc: no device memory is
    allocated by the library (its working memory is a fixed 64 MiB array that
    all calls share; calls must not overlap on the GPU).  ``out`` must be
    supplied by callers that cannot allocate."""
    import torch
    lib = load()
    r, L = _rec_host(rec)
    N = desc.N
    if out is None:
        out = torch.empty((nsteps + 1, L), device=p0.device, dtype=torch.float32)
    st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    _check(lib.pact_forward_noalloc(ctypes.byref(pact_grid_desc.from_desc(desc)),
                                    *[_dev_ptr(m, N) for m in medium], _dev_ptr(p0, N),
                                    r.ctypes.data_as(ctypes.c_void_p), L, int(nsteps),
                                    _dev_ptr(out, (nsteps + 1) * L), ctypes.c_void_p(st)))
    return out


def _dev_ptr(t, numel=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _rec_host(rec):
    r = np.ascontiguousarray(np.asarray(rec.cpu() if hasattr(rec, "cpu") else rec, dtype=np.float32).reshape(-1, 3))
    return r, r.shape[0]


class Grid:
    """One pact handle: grid, medium, wavefield and receiver tables on one GPU.

    ``stream``: a ``torch.cuda.Stream`` (default: torch's current stream at
    creation time); every call is ordered on it.
    """

    def __init__(self, desc: GridDesc, stream=None, slab=None):
        """slab=(z_lo, z_hi): a handle for planes [z_lo, z_hi) of the grid desc
        (pact_create_slab); the handle's own grid then has z_hi - z_lo planes."""
        import torch
        self.lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        if slab is None:
            self.desc = desc
            _check(self.lib.pact_create_grid(ctypes.byref(pact_grid_desc.from_desc(desc)),
                                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._h)))
        else:
            z_lo, z_hi = int(slab[0]), int(slab[1])
            _check(self.lib.pact_create_slab(ctypes.byref(pact_grid_desc.from_desc(desc)), z_lo, z_hi,
                                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._h)))
            from dataclasses import replace
            self.desc = replace(desc, nz=z_hi - z_lo)
        self.shape = self.desc.shape
        self.N = self.desc.N

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.pact_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls -------------------------------------------------------------
    def pact_set_medium(self, rho, lam, mu, alpha):
        _check(self.lib.pact_set_medium(self._h, *[_dev_ptr(a, self.N) for a in (rho, lam, mu, alpha)]), self._h)

    set_medium = pact_set_medium

    def pact_forward(self, p0, rec, nsteps: int, out=None):
        """traces = H p0, a (nsteps+1, L) float32 CUDA tensor."""
        import torch
        r, L = _rec_host(rec)
        if out is None:
            out = torch.empty((nsteps + 1, L), device=p0.device, dtype=torch.float32)
        _check(self.lib.pact_forward(self._h, _dev_ptr(p0, self.N), r.ctypes.data_as(ctypes.c_void_p), L,
                                     int(nsteps), _dev_ptr(out, (nsteps + 1) * L)), self._h)
        return out

    forward = pact_forward

    def pact_adjoint(self, traces, rec, out=None):
        """image = H^T traces, a (nz, ny, nx) float32 CUDA tensor."""
        import torch
        r, L = _rec_host(rec)
        nsteps = traces.shape[0] - 1
        if out is None:
            out = torch.empty(self.shape, device=traces.device, dtype=torch.float32)
        _check(self.lib.pact_adjoint(self._h, _dev_ptr(traces, (nsteps + 1) * L), r.ctypes.data_as(ctypes.c_void_p),
                                     L, int(nsteps), _dev_ptr(out, self.N)), self._h)
        return out

    adjoint = pact_adjoint

    def pact_forward_host(self, p0: np.ndarray, rec, nsteps: int, out: Optional[np.ndarray] = None):
        r, L = _rec_host(rec)
        p0 = np.ascontiguousarray(p0, dtype=np.float32)
        assert p0.size == self.N
        if out is None:
            out = np.empty((nsteps + 1, L), np.float32)
        _check(self.lib.pact_forward_host(self._h, p0.ctypes.data_as(ctypes.c_void_p),
                                          r.ctypes.data_as(ctypes.c_void_p), L, int(nsteps),
                                          out.ctypes.data_as(ctypes.c_void_p)), self._h)
        return out

    forward_host = pact_forward_host

    def pact_adjoint_host(self, traces: np.ndarray, rec, out: Optional[np.ndarray] = None):
        r, L = _rec_host(rec)
        tr = np.ascontiguousarray(traces, dtype=np.float32)
        nsteps = tr.shape[0] - 1
        if out is None:
            out = np.empty(self.shape, np.float32)
        _check(self.lib.pact_adjoint_host(self._h, tr.ctypes.data_as(ctypes.c_void_p),
                                          r.ctypes.data_as(ctypes.c_void_p), L, int(nsteps),
                                          out.ctypes.data_as(ctypes.c_void_p)), self._h)
        return out

    adjoint_host = pact_adjoint_host

    def pact_get_wavefield(self) -> np.ndarray:
        out = np.empty((9,) + self.shape, np.float32)
        _check(self.lib.pact_get_wavefield(self._h, out.ctypes.data_as(ctypes.c_void_p)), self._h)
        return out

    get_wavefield = pact_get_wavefield

    def pact_begin(self, is_adjoint: bool, inp, rec, nsteps: int, out):
        """Prepare a solve for pact_advance (buffers must stay alive until done)."""
        r, L = _rec_host(rec)
        n_in = (nsteps + 1) * L if is_adjoint else self.N
        n_out = self.N if is_adjoint else (nsteps + 1) * L
        _check(self.lib.pact_begin(self._h, int(bool(is_adjoint)), _dev_ptr(inp, n_in),
                                   r.ctypes.data_as(ctypes.c_void_p), L, int(nsteps), _dev_ptr(out, n_out)), self._h)

    begin = pact_begin

    def pact_support_warning(self) -> int:
        """Nonzero p0 entries within npml + 2 nodes of a face in the last forward
        solve (0 = the paper's support rule holds); waits for the stream."""
        n = ctypes.c_longlong(0)
        _check(self.lib.pact_support_warning(self._h, ctypes.byref(n)), self._h)
        return int(n.value)

    support_warning = pact_support_warning

    def pact_step_half(self, stress: bool):
        _check(self.lib.pact_step_half(self._h, int(bool(stress))), self._h)

    step_half = pact_step_half

    def pact_step_receivers(self):
        _check(self.lib.pact_step_receivers(self._h), self._h)

    step_receivers = pact_step_receivers

    def pact_field_ptr(self, field: int) -> int:
        """Device address of wavefield array `field` (0..8)."""
        ptr = ctypes.c_void_p()
        _check(self.lib.pact_field_ptr(self._h, int(field), ctypes.byref(ptr)), self._h)
        return int(ptr.value)

    field_ptr = pact_field_ptr

    def field_view(self, field: int):
        """Wavefield array `field` (0..8) as a (nz, ny, nx) float32 CUDA tensor
        sharing the handle's memory (valid while the handle lives)."""
        import torch

        class _Dev:
            pass

        d = _Dev()
        d.__cuda_array_interface__ = {"shape": self.shape, "typestr": "<f4", "strides": None,
                                      "data": (self.pact_field_ptr(field), False), "version": 3}
        return torch.as_tensor(d, device="cuda")

    def pact_poll(self) -> int:
        n = ctypes.c_int(0)
        _check(self.lib.pact_poll(self._h, ctypes.byref(n)), self._h)
        return int(n.value)

    poll = pact_poll

    def pact_profile(self, enable: bool = True):
        _check(self.lib.pact_profile(self._h, int(bool(enable))), self._h)

    profile = pact_profile

    def pact_profile_read(self):
        """{kind: (invocations, device_ms)} since the last pact_profile call,
        plus "all": (kernel launches of every role, device_ms)."""
        out = {}
        for k, name in enumerate(KINDS + ["all"]):
            n, ms = ctypes.c_longlong(0), ctypes.c_double(0.0)
            _check(self.lib.pact_profile_read(self._h, k, ctypes.byref(n), ctypes.byref(ms)), self._h)
            out[name] = (int(n.value), float(ms.value))
        return out

    profile_read = pact_profile_read

    def pact_role_points(self, kind: str):
        """(grid points, C-PML slab points) one invocation of a step role updates."""
        n, ns = ctypes.c_longlong(0), ctypes.c_longlong(0)
        _check(self.lib.pact_role_points(self._h, KINDS.index(kind), ctypes.byref(n), ctypes.byref(ns)), self._h)
        return int(n.value), int(ns.value)

    role_points = pact_role_points

    def pact_item_points(self, item_class: int) -> int:
        """Grid points of a work-item class: 1 (PACT_ITEM_DEEP: the stress update
        writes sigma^11 alone) or 2 (PACT_ITEM_NOALPHA: the velocity update
        loads no alpha)."""
        n = ctypes.c_longlong(0)
        _check(self.lib.pact_item_points(self._h, int(item_class), ctypes.byref(n)), self._h)
        return int(n.value)

    item_points = pact_item_points

    def deep_points(self) -> int:
        return self.pact_item_points(1)

    def noalpha_points(self) -> int:
        return self.pact_item_points(2)
