"""Z-slab decomposition of H and H^T: one slab of the grid per GPU.

The paper's implementation section runs the solver on several GPUs by cutting
the grid into pieces held by different GPUs and exchanging the planes at the
cuts every time step.  Here the cuts are planes of constant z: slab r owns
planes [lo_r, hi_r) and holds HALO more planes on each side that borders
another slab (its halo), as a pact handle made by pact_create_slab.  The
staggered fourth-order differences of Eq. (it) reach two planes, so after each
half step the half just written is copied into the neighbours' halos:

    forward: begin (p0 is given on the halo planes too);
             per step: velocity half -> exchange u -> stress half
                       -> exchange sigma -> sample receivers
    adjoint: begin (inject the last row) -> exchange Q;
             per step: first half -> exchange w -> second half
                       -> inject receivers -> exchange Q

(after an adjoint begin the nine slots hold w and Q; its first half writes the
w slots from the Q slots, its second the Q slots from the w slots).  Halo
planes are computed wrongly by their own slab (their stencils leave the slab)
and are overwritten before any owned plane reads them.

Receivers: receiver l interpolates planes k0 and k0+1, k0 = min(floor(z_l),
nz-2) (Eq. (interpgrid)).  The forward samples it on the slab that owns k0,
after the sigma exchange, so that plane k0+1 is current there even when it is
a halo plane.  The adjoint injects it on every slab that owns k0 or k0+1 (one
slab, or the two beside a cut), each into both planes before the Q exchange:
every owned plane receives each contribution once, and what lands on a halo
plane is overwritten.  Local receiver z is z_l - zl_r, an exact float
difference, so the weights are those of the whole grid.

The C-PML z layer stays inside the first and last slab (cuts at least
npml + 4 planes from either face), so a middle slab has no z layer.

Exchanges: ``DistExchange`` (one slab per process, torch.distributed
point-to-point over NCCL or gloo) and ``LoopbackExchange`` (all slabs in one
process on one device: plain copies).  Both take a list of ``Slab`` objects
and the field slots to exchange.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

HALO = 2
U_FIELDS = (0, 1, 2)                    # u^1 u^2 u^3 (adjoint: w)
SIGMA_FIELDS = (3, 4, 5, 6, 7, 8)       # sigma^11 .. sigma^12 (adjoint: Q)
MIN_OWNED = 8


def receiver_planes(rec: np.ndarray, nz: int) -> np.ndarray:
    """k0 of every receiver: the lower of the two z planes it interpolates."""
    z = np.asarray(rec, np.float32).reshape(-1, 3)[:, 2]
    return np.minimum(np.floor(z).astype(np.int64), nz - 2)


def partition(nz: int, R: int, npml: int) -> List[Tuple[int, int]]:
    """Owned z ranges [lo, hi) of R slabs: near-equal plane counts, every cut
    at least npml + 4 planes from both faces and every slab MIN_OWNED planes."""
    if R < 1:
        raise ValueError("R >= 1")
    lo_lim, hi_lim = npml + 4, nz - npml - 4
    cuts = [round(nz * r / R) for r in range(1, R)]
    bounds = [0] + cuts + [nz]
    for r in range(1, R):
        if not lo_lim <= bounds[r] <= hi_lim:
            raise ValueError(f"cut {bounds[r]} of {R} slabs inside the z layer's reach (nz={nz}, npml={npml})")
    if min(bounds[r + 1] - bounds[r] for r in range(R)) < MIN_OWNED:
        raise ValueError(f"{R} slabs of {nz} planes leave fewer than {MIN_OWNED} planes to a slab")
    return [(bounds[r], bounds[r + 1]) for r in range(R)]


def local_range(parts: Sequence[Tuple[int, int]], r: int) -> Tuple[int, int]:
    """Planes [zl, zh) held by slab r: its own planes and HALO more on each
    side that borders another slab."""
    lo, hi = parts[r]
    zl = lo - HALO if r > 0 else lo
    zh = hi + HALO if r < len(parts) - 1 else hi
    return zl, zh


def owners(parts: Sequence[Tuple[int, int]], rec: np.ndarray, nz: int) -> np.ndarray:
    """Slab that samples each receiver in the forward: the owner of plane k0."""
    k0 = receiver_planes(rec, nz)
    own = np.full(k0.shape, -1, np.int64)
    for r, (lo, hi) in enumerate(parts):
        own[(k0 >= lo) & (k0 < hi)] = r
    return own


def injectors(parts: Sequence[Tuple[int, int]], rec: np.ndarray, nz: int, r: int) -> np.ndarray:
    """Receivers slab r injects in the adjoint: those with plane k0 or k0+1
    owned by r (ascending, as in the whole receiver array)."""
    k0 = receiver_planes(rec, nz)
    lo, hi = parts[r]
    return np.nonzero(((k0 >= lo) & (k0 < hi)) | ((k0 + 1 >= lo) & (k0 + 1 < hi)))[0]


@dataclass
class Slab:
    """Slab r of a partition: its pact handle, its planes and its receivers."""
    r: int
    parts: List[Tuple[int, int]]
    zl: int
    zh: int
    rec_idx: np.ndarray          # receivers sampled here (forward), ascending
    rec_local: np.ndarray        # (L_r, 3) float32, z relative to zl
    inj_idx: np.ndarray          # receivers injected here (adjoint), ascending
    inj_local: np.ndarray
    grid: object = None          # pact.Grid (slab handle)
    _views: dict = field(default_factory=dict, repr=False)

    @property
    def lo(self):
        return self.parts[self.r][0]

    @property
    def hi(self):
        return self.parts[self.r][1]

    @property
    def nzl(self):
        return self.zh - self.zl

    @property
    def owned(self):
        """Slice of the local planes this slab owns."""
        return slice(self.lo - self.zl, self.hi - self.zl)

    def field(self, f: int):
        """Field slot f of the handle as a (nzl, ny, nx) CUDA tensor (no copy)."""
        if f not in self._views:
            self._views[f] = self.grid.field_view(f)
        return self._views[f]


def layout(nz: int, parts, r: int, rec: np.ndarray) -> Slab:
    """Slab r's planes and receiver table (no handle yet)."""
    zl, zh = local_range(parts, r)
    rec = np.asarray(rec, np.float32).reshape(-1, 3)

    def local(idx):
        loc = rec[idx].copy()
        loc[:, 2] = loc[:, 2] - np.float32(zl)
        return loc

    idx = np.nonzero(owners(parts, rec, nz) == r)[0]
    inj = injectors(parts, rec, nz, r)
    return Slab(r, list(parts), zl, zh, idx, local(idx), inj, local(inj))


def make_slab(desc, parts, r, rec: np.ndarray, stream=None) -> Slab:
    """Slab r with its handle (pact_create_slab); the medium and p0 of the
    slab are the whole grid's planes [zl, zh)."""
    from . import pact
    s = layout(desc.nz, parts, r, rec)
    s.grid = pact.Grid(desc, stream=stream, slab=(s.zl, s.zh))
    return s


# -- exchanges ------------------------------------------------------------------

def _halo_pairs(s: Slab):
    """(send slice, recv slice, neighbour) for each neighbour of slab s: the
    HALO owned planes next to the cut go out, the HALO halo planes come in."""
    out = []
    R = len(s.parts)
    n = s.nzl
    if s.r > 0:
        out.append((slice(HALO, 2 * HALO), slice(0, HALO), s.r - 1))
    if s.r < R - 1:
        out.append((slice(n - 2 * HALO, n - HALO), slice(n - HALO, n), s.r + 1))
    return out


class LoopbackExchange:
    """All slabs in one process (one device): halo planes copied directly."""

    def __call__(self, slabs: List[Slab], fields: Sequence[int]):
        by_r = {s.r: s for s in slabs}
        for s in slabs:
            for _send, recv, nb in _halo_pairs(s):
                t = by_r[nb]
                # the neighbour's owned planes next to the cut
                src = slice(HALO, 2 * HALO) if nb > s.r else slice(t.nzl - 2 * HALO, t.nzl - HALO)
                for f in fields:
                    s.field(f)[recv].copy_(t.field(f)[src])


class DistExchange:
    """One slab per process: torch.distributed point-to-point (NCCL between
    GPUs, gloo on CPU), one batched round of isend/irecv per exchange.
    ``field_of(slab, f)`` returns the (nzl, ny, nx) tensor of slot f (default:
    the handle's device memory)."""

    def __init__(self, field_of=None, group=None):
        self.field_of = field_of or (lambda s, f: s.field(f))
        self.group = group

    def __call__(self, slabs: List[Slab], fields: Sequence[int]):
        import torch.distributed as dist
        ops = []
        for s in slabs:
            for send, recv, nb in _halo_pairs(s):
                for f in fields:
                    t = self.field_of(s, f)
                    ops.append(dist.P2POp(dist.isend, t[send].contiguous(), nb, self.group))
                    ops.append(dist.P2POp(dist.irecv, t[recv], nb, self.group))
        if ops:
            for q in dist.batch_isend_irecv(ops):
                q.wait()


# -- solves -----------------------------------------------------------------------

def forward(slabs: List[Slab], p0s, nsteps: int, exchange):
    """traces_r = (H p0) at slab r's sampled receivers (rec_idx), for every
    slab held here.  p0s[i]: slab i's planes [zl, zh) of p0 (CUDA, float32)."""
    import torch
    outs = []
    for s, p0 in zip(slabs, p0s):
        tr = torch.empty((nsteps + 1, len(s.rec_idx)), device=p0.device, dtype=torch.float32)
        s.grid.begin(False, p0, s.rec_local, nsteps, tr)
        outs.append(tr)
    for _ in range(nsteps):
        _halves(slabs, exchange)
        exchange(slabs, SIGMA_FIELDS)
        for s in slabs:
            s.grid.step_receivers()
    return outs


def adjoint(slabs: List[Slab], traces, nsteps: int, exchange):
    """image_r = (H^T y) on slab r's planes [zl, zh) (owned planes exact);
    traces[i]: the (nsteps+1, len(inj_idx)) columns of y of slab i's
    injected receivers."""
    import torch
    outs = []
    for s, y in zip(slabs, traces):
        img = torch.empty(s.grid.shape, device=y.device, dtype=torch.float32)
        s.grid.begin(True, y.contiguous(), s.inj_local, nsteps, img)
        outs.append(img)
    exchange(slabs, SIGMA_FIELDS)
    for _ in range(nsteps):
        _halves(slabs, exchange)
        for s in slabs:
            s.grid.step_receivers()
        exchange(slabs, SIGMA_FIELDS)
    return outs


def _halves(slabs, exchange):
    for s in slabs:
        s.grid.step_half(False)
    exchange(slabs, U_FIELDS)
    for s in slabs:
        s.grid.step_half(True)


def gather_traces(slabs: List[Slab], outs, L: int):
    """The whole (nsteps+1, L) trace array from the slabs' sampled columns."""
    import torch
    full = torch.empty((outs[0].shape[0], L), device=outs[0].device, dtype=torch.float32)
    for s, tr in zip(slabs, outs):
        if len(s.rec_idx):
            full[:, torch.as_tensor(s.rec_idx, device=full.device)] = tr
    return full


def assemble_image(slabs: List[Slab], outs):
    """The whole image from the slabs' owned planes (z order)."""
    import torch
    order = sorted(range(len(slabs)), key=lambda i: slabs[i].r)
    return torch.cat([outs[i][slabs[i].owned] for i in order], dim=0)


# -- results across processes (one slab per rank) ---------------------------------

def dist_gather_traces(s: Slab, tr, L: int, group=None):
    """The whole (nsteps+1, L) trace array on every rank, from each rank's
    sampled columns: every column is sampled by exactly one slab, so a sum
    all-reduce over zero-filled arrays gathers them exactly (x + 0 = x)."""
    import torch
    import torch.distributed as dist
    full = torch.zeros((tr.shape[0], L), dtype=tr.dtype, device=tr.device)
    if len(s.rec_idx):
        full[:, torch.as_tensor(s.rec_idx, device=tr.device)] = tr
    dist.all_reduce(full, group=group)
    return full


def dist_assemble_image(s: Slab, img, nz: int, group=None):
    """The whole (nz, ny, nx) image on every rank from each rank's owned planes
    (disjoint, so the sum all-reduce is exact)."""
    import torch
    import torch.distributed as dist
    full = torch.zeros((nz,) + tuple(img.shape[1:]), dtype=img.dtype, device=img.device)
    full[s.lo:s.hi] = img[s.owned]
    dist.all_reduce(full, group=group)
    return full


def dist_dot(a, b, group=None) -> float:
    """sum(a * b) over all ranks in float64 (one scalar all-reduce): the
    partial sums of the inner-product test <H p, y> = <p, H^T y> when each
    rank holds its own columns (traces) or owned planes (images)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float((a.double() * b.double()).sum())], dtype=torch.float64,
                     device=a.device)
    dist.all_reduce(t, group=group)
    return float(t.item())
