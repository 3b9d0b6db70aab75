"""Continuous-batching server for forward (H) and adjoint (H^T) solves.

Requests of different grid sizes arrive over time.  The server keeps each
admitted solve's medium, wavefield and buffers resident on the GPU, admits
queued requests first-come-first-served while an HBM budget (and a slot limit)
allows, and advances all admitted solves together: every ``pact_advance`` call
replays a CUDA graph of k multi-instance steps (persistent step kernels that
walk a device table of the admitted solves).  Solves finish independently;
their memory is released and waiting requests are admitted in the same loop.

The one-at-a-time baseline (``run_one_at_a_time``) solves the same requests in
arrival order with ``pact_forward`` / ``pact_adjoint`` alone on the GPU.

Host-side pieces (``Admission``) have no GPU dependency and are tested on CPU.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np

from . import synth
from .synth import GridDesc

MAX_SLOTS = 64  # pact_advance takes at most 64 handles


@dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the stream
    adjoint: bool
    n: int                   # cubic grid side
    nsteps: int
    L: int
    seed: int
    # filled by the server
    admitted: Optional[float] = None
    done: Optional[float] = None
    result: Optional[object] = field(default=None, repr=False)

    @property
    def updates(self) -> float:
        return float(self.n) ** 3 * self.nsteps

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def make_stream(nreq=200, rate=40.0, seed=5, n_range=(96, 320), n_step=8, steps_range=(800, 2500),
                L_range=(64, 512)) -> List[Request]:
    """Seeded Poisson stream: exponential gaps (mean 1/rate), side uniform over
    multiples of n_step in n_range, nsteps and L uniform, forward/adjoint 50/50."""
    rng = np.random.default_rng(seed)
    t = 0.0
    sides = np.arange(n_range[0], n_range[1] + 1, n_step)
    out = []
    for k in range(nreq):
        t += rng.exponential(1.0 / rate)
        out.append(Request(rid=k, arrival=t, adjoint=bool(rng.random() < 0.5), n=int(rng.choice(sides)),
                           nsteps=int(rng.integers(steps_range[0], steps_range[1] + 1)),
                           L=int(rng.integers(L_range[0], L_range[1] + 1)), seed=int(seed * 1000 + k)))
    return out


class Admission:
    """First-come-first-served admission under a byte budget and a slot limit."""

    def __init__(self, budget_bytes: int, max_slots: int = MAX_SLOTS):
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.used = 0
        self.slots = 0

    def fits(self, nbytes: int) -> bool:
        return self.slots < self.max_slots and self.used + nbytes <= self.budget

    def take(self, nbytes: int) -> None:
        assert self.fits(nbytes)
        self.used += nbytes
        self.slots += 1

    def release(self, nbytes: int) -> None:
        self.used -= nbytes
        self.slots -= 1
        assert self.used >= 0 and self.slots >= 0

    def admit(self, queue: List, size_of: Callable[[object], int]) -> List:
        """Pop and return the longest prefix of the queue that fits (FIFO: a
        request that does not fit blocks the ones behind it)."""
        out = []
        while queue and self.fits(size_of(queue[0])):
            r = queue.pop(0)
            self.take(size_of(r))
            out.append(r)
        return out


# ---------------------------------------------------------------------------
# inputs (cached per grid side: the media are generated once)
# ---------------------------------------------------------------------------
SERVE_DX = 0.4e-3
SERVE_NPML = 10


class InputCache:
    def __init__(self):
        self._med: Dict[int, tuple] = {}

    def workload(self, n: int):
        if n not in self._med:
            d = GridDesc(n, n, n, SERVE_DX, synth.CFL * SERVE_DX / synth.SKULL_VMAX, npml=SERVE_NPML,
                         pml_vmax=synth.SKULL_VMAX)
            med = synth.skull_medium(n, SERVE_DX, SERVE_NPML, seed=n)
            p0 = synth.tubes_p0(n, SERVE_DX, SERVE_NPML, seed=n)
            self._med[n] = (d, med, p0)
        return self._med[n]

    def device_workload(self, n: int):
        """(desc, medium on the GPU, p0 on the GPU), uploaded once per grid side."""
        import torch
        if not hasattr(self, "_dev"):
            self._dev = {}
        if n not in self._dev:
            d, med, p0 = self.workload(n)
            self._dev[n] = (d, [torch.from_numpy(m).cuda() for m in med], torch.from_numpy(p0).cuda())
        return self._dev[n]

    def receivers(self, n: int, L: int):
        geo = synth.skull_geometry(n, SERVE_DX, SERVE_NPML)
        c = (n - 1) / 2.0
        return synth.fibonacci_hemisphere(L, geo.R_rec / SERVE_DX, (c, c, c))

    def traces(self, r: Request, dt: float):
        return synth.band_limited_traces(r.nsteps, r.L, r.seed, dt)


def handle_bytes(n: int, L: int, cache: InputCache) -> int:
    """Device bytes of a solver handle for an n^3 grid (pact_query_bytes)."""
    from .pact import pact_query_bytes
    return pact_query_bytes(cache.workload(n)[0], L, -1)


def io_bytes(r: Request) -> int:
    """Device bytes of a request's input and output buffers."""
    return (r.n ** 3 + (r.nsteps + 1) * r.L) * 4


def request_bytes(r: Request, cache: InputCache) -> int:
    """Device bytes a request holds while admitted: the handle (pact_query_bytes)
    plus its medium copy, input and output buffers."""
    return handle_bytes(r.n, r.L, cache) + 4 * r.n ** 3 * 4 + io_bytes(r)


class GridPool:
    """Idle solver handles by grid side, their medium already set.  A retired
    solve's handle serves the next request of the same size, so the serving
    loop neither allocates nor frees device memory while solves are in flight
    (a free synchronises the device).  Idle handles stay counted against the
    budget; the largest ones are closed when a new size needs room."""

    def __init__(self, cache: InputCache, stream):
        self.cache, self.stream = cache, stream
        self.idle: Dict[int, list] = {}

    def take(self, n: int):
        lst = self.idle.get(n)
        return lst.pop() if lst else None

    def put(self, n: int, g) -> None:
        self.idle.setdefault(n, []).append(g)

    def make(self, n: int):
        """A new handle for side n with its medium set (on the pool's stream)."""
        import torch
        from .pact import Grid
        d, dmed, _ = self.cache.device_workload(n)
        with torch.cuda.stream(self.stream):
            g = Grid(d, stream=self.stream)
            g.set_medium(*dmed)
        return g

    def evict(self):
        """Close one idle handle of the largest side; returns that side or None."""
        sides = [n for n, lst in self.idle.items() if lst]
        if not sides:
            return None
        n = max(sides)
        self.idle[n].pop().close()
        return n

    def close(self) -> None:
        for lst in self.idle.values():
            for g in lst:
                g.close()
        self.idle.clear()


# ---------------------------------------------------------------------------
# the server
# ---------------------------------------------------------------------------
class _Active:
    __slots__ = ("req", "grid", "bufs", "nbytes", "ev")

    def __init__(self, req, grid, bufs, nbytes):
        self.req, self.grid, self.bufs, self.nbytes, self.ev = req, grid, bufs, nbytes, None


def _buffers(r: Request, cache: InputCache, stream):
    """Receivers and the input / output buffers of one request, on `stream`."""
    import torch
    d, _, p0 = cache.device_workload(r.n)
    rec = cache.receivers(r.n, r.L)
    with torch.cuda.stream(stream):
        if r.adjoint:
            inp = torch.from_numpy(cache.traces(r, d.dt)).to("cuda", non_blocking=False)
            out = torch.empty(d.shape, device="cuda")
        else:
            inp = p0
            out = torch.empty((r.nsteps + 1, r.L), device="cuda")
    return rec, inp, out


FILL_POINTS = 24_000_000  # grid points in flight that keep one B300 busy (a ~290^3 grid)
ADVANCE_POINTS = 4_000_000  # grid points one chunk advances under the "srpt" policy


def pick_to_advance(remaining: List[float], points: List[int], advance_points: int) -> List[int]:
    """Shortest remaining work first: the indices of the solves to advance in
    the next chunk, by ascending remaining updates, until their grid points
    reach advance_points (at least one solve).  On a GPU that one solve of
    this size already keeps busy, the order changes no solve's cost, so the
    total time stays and the solves that are nearly done finish first."""
    order = sorted(range(len(remaining)), key=lambda i: (remaining[i], i))
    out, held = [], 0
    for i in order:
        if out and held >= advance_points:
            break
        out.append(i)
        held += points[i]
    return out


def run_continuous(requests: List[Request], budget_bytes: int, ksteps: int = 16, max_slots: int = 32,
                   cache: Optional[InputCache] = None, realtime: bool = True,
                   fill_points: Optional[int] = None, policy: str = "srpt",
                   advance_points: int = ADVANCE_POINTS) -> Dict:
    """Serve the stream with continuous batching; returns statistics.

    Admission is first-come-first-served under the HBM budget and the slot
    limit, and (fill_points) only while the admitted solves hold fewer grid
    points than keep the GPU busy: a large grid then runs nearly alone, as fast
    as it would one at a time, while small grids, which cannot fill the GPU
    alone, are advanced together.  fill_points=None (the default) admits up
    to the slot limit: with the persistent multi-instance kernels a nearly
    lone large grid advances slower than through pact_forward / pact_adjoint,
    and on the 40-request stream the cap lowered throughput to 0.61x.

    Loop: move arrived requests to the queue; admit FIFO while the budget and
    the slots allow (a handle is reused from the pool when one of the same
    size is idle, otherwise made, closing idle handles of other sizes if the
    budget needs room; its buffers are set up on a side stream that the
    serving stream then waits for); replay one k-step multi-instance graph over
    all admitted solves; retire solves whose last step has executed (their
    handles return to the pool).  At most two graph replays are in flight, so
    admissions and completions are seen within one chunk.  realtime=False
    skips idle waits (arrivals are then virtual).

    policy="all" advances every admitted solve in every chunk (processor
    sharing); policy="srpt" (the default) advances the admitted solves with
    the least remaining work, as many as hold advance_points grid points
    (pick_to_advance): the others stay resident and wait.  With one solve
    already keeping the GPU busy, both give the same total time; "srpt"
    finishes short solves first."""
    import collections

    import torch
    from .pact import pact_advance
    cache = cache or InputCache()
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    pool = GridPool(cache, side)
    adm = Admission(budget_bytes, min(max_slots, MAX_SLOTS))
    pending = sorted(requests, key=lambda r: r.arrival)
    queue: List[Request] = []
    active: List[_Active] = []
    finished: List[Request] = []
    hb = {n: handle_bytes(n, 512, cache) + 4 * n ** 3 * 4 for n in {r.n for r in requests}}
    for n in sorted(hb):
        cache.device_workload(n)
    torch.cuda.synchronize()
    clock = {"t0": time.perf_counter()}
    now = lambda: time.perf_counter() - clock["t0"]
    inflight = collections.deque()
    while pending or queue or active:
        if not realtime and not active and not queue and pending and pending[0].arrival > now():
            clock["t0"] -= pending[0].arrival - now()  # idle: jump to the next arrival
        while pending and pending[0].arrival <= now():
            queue.append(pending.pop(0))
        admitted = False
        while queue and adm.slots < adm.max_slots:
            r = queue[0]
            if fill_points is not None and active and \
                    sum(a.req.n ** 3 for a in active if a.ev is None) + r.n ** 3 > fill_points:
                break  # the GPU is busy enough: the head waits (FIFO)
            g = pool.take(r.n)
            if g is None:
                need = hb[r.n] + io_bytes(r)
                while not adm.fits(need):
                    n_ev = pool.evict()
                    if n_ev is None:
                        break
                    adm.used -= hb[n_ev]
                if not adm.fits(need):
                    break  # FIFO: the head waits for memory
                adm.take(need)
                g = pool.make(r.n)
            else:
                if adm.used + io_bytes(r) > adm.budget:
                    pool.put(r.n, g)
                    break
                adm.used += io_bytes(r)  # the handle's bytes are already counted
                adm.slots += 1
            queue.pop(0)
            r.admitted = now()
            rec, inp, out = _buffers(r, cache, side)
            with torch.cuda.stream(side):
                g.begin(r.adjoint, inp, rec, r.nsteps, out)
            active.append(_Active(r, g, (inp, out), io_bytes(r)))
            admitted = True
        if admitted:
            stream.wait_stream(side)
        if not active:
            if pending:
                time.sleep(max(0.0, min(pending[0].arrival - now(), 0.005)))
            continue
        running = [a for a in active if a.ev is None]
        if policy == "srpt" and running:
            rem = [float(a.req.n) ** 3 * (a.req.nsteps - a.grid.poll()) for a in running]
            running = [running[i] for i in pick_to_advance(rem, [a.req.n ** 3 for a in running], advance_points)]
        if running:
            pact_advance([a.grid for a in running], ksteps, stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        inflight.append(ev)
        for a in running:
            if a.ev is None and a.grid.poll() >= a.req.nsteps:
                a.ev = ev
        while len(inflight) > 1:
            inflight.popleft().synchronize()
        still = []
        for a in active:
            if a.ev is not None and a.ev.query():
                a.req.done = now()
                a.req.result = a.bufs[1]
                adm.used -= a.nbytes  # the handle stays counted while idle in the pool
                adm.slots -= 1
                side.wait_event(a.ev)  # the handle's next solve starts after this one
                pool.put(a.req.n, a.grid)
                finished.append(a.req)
            else:
                still.append(a)
        active = still
    torch.cuda.synchronize()
    stats = summarize(finished, now())
    pool.close()
    return stats


def run_one_at_a_time(requests: List[Request], cache: Optional[InputCache] = None, realtime: bool = True) -> Dict:
    """Baseline: each request alone on the GPU, in arrival order (handles
    reused from a pool of the same kind as the server's)."""
    import torch
    cache = cache or InputCache()
    stream = torch.cuda.current_stream()
    pool = GridPool(cache, stream)
    for n in sorted({r.n for r in requests}):
        cache.device_workload(n)
    torch.cuda.synchronize()
    clock = {"t0": time.perf_counter()}
    now = lambda: time.perf_counter() - clock["t0"]
    done = []
    for r in sorted(requests, key=lambda q: q.arrival):
        if now() < r.arrival:
            if realtime:
                time.sleep(r.arrival - now())
            else:
                clock["t0"] -= r.arrival - now()
        r.admitted = now()
        g = pool.take(r.n) or pool.make(r.n)
        rec, inp, out = _buffers(r, cache, stream)
        if r.adjoint:
            g.adjoint(inp, rec, out=out)
        else:
            g.forward(inp, rec, r.nsteps, out=out)
        torch.cuda.synchronize()
        r.done = now()
        r.result = out
        pool.put(r.n, g)
        done.append(r)
    stats = summarize(done, now())
    pool.close()
    return stats


def summarize(done: List[Request], wall: float) -> Dict:
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    upd = sum(r.updates for r in done)
    return {"requests": len(done), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "wall_s": wall, "updates": upd,
            "updates_per_s": upd / wall if wall > 0 else math.nan}
