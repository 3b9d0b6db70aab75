#!/usr/bin/env python
"""Benchmark of the elastic FDTD operator pair H, H^T on B300.

One bench step = one time step of the forward operator H (velocity + phi,
stress + psi, receiver sampling) and one time step of its adjoint H^T
(transposed halves, receiver injection) over the full grid.  The timed region
runs pact_forward over K time steps and then pact_adjoint over the resulting
(K+1) x L traces: one application of H and one of H^T, as in one gradient
evaluation of a least-squares reconstruction.

Workload (default): the skull-like 512^3 grid, dx 0.2 mm, 20-cell C-PML,
1024 hemisphere receivers, dt at CFL 0.3.  Inputs are synthetic and seeded.
The nine wavefield arrays (537 MB each) exceed the 126 MB L2, so no L2 flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica of the workload (weak scaling, no collective on the data
path); value = updates of all ranks / max-over-ranks time.  With
--decomp slabs the ranks split one solve into z slabs instead (strong
scaling, halo planes exchanged over NCCL).  The default line also carries a
short serving leg (--serving-requests): a seeded request stream served with
continuous batching and one at a time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "elastic FDTD grid-pt updates/s (fwd+adj)"
UNIT = "grid-pt updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["skull-512", "skull-256", "skull-192"], default="skull-512")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mu0", action="store_true",
                    help="acoustic ablation H_{mu=0}: shear modulus set to 0 (lambda + 2 mu kept)")
    ap.add_argument("--serving", action="store_true",
                    help="serve a seeded Poisson stream (continuous batching vs one at a time)")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--ksteps", type=int, default=16)
    ap.add_argument("--fill-points", type=int, default=None,
                    help="serving: admit while the admitted solves hold fewer grid points than this")
    ap.add_argument("--policy", choices=["srpt", "all"], default="srpt",
                    help="serving: advance the shortest remaining solves (srpt) or every admitted one (all)")
    ap.add_argument("--decomp", choices=["replicas", "slabs"], default="replicas",
                    help="N > 1: independent solves per rank (replicas, weak scaling) or one solve split "
                         "into z slabs over the ranks (strong scaling)")
    ap.add_argument("--serving-requests", type=int, default=40,
                    help="requests of the serving leg of the default bench line (0: no serving leg)")
    return ap.parse_args()


def make_workload(name):
    from paper_1709_02733_b300 import synth
    return {"skull-512": synth.skull_512, "skull-256": synth.skull_256, "skull-192": synth.skull_192}[name]()


def workload_config(w, name):
    d = w.desc
    return {
        "workload": f"{name}: {d.nx}^3 skull-like elastic medium (water / 7 mm shell / tissue), dx {d.dx * 1e3:.2f} mm, "
                    f"dt {d.dt * 1e9:.2f} ns, {d.npml}-cell C-PML, {w.rec.shape[0]} hemisphere receivers, "
                    f"forward + adjoint",
        "grid": [d.nx, d.ny, d.nz],
        "receivers": int(w.rec.shape[0]),
        "npml": d.npml,
        "full_solve_steps": w.nsteps,
        "l2": "no flush: inputs larger than L2 (9 wavefield arrays of %.0f MB each)" % (d.N * 4 / 1e6),
    }


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    """SM clock and clock-event reasons of the bench's GPU while the timed
    region runs: every 20 ms from a thread through NVML (read-only queries)
    where its Python binding is installed, else nvidia-smi's query loop every
    50 ms.  The GPU is found by its PCI address, so that the sample is of the
    device torch uses whatever CUDA_VISIBLE_DEVICES holds."""
    PERIOD = 0.02

    def __init__(self, device_index):
        self.dev = device_index
        self.rows = []
        self.h = None
        self.thread = None
        self.proc = None

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def _bus(self):
        import torch
        pr = torch.cuda.get_device_properties(self.dev)
        return f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"

    def start(self):
        import threading
        self.proc = None
        try:
            import pynvml
            pynvml.nvmlInit()
            self.h = pynvml.nvmlDeviceGetHandleByPciBusId(self._bus())
            self.smax = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
        except Exception:
            # no NVML binding: nvidia-smi's query loop (50 ms) on the same GPU
            self.h = None
            try:
                fd, self.path = tempfile.mkstemp(suffix=".csv")
                os.close(fd)
                self.f = open(self.path, "w")
                self.proc = subprocess.Popen(["nvidia-smi", "-i", self._bus(), f"--query-gpu={self.Q}",
                                              "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                             stderr=subprocess.DEVNULL)
            except Exception:
                self.proc = None
            return
        self.stop_flag = threading.Event()

        def run():
            import pynvml
            while True:
                try:
                    sm = pynvml.nvmlDeviceGetClockInfo(self.h, pynvml.NVML_CLOCK_SM)
                    rs = pynvml.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                    self.rows.append((sm, rs))
                except Exception:
                    pass
                if self.stop_flag.wait(self.PERIOD):
                    break

        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()

    def _stop_smi(self):
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 6 and parts[0].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower() == "active"})
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(float(r[0]) for r in rows), "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi, 50 ms"}

    def stop(self):
        if self.proc is not None:
            return self._stop_smi()
        if self.h is None or self.thread is None:
            return None
        self.stop_flag.set()
        self.thread.join(timeout=5)
        import pynvml
        if not self.rows:
            return None
        bits = {"hw_slowdown": pynvml.nvmlClocksEventReasonHwSlowdown,
                "hw_thermal_slowdown": pynvml.nvmlClocksEventReasonHwThermalSlowdown,
                "sw_thermal_slowdown": pynvml.nvmlClocksEventReasonSwThermalSlowdown,
                "sw_power_cap": pynvml.nvmlClocksEventReasonSwPowerCap}
        reasons = sorted({k for _, rs in self.rows for k, b in bits.items() if rs & b})
        return {"sm_mhz": statistics.median(r[0] for r in self.rows), "sm_max_mhz": self.smax,
                "reasons": reasons, "samples": len(self.rows), "source": "NVML, 20 ms"}


# --------------------------------------------------------------------------
# algorithmic bytes of each kernel role (one launch over the whole grid)
# --------------------------------------------------------------------------
def slab_points(d):
    if d.npml <= 0:
        return [0, 0, 0]
    W = 2 * d.npml + 1
    return [d.nz * d.ny * W, d.nz * W * d.nx, W * d.ny * d.nx]


def algorithmic_bytes(kind, d, L, points=None, slab=None):
    """Bytes one launch set of a role is designed to move: every array its
    kernels read once and write once at the points they update (neighbour
    reads served from cache are not counted).  This is the library's own
    per-role figure (the two-pass roles re-read the fields the other pass
    wrote); the roofline's compulsory bytes are compulsory_bytes_per_step.  points / slab: grid
    points and C-PML slab points the role updates (default: the whole grid)."""
    N = d.N if points is None else points
    S = sum(slab_points(d)) if slab is None else slab
    f = 4
    if kind == "fwd_velocity":   # read 6 sigma, 3 u, rho, alpha; write 3 u; phi^{ij} r+w on slabs
        return f * (11 * N + 3 * N) + 2 * f * 3 * S
    if kind == "fwd_stress":     # read 3 u, 6 sigma, lambda, mu; write 6 sigma; psi^{ij} r+w on slabs
        return f * (11 * N + 6 * N) + 2 * f * 3 * S
    if kind == "adj_a":          # read 6 Q, 3 w, rho, alpha; write 3 w; psi^ read, phi~ r+w on slabs
        return f * (11 * N + 3 * N) + f * 3 * S + 2 * f * 3 * S
    if kind == "adj_b":          # read 3 w, 6 Q, lambda, mu; write 6 Q; phi~ read, psi^ r+w on slabs
        return f * (11 * N + 6 * N) + f * 3 * S + 2 * f * 3 * S
    if kind in ("fwd_fused", "adj_fused"):  # read 9 fields, rho, alpha, lambda, 1/mu; write 9 fields
        return f * (9 + 4 + 9) * N
    if kind in ("fwd_ac_vel", "adj_ac_a"):  # acoustic: read s, u x3, rho, alpha; write u x3
        return f * 9 * N
    if kind in ("fwd_ac_str", "adj_ac_b"):  # acoustic: read u x3, s, lambda; write s x3 (the normal stresses)
        return f * 8 * N
    if kind == "sample":
        return f * (3 * 8 * L + L) + 8 * 8 * L
    if kind == "inject":         # 3 normal Q r+w and lambda, mu at the 8 corners of each receiver
        return f * (2 * 3 * 8 * L + 2 * 8 * L + L) + 8 * 8 * L
    return 0


def compulsory_bytes_per_step(d):
    """Compulsory DRAM bytes of one time step of one operator (H or H^T) over
    the whole grid, for the single-pass update of Eq. (it) with the C-PML of
    Appendix A.3: the nine wavefield fields read once and written once (72 B)
    and the four medium arrays rho, lambda, mu, alpha read once (16 B) at
    every grid point, plus the six memory variables of each axis read and
    written (48 B) at every point of that axis's two slabs (the library keeps
    2P + 1 planes per axis).  88 B per point in the interior, 99.5 B per point
    on average at 512^3 with a 20-cell layer."""
    return 88 * d.N + 48 * sum(slab_points(d))


def source_sha():
    from paper_1709_02733_b300.profiling import source_sha as sha
    return sha()


def traffic_for(kind, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources and on this workload (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
    except Exception:
        return None
    e = t.get(kind)
    if not e or e.get("source_sha") != source_sha() or e.get("workload") != workload:
        return None
    return e.get("dram_bytes_per_launch")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "of measured"
    except Exception:
        return {"hbm_gbs": 6400.0}, "of fallback"


# --------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# --------------------------------------------------------------------------
def crop_workload(w, n):
    import numpy as np
    from paper_1709_02733_b300.synth import GridDesc
    c = w.desc.nx // 2
    lo = c - n // 2
    sl = (slice(lo, lo + n),) * 3
    d = GridDesc(n, n, n, w.desc.dx, w.desc.dt, npml=min(w.desc.npml, max(0, (n - 2) // 2 - 1)),
                 pml_vmax=w.desc.pml_vmax)
    med = [np.ascontiguousarray(m[sl]) for m in w.medium]
    return d, med, np.ascontiguousarray(w.p0[sl])


def oracle_rate(w, n, fwd_steps, adj_steps, max_seconds=None):
    """Time the oracle's own forward step and transposed step on an n^3 crop of
    the workload; returns (updates/s, steps done, seconds)."""
    from oracle import Oracle
    d, med, p0 = crop_workload(w, n)
    o = Oracle(d.as_dict(), *med)
    st = o.inject(p0)
    st2 = o.inject(p0)
    done, t = 0, 0.0
    for k in range(max(fwd_steps, adj_steps)):
        if k < fwd_steps:
            t0 = time.perf_counter()
            o.step(st)
            t += time.perf_counter() - t0
            done += 1
        if k < adj_steps:
            t0 = time.perf_counter()
            o.step_T(st2)
            t += time.perf_counter() - t0
            done += 1
        if max_seconds is not None and t > max_seconds:
            break
    return done * d.N / t, done, t, d


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def cpu_baseline(w):
    import oracle
    oracle.build()
    rate, done, t, d = oracle_rate(w, 256 if w.desc.nx >= 256 else w.desc.nx, 10, 10, max_seconds=20.0)
    return {"value": rate, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"FP64 C oracle (OpenMP) on the central {d.nx}^3 crop of the workload "
                      f"({d.npml}-cell C-PML), {done} single time steps alternating forward W' and "
                      f"transposed W'^T, {t:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = make_workload(args.workload)
    # calibrate, then size the crop so the whole run takes about two minutes
    r0, _, _, _ = oracle_rate(w, 64, 1, 1)
    per_step = 120.0 / max(1, args.steps + args.warmup)
    n = int(max(24, min(256, w.desc.nx, (per_step * r0 / 2.0) ** (1.0 / 3.0))))
    from oracle import Oracle
    d, med, p0 = crop_workload(w, n)
    o = Oracle(d.as_dict(), *med)
    st = o.inject(p0)
    st2 = o.inject(p0)
    for _ in range(args.warmup):
        o.step(st)
        o.step_T(st2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(st)
        o.step_T(st2)
    t = time.perf_counter() - t0
    value = 2.0 * d.N * args.steps / t
    sample = (f"FP64 C oracle on the central {n}^3 crop of the {args.workload} workload; each step one forward "
              f"W' and one transposed W'^T time step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(w, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# replicas on several GPUs (weak scaling, no collective on the data path)
# --------------------------------------------------------------------------
def max_over_ranks_of(x, world, device="cpu"):
    """The slowest rank's value of x (one scalar all-reduce; x itself with
    one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(updates_per_rank, ms_local, world, device="cpu"):
    """(job ms, whole-job updates/s): every rank runs its own replica of the
    workload, the job takes as long as the slowest rank, and the value counts
    the updates of all ranks."""
    ms = max_over_ranks_of(ms_local, world, device)
    return ms, updates_per_rank * world / (ms * 1e-3)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1709_02733_b300 import build as pbuild
    from paper_1709_02733_b300 import pact

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pbuild.build()
    if world > 1:
        dist.barrier()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return max_over_ranks_of(x, world, device="cuda")

    w = make_workload(args.workload)
    if args.mu0:
        w.lam = (w.lam + 2.0 * w.mu).astype(np.float32)
        w.mu = np.zeros_like(w.mu)
    d = w.desc
    K, W = args.steps, args.warmup
    L = w.rec.shape[0]
    stream = torch.cuda.current_stream()
    g = pact.Grid(d, stream=stream)
    g.set_medium(*[torch.from_numpy(m).cuda() for m in w.medium])
    p0 = torch.from_numpy(w.p0).cuda()
    traces = torch.empty((K + 1, L), device="cuda")
    image = torch.empty(d.shape, device="cuda")

    # warm-up
    wt = g.forward(p0, w.rec, W)
    g.adjoint(wt, w.rec)
    torch.cuda.synchronize()

    # timed region: H over K steps, then H^T over the K+1 samples, on the
    # product path (pact_forward / pact_adjoint replaying their step graphs);
    # pact_profile(False) only resets the launch counts
    g.profile(False)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.forward(p0, w.rec, K, out=traces)
    g.adjoint(traces, w.rec, out=image)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms, value = replica_rate(2.0 * d.N * K, e0.elapsed_time(e1), world, device="cuda")
    gpu_launches = int(g.profile_read()["all"][0])  # kernel launches in the timed region
    updates = 2.0 * d.N * K * world

    # per-role device times from a second, profiled pass (events after every
    # launch, so launched directly rather than from the step graphs) over
    # Kp <= K steps; Kp takes the place of K in the per-launch figures below
    Kp = min(K, 200)
    g.profile(True)
    g.forward(p0, w.rec, Kp, out=traces[:Kp + 1])
    g.adjoint(traces[:Kp + 1], w.rec, out=image)
    torch.cuda.synchronize()
    prof = g.profile_read()
    g.profile(False)

    # roofline of the whole step pair (measured live over the timed region):
    # the compulsory bytes of the single-pass update (compulsory_bytes_per_step)
    # of H and of H^T over the device time of one forward + adjoint step
    pk, which = peaks()
    steps_kinds = ["fwd_velocity", "fwd_stress", "adj_a", "adj_b", "fwd_fused", "adj_fused", "fwd_ac_vel",
                   "fwd_ac_str", "adj_ac_a", "adj_ac_b"]
    pts = {k: g.role_points(k) for k in steps_kinds}
    pair_bytes = 2.0 * compulsory_bytes_per_step(d)
    achieved = pair_bytes / (ms / K * 1e-3) / 1e9
    wl = args.workload + (" mu=0" if args.mu0 else "")
    ran = [k for k in steps_kinds if prof[k][0]]
    tr = [traffic_for(k, wl) for k in ran]
    roofline = {"bound": "hbm", "kernel": "forward + adjoint step pair (every step kernel)", "achieved": achieved,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                "peak_source": which + " (hbm_gbs, STREAM-style copy)",
                "traffic": (sum(tr) if ran and all(t is not None for t in tr) else None),
                "algorithmic_bytes_per_step_pair": pair_bytes, "bytes_per_update": pair_bytes / (2.0 * d.N),
                "basis": "88 B per grid point (9 fields read + written, rho lambda mu alpha read) + 48 B per "
                         "C-PML slab point per axis (6 memory variables read + written), per operator step; "
                         "time = ms_per_step (CUDA events around the timed region)"}
    # Bytes the library's kernels are designed to move per role launch set
    # (in a medium-adaptive step the fluid work items run the acoustic kernels
    # inside the velocity and stress roles: their points count at the acoustic
    # bytes)
    def merged_ac(k):
        ac = {"fwd_velocity": "fwd_ac_vel", "fwd_stress": "fwd_ac_str", "adj_a": "adj_ac_a", "adj_b": "adj_ac_b"}.get(k)
        return ac if ac and prof[ac][0] == 0 and pts[ac][0] > 0 else None

    # medium-adaptive item classes: stress-family points writing sigma^11
    # alone move 8 B fewer, velocity-family points loading no alpha 4 B fewer
    deep, noalpha = g.deep_points(), g.noalpha_points()

    def role_bytes(k):
        ac = merged_ac(k)
        b = algorithmic_bytes(k, d, L, *pts[k]) + (algorithmic_bytes(ac, d, L, *pts[ac]) if ac else 0)
        return b - (8 * deep if k in ("fwd_stress", "adj_b") else 4 * noalpha)

    def role_points(k):
        ac = merged_ac(k)
        return pts[k][0] + (pts[ac][0] if ac else 0)
    # the dominant kernel role, against the bytes its own design moves
    dom = max(steps_kinds, key=lambda k: prof[k][1])
    n_launch, dom_ms = prof[dom]
    avg_s = dom_ms * 1e-3 / max(n_launch, 1)
    dbytes = role_bytes(dom)
    roofline["dominant_kernel"] = {"kernel": dom, "design_bytes_per_launch": dbytes, "avg_launch_ms": avg_s * 1e3,
                                   "achieved": dbytes / avg_s / 1e9, "frac": dbytes / avg_s / 1e9 / pk["hbm_gbs"],
                                   "grid_points_per_launch": role_points(dom),
                                   "design_bytes_per_update": dbytes / max(1, role_points(dom)),
                                   "traffic": traffic_for(dom, wl), "profiled_steps": Kp}
    # the bytes the library's kernels are designed to move, over the step's device time
    step_bytes = sum(role_bytes(k) * prof[k][0] for k in steps_kinds if prof[k][0])
    step_ms = sum(prof[k][1] for k in steps_kinds)
    roofline["design"] = {"bytes_per_step_pair": step_bytes / Kp, "bytes_per_update": step_bytes / (2.0 * d.N * Kp),
                          "achieved": step_bytes / (step_ms * 1e-3) / 1e9,
                          "frac": step_bytes / (step_ms * 1e-3) / 1e9 / pk["hbm_gbs"]}
    kernels = {k: {"invocations": v[0], "ms": v[1]} for k, v in prof.items() if v[0] and k != "all"}

    # end to end through the host-pointer C-ABI calls (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        hp0 = torch.from_numpy(w.p0).pin_memory().numpy()
        htr = torch.empty((K + 1, L), dtype=torch.float32).pin_memory().numpy()
        him = torch.empty(d.shape, dtype=torch.float32).pin_memory().numpy()
        barrier()
        t0 = time.perf_counter()
        g.forward_host(hp0, w.rec, K, out=htr)
        g.adjoint_host(htr, w.rec, out=him)
        barrier()
        te = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": updates / te, "unit": UNIT, "h2d_bytes_per_step": (d.N * 4 + (K + 1) * L * 4) / K,
               "d2h_bytes_per_step": ((K + 1) * L * 4 + d.N * 4) / K,
               "note": "pact_forward_host + pact_adjoint_host: p0 in, traces out, traces in, image out"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    # the metric's latency half: a short seeded serving stream, both arms
    # (one GPU; rank 0 of a single-process run)
    g.close()
    serving = None
    if rank == 0 and world == 1 and args.serving_requests > 0:
        serving = serving_leg(args.serving_requests, args.ksteps, args.fill_points, args.policy)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded skull-like medium, vessel tubes, Fibonacci receivers)",
                "config": dict(workload_config(w, args.workload), parallelism=f"replicas x{world}",
                               **({"medium": "mu = 0 (acoustic ablation, lambda + 2 mu kept)"} if args.mu0 else {})),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
                "kernels": kernels, "clocks": clk, "serving": serving}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


SERVE_KW = dict(rate=40.0, seed=5, n_range=(96, 320), n_step=8, steps_range=(800, 2500), L_range=(64, 512))
SERVE_BUDGET = 120 * 10 ** 9
SERVE_SLOTS = 32


def serving_leg(requests, ksteps, fill_points=None, policy="srpt"):
    """Serving workload: Poisson arrivals at 40 req/s, cubic grids of side 96..320
    (multiples of 8), dx 0.4 mm, 10-cell C-PML, 800..2500 steps, 64..512
    hemisphere receivers, forward/adjoint 50/50, 120 GB HBM budget, 32 slots.
    The same requests are served (a) with continuous batching through
    pact_advance and (b) one at a time with pact_forward / pact_adjoint, in
    real time on this GPU; returns both arms' statistics and their ratios.
    policy: which admitted solves each chunk advances (serving.run_continuous:
    "srpt", shortest remaining work first, or "all")."""
    from paper_1709_02733_b300 import serving
    cache = serving.InputCache()
    cont = serving.run_continuous(serving.make_stream(requests, **SERVE_KW), SERVE_BUDGET, ksteps=ksteps,
                                  max_slots=SERVE_SLOTS, cache=cache, realtime=True, fill_points=fill_points,
                                  policy=policy)
    solo = serving.run_one_at_a_time(serving.make_stream(requests, **SERVE_KW), cache=cache, realtime=True)
    return {"workload": f"serving stream: {requests} seeded Poisson requests at 40 req/s, sides 96..320 step 8, "
                        "800..2500 steps, 64..512 receivers, fwd/adj 50/50, 120 GB budget, 32 slots",
            "ksteps": ksteps, "fill_points": fill_points, "policy": policy, "continuous": cont, "one_at_a_time": solo,
            "throughput_ratio": cont["updates_per_s"] / solo["updates_per_s"],
            "p50_ratio": cont["p50_s"] / solo["p50_s"], "p99_ratio": cont["p99_s"] / solo["p99_s"]}


def run_serving(args):
    """The serving workload alone (serving_leg), as its own JSON line."""
    import torch
    from paper_1709_02733_b300 import build as pbuild
    pbuild.build()
    torch.cuda.set_device(0)
    sv = serving_leg(args.requests, args.ksteps, args.fill_points, args.policy)
    line = {"metric": "served p50/p99 latency beside throughput", "value": sv["continuous"]["p99_s"],
            "unit": "s (p99)", "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": sv["workload"], "ksteps": args.ksteps, "fill_points": args.fill_points,
                       "policy": args.policy}}
    line.update({k: sv[k] for k in ("continuous", "one_at_a_time", "throughput_ratio", "p50_ratio", "p99_ratio")})
    print(json.dumps(line), flush=True)


def run_slabs(args):
    """One solve of the workload split into z slabs over the WORLD_SIZE ranks
    (slabs.py: halo planes exchanged over NCCL between the half steps), timed
    like run_ours: K forward steps then K adjoint steps, max over ranks;
    value = the whole grid's updates / that time (strong scaling)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1709_02733_b300 import build as pbuild
    from paper_1709_02733_b300 import slabs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pbuild.build()
    if world > 1:
        dist.barrier()
    w = make_workload(args.workload)
    d = w.desc
    K, W = args.steps, args.warmup
    parts = slabs.partition(d.nz, world, d.npml)
    s = slabs.make_slab(d, parts, rank, w.rec)
    s.grid.set_medium(*[torch.from_numpy(np.ascontiguousarray(m[s.zl:s.zh])).cuda() for m in w.medium])
    p0 = torch.from_numpy(np.ascontiguousarray(w.p0[s.zl:s.zh])).cuda()
    y = torch.randn((K + 1, len(s.inj_idx)), device="cuda")
    ex = slabs.DistExchange() if world > 1 else (lambda sl, f: None)
    slabs.forward([s], [p0], W, ex)
    slabs.adjoint([s], [y[:W + 1].contiguous()], W, ex)

    def barrier():
        if world > 1:
            dist.barrier()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    slabs.forward([s], [p0], K, ex)
    slabs.adjoint([s], [y], K, ex)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks_of(e0.elapsed_time(e1), world, device="cuda")
    value = 2.0 * d.N * K / (ms * 1e-3)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms / K, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded skull-like medium, vessel tubes, Fibonacci receivers)",
                "config": dict(workload_config(w, args.workload), parallelism=f"z-slabs x{world}",
                               slabs=[list(p) for p in parts]),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    s.grid.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.serving:
        run_serving(args)
        return
    if args.decomp == "slabs" and args.impl == "ours":
        run_slabs(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
