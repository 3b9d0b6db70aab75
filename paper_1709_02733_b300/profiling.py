"""Summaries of Nsight Compute CSV output for the step kernels.

    python -m paper_1709_02733_b300.profiling launches <ncu.csv>
        per-kernel launches, device time and share (markdown table)
    python -m paper_1709_02733_b300.profiling fullset <raw.csv>
        key counters of a full-set capture (``ncu -i rep --page raw --csv``):
        duration, DRAM bytes and throughput, occupancy, issue activity and the
        top warp-stall reasons of every captured launch (markdown)
    python -m paper_1709_02733_b300.profiling traffic <ncu.csv> <out.json> [--scale F] [--workload W]
        DRAM bytes (read + write) per half step of each kernel role, as read by
        bench.py for the roofline "traffic" field; F scales a capture of a
        smaller grid to the full one (ratio of grid points); W names the bench
        workload the capture ran (default skull-512; " mu=0" appended for the
        acoustic ablation), and bench.py only reports the figure for that one

The CSV is ``ncu --csv --log-file`` output with one row per (launch, metric).
A kernel role of bench.py (fwd_velocity, fwd_stress, adj_a, adj_b) is one
half step, i.e. the C-PML launch plus the interior launch of that family.
"""
from __future__ import annotations

import collections
import csv
import hashlib
import json
import os
import sys

_PKG = os.path.dirname(os.path.abspath(__file__))


def source_sha() -> str:
    """Hash of the CUDA sources: a recorded traffic figure is only valid for them."""
    h = hashlib.sha256()
    csrc = os.path.join(_PKG, "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def role_of(kernel_name: str):
    """bench.py kernel role of a launch (None for the small kernels).  In a
    medium-adaptive step the fluid kernels (k_fluid<STR, ADJ, PM>, k_ac_vel,
    k_ac_str) run inside the velocity and stress roles."""
    k = kernel_name.replace(" ", "")
    for prefix, adj, role in (("k_fluid<0,0", False, "fwd_velocity"), ("k_fluid<1,0", False, "fwd_stress"),
                              ("k_fluid<0,1", True, "adj_a"), ("k_fluid<1,1", True, "adj_b"),
                              ("k_ac_vel<0", False, "fwd_velocity"), ("k_ac_str<0", False, "fwd_stress"),
                              ("k_ac_vel<1", True, "adj_a"), ("k_ac_str<1", True, "adj_b"),
                              ("k_vel_tiled<0", False, "fwd_velocity"), ("k_str_tiled<0", False, "fwd_stress"),
                              ("k_vel_tiled<1", True, "adj_a"), ("k_str_tiled<1", True, "adj_b"),
                              ("k_fwd_velocity", False, "fwd_velocity"), ("k_fwd_stress", False, "fwd_stress"),
                              ("k_adj_a", True, "adj_a"), ("k_adj_b", True, "adj_b")):
        if prefix in k:
            return role
    return None


def read(path):
    rows = [r for r in csv.reader(open(path)) if len(r) > 5]
    hdr = rows[0]
    ki, vi, mi, ii = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Name"), hdr.index("ID")
    launches = collections.OrderedDict()
    for r in rows[1:]:
        launches.setdefault(r[ii], {"name": r[ki].split("(")[0].strip()})[r[mi]] = float(r[vi].replace(",", ""))
    return list(launches.values())


def launch_table(path) -> str:
    agg = collections.defaultdict(lambda: [0, 0.0])
    for L in read(path):
        if "gpu__time_duration.sum" in L:
            agg[L["name"]][0] += 1
            agg[L["name"]][1] += L["gpu__time_duration.sum"]
    tot = sum(v[1] for v in agg.values()) or 1.0
    out = ["| kernel | launches | total device time [us] | per launch [us] | share |", "|---|---|---|---|---|"]
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append(f"| `{k}` | {n} | {t / 1e3:.1f} | {t / n / 1e3:.1f} | {100 * t / tot:.1f} % |")
    return "\n".join(out)


def traffic(path, scale: float = 1.0, workload: str = "skull-512") -> dict:
    """DRAM bytes per half step of each role: every kernel of a role runs once
    per half step, so the role's figure is the sum over its kernels of their
    mean bytes per launch."""
    per_kernel = collections.defaultdict(lambda: [0, 0.0])
    for L in read(path):
        if role_of(L["name"]) and "dram__bytes_read.sum" in L:
            k = per_kernel[L["name"]]
            k[0] += 1
            k[1] += L["dram__bytes_read.sum"] + L["dram__bytes_write.sum"]
    acc = collections.defaultdict(float)
    for name, (n, b) in per_kernel.items():
        acc[role_of(name)] += b / n * scale
    sha = source_sha()
    return {role: {"dram_bytes_per_launch": b, "source_sha": sha, "scale": scale, "workload": workload}
            for role, b in acc.items()}


FULLSET_KEYS = [
    ("gpu__time_duration.sum", "duration [us]", "us"),
    ("dram__bytes_read.sum", "DRAM read [MB]", "MB"),
    ("dram__bytes_write.sum", "DRAM write [MB]", "MB"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput [% of peak]", 1.0),
    ("launch__registers_per_thread", "registers / thread", 1.0),
    ("launch__occupancy_limit_registers", "blocks / SM (register limit)", 1.0),
    ("launch__occupancy_limit_shared_mem", "blocks / SM (shared-memory limit)", 1.0),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active [% of peak]", 1.0),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active [% of peak]", 1.0),
    ("smsp__inst_executed.sum", "warp instructions [M]", 1e-6),
    ("lts__t_sector_hit_rate.pct", "L2 hit rate [%]", 1.0),
    ("sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active", "tensor pipe active [%]", 1.0),
]


def fullset_table(path) -> str:
    """Markdown summary of a raw-page CSV export (one row per launch)."""
    rows = [r for r in csv.reader(open(path)) if len(r) > 5]
    hdr, units, data = rows[0], rows[1], rows[2:]
    col = {h: i for i, h in enumerate(hdr)}
    to_us = {"nsecond": 1e-3, "usecond": 1.0, "msecond": 1e3, "second": 1e6}
    to_mb = {"byte": 1e-6, "Kbyte": 1e-3, "Mbyte": 1.0, "Gbyte": 1e3}

    def num(r, k):
        try:
            return float(r[col[k]].replace(",", ""))
        except (KeyError, ValueError):
            return None

    def factor(k, scale):
        u = units[col[k]] if k in col else ""
        if scale == "us":
            return to_us.get(u, 1.0)
        if scale == "MB":
            return to_mb.get(u, 1.0)
        return scale

    names = [r[col["Kernel Name"]].split("(")[0].strip() for r in data]
    out = ["| counter | " + " | ".join(f"`{n}`" for n in names) + " |", "|---|" + "---|" * len(names)]
    for key, label, scale in FULLSET_KEYS:
        vals = [num(r, key) for r in data]
        if all(v is None for v in vals):
            continue
        f = factor(key, scale)
        out.append(f"| {label} | " + " | ".join("" if v is None else f"{v * f:.4g}" for v in vals) + " |")
    stall = [h for h in hdr if h.startswith("smsp__average_warps_issue_stalled_")
             and h.endswith("_per_issue_active.ratio")]
    for r, n in zip(data, names):
        top = sorted(((num(r, h) or 0.0, h[len("smsp__average_warps_issue_stalled_"):-len("_per_issue_active.ratio")])
                      for h in stall), reverse=True)[:5]
        out.append("")
        out.append(f"`{n}` top stall reasons (warps per issue): " + ", ".join(f"{k} {v:.2f}" for v, k in top))
    return "\n".join(out)


def main(argv):
    if len(argv) >= 2 and argv[0] == "launches":
        print(launch_table(argv[1]))
    elif len(argv) >= 2 and argv[0] == "fullset":
        print(fullset_table(argv[1]))
    elif len(argv) >= 3 and argv[0] == "traffic":
        scale = float(argv[argv.index("--scale") + 1]) if "--scale" in argv else 1.0
        workload = argv[argv.index("--workload") + 1] if "--workload" in argv else "skull-512"
        with open(argv[2], "w") as f:
            json.dump(traffic(argv[1], scale, workload), f, indent=1)
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
