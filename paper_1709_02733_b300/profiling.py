"""Summaries of Nsight Compute CSV output for the step kernels.

    python -m paper_1709_02733_b300.profiling launches <ncu.csv>
        per-kernel launches, device time and share (markdown table)
    python -m paper_1709_02733_b300.profiling traffic <ncu.csv> <out.json> [--scale F]
        DRAM bytes (read + write) per half step of each kernel role, as read by
        bench.py for the roofline "traffic" field; F scales a capture of a
        smaller grid to the full one (ratio of grid points)

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
    """bench.py kernel role of a launch (None for the small kernels)."""
    k = kernel_name.replace(" ", "")
    for prefix, adj, role in (("k_vel_tiled<0", False, "fwd_velocity"), ("k_str_tiled<0", False, "fwd_stress"),
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


def traffic(path, scale: float = 1.0) -> dict:
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
    return {role: {"dram_bytes_per_launch": b, "source_sha": sha, "scale": scale} for role, b in acc.items()}


def main(argv):
    if len(argv) >= 2 and argv[0] == "launches":
        print(launch_table(argv[1]))
    elif len(argv) >= 3 and argv[0] == "traffic":
        scale = float(argv[argv.index("--scale") + 1]) if "--scale" in argv else 1.0
        with open(argv[2], "w") as f:
            json.dump(traffic(argv[1], scale), f, indent=1)
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
