"""Host logic of the measurement path (no GPU): ncu CSV parsing and the
per-role traffic figures, the source-hash keying of those figures, the
nvidia-smi clock summary, and the algorithmic byte counts behind the roofline."""
import csv
import json
import os

import pytest

import bench
from paper_1709_02733_b300 import profiling, synth

HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _write_launches(path, launches):
    """launches: (kernel name, time ns, read bytes, write bytes), one ncu row per metric."""
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(HDR)
        for i, (name, t, rd, wr) in enumerate(launches):
            for metric, unit, val in (("gpu__time_duration.sum", "nsecond", t), ("dram__bytes_read.sum", "byte", rd),
                                      ("dram__bytes_write.sum", "byte", wr)):
                w.writerow([str(i), "1", "python", "h", f"{name}(StepParams)", "1", "7", "(256, 1, 1)", "(10, 1, 1)",
                            "0", "10.3", "Command line profiler metrics", metric, unit, f"{val:,}"])


LAUNCHES = [
    ("void k_vel_tiled<0, 0>", 1000, 6_000, 1_000), ("void k_vel_tiled<0, 3>", 400, 2_000, 500),
    ("void k_vel_tiled<0, 1>", 50, 100, 20), ("void k_str_tiled<0, 0>", 1200, 7_000, 2_000),
    ("k_sample", 6, 10, 2), ("void k_vel_tiled<0, 0>", 1100, 6_200, 1_000),
    ("void k_vel_tiled<1, 0>", 1300, 7_000, 1_500), ("void k_str_tiled<1, 3>", 700, 3_000, 900),
]


def test_launch_table_shares(tmp_path):
    p = tmp_path / "l.csv"
    _write_launches(p, LAUNCHES)
    rows = profiling.read(p)
    assert len(rows) == len(LAUNCHES)
    assert rows[0]["dram__bytes_read.sum"] == 6000.0           # thousands separators parsed
    table = profiling.launch_table(p).splitlines()
    body = [r for r in table[2:]]
    assert body[0].startswith("| `void k_vel_tiled<0, 0>` | 2 | 2.1 | 1.1 |")   # two launches, 2100 ns
    shares = [float(r.split("|")[5].strip().rstrip(" %")) for r in body]
    assert sum(shares) == pytest.approx(100.0, abs=0.3)
    assert shares == sorted(shares, reverse=True)


def test_roles_and_traffic_per_half_step(tmp_path, monkeypatch):
    assert profiling.role_of("void k_vel_tiled<1, 3>(StepParams)") == "adj_a"
    assert profiling.role_of("void k_str_tiled<0, 1>") == "fwd_stress"
    assert profiling.role_of("k_adj_b(StepParams)") == "adj_b"
    assert profiling.role_of("k_sample") is None
    p = tmp_path / "l.csv"
    _write_launches(p, LAUNCHES)
    monkeypatch.setattr(profiling, "source_sha", lambda: "abc")
    t = profiling.traffic(p)
    # role figure = sum over its kernels of their mean bytes per launch
    assert t["fwd_velocity"]["dram_bytes_per_launch"] == pytest.approx((7000 + 7200) / 2 + 2500 + 120)
    assert t["fwd_stress"]["dram_bytes_per_launch"] == pytest.approx(9000)
    assert t["adj_a"]["dram_bytes_per_launch"] == pytest.approx(8500)
    assert t["adj_b"]["dram_bytes_per_launch"] == pytest.approx(3900)
    assert all(v["source_sha"] == "abc" and v["workload"] == "skull-512" for v in t.values())
    assert profiling.traffic(p, workload="skull-256")["adj_b"]["workload"] == "skull-256"
    assert profiling.traffic(p, scale=8.0)["adj_b"]["dram_bytes_per_launch"] == pytest.approx(31200)


def test_traffic_is_dropped_when_sources_or_workload_change(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    json.dump({"adj_b": {"dram_bytes_per_launch": 5.0, "source_sha": "old", "scale": 1.0, "workload": "skull-512"}},
              open(prof / "traffic.json", "w"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_sha", lambda: "old")
    assert bench.traffic_for("adj_b", "skull-512") == 5.0
    assert bench.traffic_for("adj_a", "skull-512") is None
    # another workload (or the acoustic ablation) never takes the skull-512 figure
    assert bench.traffic_for("adj_b", "skull-256") is None
    assert bench.traffic_for("adj_b", "skull-512 mu=0") is None
    monkeypatch.setattr(bench, "source_sha", lambda: "new")
    assert bench.traffic_for("adj_b", "skull-512") is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary(tmp_path):
    """nvidia-smi's query loop (no NVML binding): rows of SM clock, max clock
    and the four reasons; rows without a clock reading are dropped."""
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clk.csv")
    with open(s.path, "w") as f:
        for mhz, cap in ((2032, "Not Active"), (1995, "Active"), (2010, "Active"), ("[N/A]", "Not Active")):
            f.write(f"{mhz}, 2032, Not Active, Not Active, Not Active, {cap}\n")
    s.f = open(os.devnull, "w")
    s.proc = _Done()
    r = s.stop()
    assert r["sm_mhz"] == 2010.0 and r["sm_max_mhz"] == 2032.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 3
    assert not os.path.exists(s.path)


def test_clock_summary_nvml():
    """NVML samples: (SM clock, reason bit mask) pairs."""
    pynvml = pytest.importorskip("pynvml")

    class _Joined:
        def join(self, timeout=None):
            pass

    import threading
    s = bench.ClockSampler(0)
    s.h, s.smax, s.thread, s.stop_flag = object(), 2032, _Joined(), threading.Event()
    hw = pynvml.nvmlClocksEventReasonHwSlowdown
    s.rows = [(2032, 0), (1900, hw), (2032, pynvml.nvmlClocksEventReasonGpuIdle)]
    r = s.stop()
    assert r["sm_mhz"] == 2032 and r["sm_max_mhz"] == 2032 and r["samples"] == 3
    assert r["reasons"] == ["hw_slowdown"]


def test_algorithmic_bytes_of_the_step():
    """Per grid point away from the layers the two-pass step moves 56 + 68 B
    forward and 56 + 68 B adjoint; with skull-512's slabs the step pair is
    37,155,241,984 B (138.4 B per update of each operator)."""
    d = synth.GridDesc(512, 512, 512, 0.2e-3, 19.7e-9, npml=20)
    N = d.N
    assert bench.algorithmic_bytes("fwd_velocity", d, 0, slab=0) == 56 * N
    assert bench.algorithmic_bytes("fwd_stress", d, 0, slab=0) == 68 * N
    assert bench.algorithmic_bytes("adj_a", d, 0, slab=0) == 56 * N
    assert bench.algorithmic_bytes("fwd_fused", d, 0) == 88 * N
    assert bench.slab_points(d) == [512 * 512 * 41] * 3
    total = sum(bench.algorithmic_bytes(k, d, 0) for k in ("fwd_velocity", "fwd_stress", "adj_a", "adj_b"))
    assert total == 37155241984
    assert total / (2 * N) == pytest.approx(138.414, abs=1e-3)
    assert bench.algorithmic_bytes("fwd_velocity", synth.GridDesc(8, 8, 8, 1e-3, 1e-7, npml=0), 0) == 56 * 512


def test_compulsory_bytes_of_the_single_pass_step():
    """The roofline's bytes: 88 B per grid point (nine fields read and written,
    four medium arrays read) plus 48 B per C-PML slab point of each axis (six
    memory variables read and written).  At 512^3 with a 20-cell layer (41
    slab planes per axis) that is 99.53 B per update, 26.7 GB per forward +
    adjoint step pair; a 7.581 ms step pair then runs at 0.554 of 6429 GB/s."""
    d = synth.GridDesc(512, 512, 512, 0.2e-3, 19.7e-9, npml=20)
    b = bench.compulsory_bytes_per_step(d)
    assert b == 88 * d.N + 48 * 3 * 512 * 512 * 41
    assert b / d.N == pytest.approx(99.53, abs=5e-3)
    assert 2 * b / 7.581e-3 / 1e9 / 6429.0 == pytest.approx(0.548, abs=2e-3)
    d0 = synth.GridDesc(64, 64, 64, 0.5e-3, 1e-7, npml=0)
    assert bench.compulsory_bytes_per_step(d0) == 88 * 64 ** 3
