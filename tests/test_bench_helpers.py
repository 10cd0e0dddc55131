"""Host-side helpers of bench.py: the DRAM-traffic figure from the committed
ncu capture (used only while the bulk kernel's source is unchanged), the
bulk-node counts of the benchmark workloads, and the CPU baseline's one-thread
leg (which restores the oracle's thread count)."""
import hashlib
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import lbm_workloads as W  # noqa: E402
import oracle  # noqa: E402


def test_traffic_capture_matches_the_current_bulk_source():
    line = [l for l in open(os.path.join(ROOT, "profiles", "k_bulk_d2q37_traffic.txt"))
            if l.startswith("traffic")][0]
    m = re.match(r"traffic\s+storage=(\w+)\s+nodes=(\d+)\s+bytes=(\d+)\s+src=(\w+)", line)
    src = open(os.path.join(ROOT, "paper_2307_16766_gb300", "csrc", "bulk.cu"), "rb").read()
    assert m.group(4) == hashlib.sha256(src).hexdigest()[:12]
    nodes, b = int(m.group(2)), int(m.group(3))
    assert bench.bulk_traffic("f32", nodes) == b
    assert abs(bench.bulk_traffic("f32", 2 * nodes) - 2 * b) <= 1
    assert bench.bulk_traffic("f64", nodes) is None          # no capture for that storage


def test_fp64_flop_count_matches_the_current_bulk_source():
    line = [l for l in open(os.path.join(ROOT, "profiles", "k_bulk_d2q37_f64_flops.txt"))
            if l.startswith("flops")][0]
    m = re.match(r"flops\s+nodes=(\d+)\s+dfma=(\d+)\s+dadd=(\d+)\s+dmul=(\d+)\s+src=(\w+)", line)
    h = hashlib.sha256()
    for f in ("bulk.cu", "collide.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2307_16766_gb300", "csrc", f), "rb").read())
    assert m.group(5) == h.hexdigest()[:12]
    n, fma, add, mul = (int(m.group(k)) for k in range(1, 5))
    c = bench.bulk_fp64_flops()
    assert c["flops"] == (2 * fma + add + mul) / n and c["instructions"] == (fma + add + mul) / n


def test_bulk_nodes_of_the_workloads():
    cfg, _ = bench.workload(1024, 512, "f32", 1)                    # inflow | CBC, periodic y
    assert bench.bulk_nodes(cfg) == (1024 - 6) * 512
    cfg, _ = W.pulse_d2q37(64, storage="f32")                       # four characteristic sides
    assert bench.bulk_nodes(cfg) == (64 - 6) ** 2
    cfg = W.run("D2Q9", 40, 30, 0.6, sides=("cbc",) * 4)
    assert bench.bulk_nodes(cfg) == 38 * 28


def test_cpu_baseline_reports_one_thread_and_restores_threads():
    cfg, f = W.vortex_d2q37(64, 32, steps=1, storage="f64")
    n = oracle.threads()
    r = bench.cpu_baseline(cfg, f, seconds=0.2, seconds_1t=0.2)
    assert oracle.threads() == n
    assert r["cores"] == n and r["kind"] == "oracle" and r["value"] > 0 and r["single_thread_value"] > 0
    assert isinstance(r["cpu"], str) and r["cpu"]


def test_clock_sampler_counts_only_the_timed_region():
    """Samples taken before ready() (nvidia-smi start-up, warm-up) are not
    counted; throttle reasons of the counted samples are reported."""
    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc = FakeProc()
    s.lines = ["0, 1200, 2070, 500, 0x4, Active, Not Active, Not Active, Not Active"]
    s.ready(timeout=0.0)
    s.lines += ["0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 2060, 2070, 950, 0x4, Not Active, Not Active, Not Active, Active"]
    c = s.stop()
    assert c["samples"] == 2 and c["sm_mhz"] == 2065.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
