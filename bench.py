"""Benchmark: MLUPS and fraction of the HBM roofline of the thermal LBM step
with the characteristic boundary condition, on the D2Q37 isentropic-vortex
workload (1024 x 512, inflow | CBC-RELAX outlet, periodic y).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage f32|f64|f16]
                  [--impl gb300|reference]

Prints one JSON line.  Timing: W untimed warm-up steps, then K steps, each
bracketed by CUDA events on the solver's stream with an L2 flush (a write,
then a read, of a 512 MB buffer) between timed steps; barrier + synchronize
around the timed region; the max over ranks is reported.  A step is one
lbm_step(1): the band kernel (strip nodes + characteristic boundary solver)
and the bulk kernel beside it.  The bulk kernel's duration (the roofline's
kernel time) comes from a second loop over the same steps in which the
library records the caller's events around each launch.  A third loop runs
the phases in sequence (breakdown), and a batched 96-run coefficient sweep
is timed beside the same runs stepped one after another; a 4096^2 pulse
(5 GB of populations) gives the step's throughput where the bulk dominates.
N > 1 runs
independent replicas, one per GPU (weak scaling; the method has no
cross-GPU exchange in this configuration).  The reference arm times the
FP64 CPU oracle on this host on the same workload and metric.
"""
import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbm_workloads as W  # noqa: E402

METRIC = "MLUPS (lattice updates/s / 1e6), D2Q37 thermal LBM + CBC step"
BYTES_PER_VALUE = {"f64": 8, "f32": 4, "f16": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "f16"])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--no-fp16-leg", action="store_true")
    ap.add_argument("--no-reference-leg", action="store_true",
                    help="skip the leg with populations held relative to the stream's equilibrium")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch-leg", action="store_true")
    ap.add_argument("--no-gradient-leg", action="store_true")
    ap.add_argument("--no-large-leg", action="store_true", help="skip the 4096^2 pulse throughput leg")
    ap.add_argument("--gradient-steps", type=int, default=1500)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--batch-steps", type=int, default=1000)
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(nx, ny, storage, steps, reference=False):
    """The benchmark vortex; with `reference` the populations are held
    relative to the stream's equilibrium (u_ref = (U0, 0))."""
    cfg, fields = W.vortex_d2q37(nx, ny, Ma=0.1, steps=steps, storage=storage, reference=reference)
    return cfg, fields


def workload_config(cfg, extra=None):
    d = {"workload": cfg["name"], "lattice": cfg["lattice"], "nx": cfg["nx"], "ny": cfg["ny"],
         "tau": cfg["tau"], "sides": cfg["sides"], "scheme_outlet": cfg["schemes"][1],
         "viscous": cfg["viscous"], "storage": cfg["storage"], "l2": "flushed between timed steps (512 MB write + read)"}
    if extra:
        d.update(extra)
    return d


# ------------------------------------------------------------ clocks ---

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    PERIOD_MS = 20      # the timed region of the default run is ~60 ms

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None
        self.first = 0      # samples before the timed region (not counted)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def ready(self, timeout=5.0):
        """Wait until nvidia-smi delivers samples, then count only the
        samples from now on (those of the timed region)."""
        end = time.perf_counter() + timeout
        while self.proc is not None and not self.lines and time.perf_counter() < end:
            time.sleep(0.01)
        self.first = len(self.lines)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines[self.first:]:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- peaks ---

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def bulk_traffic(storage, launch_nodes):
    """DRAM bytes per interior bulk-kernel launch from the committed ncu
    summary, if it was taken on the current kernel source (scaled by the
    nodes of the launch)."""
    src = os.path.join(ROOT, "paper_2307_16766_gb300", "csrc", "bulk.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:12]
    path = os.path.join(ROOT, "profiles", "k_bulk_d2q37_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        m = re.match(r"traffic\s+storage=(\w+)\s+nodes=(\d+)\s+bytes=(\d+)\s+src=(\w+)", line.strip())
        if m and m.group(1) == storage and m.group(4) == sha:
            nodes = int(m.group(2))
            return int(m.group(3)) * launch_nodes / nodes
    return None


def bulk_fp64_flops():
    """FP64 flops per node update of k_bulk<D2Q37, double> (2 per FMA, 1 per
    add or multiply) from the committed ncu counter capture, if it was taken
    on the current sources of the kernel (bulk.cu and collide.cuh)."""
    h = hashlib.sha256()
    for f in ("bulk.cu", "collide.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2307_16766_gb300", "csrc", f), "rb").read())
    sha = h.hexdigest()[:12]
    path = os.path.join(ROOT, "profiles", "k_bulk_d2q37_f64_flops.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        m = re.match(r"flops\s+nodes=(\d+)\s+dfma=(\d+)\s+dadd=(\d+)\s+dmul=(\d+)\s+src=(\w+)", line.strip())
        if m and m.group(5) == sha:
            n, fma, add, mul = (int(m.group(k)) for k in range(1, 5))
            return {"flops": (2 * fma + add + mul) / n, "instructions": (fma + add + mul) / n}
    return None


def fp64_roofline(interior_nodes, interior_ms):
    """The FP64 bulk kernel against the FP64 FMA throughput measured now on
    this GPU (lbm_fp64_fma_rate), with the flop count per update above."""
    import paper_2307_16766_gb300 as lbm
    peak = lbm.fp64_fma_rate() / 1e12
    cnt = bulk_fp64_flops()
    d = {"bound": "alu", "peak": peak, "unit": "TFLOP/s", "kernel": "k_bulk<D2Q37, double>",
         "peak_kind": "measured FP64 FMA throughput (lbm_fp64_fma_rate, this run)",
         "flops_per_update": None, "achieved": None, "frac": None, "issue_frac": None}
    if cnt is not None:
        rate = interior_nodes / (interior_ms / 1e3)
        d["flops_per_update"] = cnt["flops"]
        d["fp64_instructions_per_update"] = cnt["instructions"]
        d["achieved"] = cnt["flops"] * rate / 1e12
        d["frac"] = d["achieved"] / peak
        # FP64 instructions issued against the pipe's rate (an FMA is 2 flops, one issue)
        d["issue_frac"] = cnt["instructions"] * rate / (peak * 1e12 / 2)
    return d


def _open_axes(cfg):
    per_x = cfg["sides"][0] == "periodic"
    per_y = cfg["sides"][2] == "periodic"
    M = 3 if cfg["lattice"] == "D2Q37" else 1
    return per_x, per_y, M


def bulk_nodes(cfg):
    per_x, per_y, M = _open_axes(cfg)
    return (cfg["nx"] - (0 if per_x else 2 * M)) * (cfg["ny"] - (0 if per_y else 2 * M))


def interior_nodes(cfg):
    """Nodes of the bulk launch: every bulk node."""
    return bulk_nodes(cfg)


# -------------------------------------------------------- GPU measurement ---

def run_gpu(args, rank, world, local_rank, storage, want_e2e=True, reference=False):
    import torch
    import paper_2307_16766_gb300 as lbm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg, fields = workload(args.nx, args.ny, storage, args.steps, reference)
    sim = lbm.Simulation(cfg, device=dev)
    sim.init_fields(*fields)
    stream = sim.stream
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_sum = torch.empty((), dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize(dev)

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local_rank)
    sampler.start()
    sampler.ready()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(K):
            # Evict L2 between timed steps: write a 512 MB buffer, then read it
            # back so that the lines left in L2 are clean (no write-back of the
            # flush lands inside the next timed step).
            flush.fill_(float(k))
            torch.sum(flush, dim=0, out=flush_sum)
            ev[k][0].record(stream)
            sim.step(1)                 # band kernel, bulk kernel beside it
            ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = np.array([ev[k][0].elapsed_time(ev[k][1]) for k in range(K)])

    # Kernel durations while the two kernels run side by side: the same steps
    # with the library's timing hook, which records events around each
    # launch (the bulk kernel then runs on the solver's internal stream,
    # forked from and joined to the solver's stream).
    KE = min(K, 50)
    kev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(KE)]
    with torch.cuda.stream(stream):
        for evs in kev:                # events exist once recorded
            for e in evs:
                e.record(stream)
        for k in range(KE):
            flush.fill_(float(k))
            torch.sum(flush, dim=0, out=flush_sum)
            lbm.lbm_set_kernel_events(sim.handle, [e.cuda_event for e in kev[k]])
            sim.step(1)
    torch.cuda.synchronize(dev)
    lbm.lbm_set_kernel_events(sim.handle, [])
    interior_ms = np.array([kev[k][0].elapsed_time(kev[k][1]) for k in range(KE)])
    chain_ms = np.array([kev[k][3].elapsed_time(kev[k][4]) for k in range(KE)])

    # Breakdown, not part of the headline: the same steps with the phases in
    # sequence (bulk = rim + interior, then the boundary phase).
    KB = min(K, 20)
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(KB)]
    with torch.cuda.stream(stream):
        for k in range(KB):
            flush.fill_(float(k))
            torch.sum(flush, dim=0, out=flush_sum)
            pev[k][0].record(stream)
            sim.step_phase(0)
            pev[k][1].record(stream)
            sim.step_phase(1)
            pev[k][2].record(stream)
    torch.cuda.synchronize(dev)
    bulk_ms = np.array([pev[k][0].elapsed_time(pev[k][1]) for k in range(KB)])
    bnd_ms = np.array([pev[k][1].elapsed_time(pev[k][2]) for k in range(KB)])
    rho, ux, uy, T = sim.macros()
    finite = bool(np.all(np.isfinite(rho)) and np.all(np.isfinite(ux)))

    res = {"step_ms_total": float(step_ms.sum()), "interior_ms_mean": float(interior_ms.mean()),
           "boundary_overlapped_ms_mean": float(chain_ms.mean()),
           "bulk_ms_mean": float(bulk_ms.mean()), "boundary_ms_mean": float(bnd_ms.mean()),
           "wall_s": wall, "clocks": clocks, "finite": finite, "cfg": cfg,
           "bulk_nodes": bulk_nodes(cfg), "interior_nodes": interior_nodes(cfg)}

    if want_e2e:
        # End to end through the C ABI with pinned host buffers: every segment
        # copies the initial fields in, runs S steps and reads the macros back.
        S = 100
        n = sim.nx * sim.ny
        host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in fields]
        host_out = [torch.empty((sim.ny, sim.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
        segs = max(1, min(5, K // S))
        lbm.lbm_init_fields(sim.handle, n, *[t.numpy() for t in host_in])
        lbm.lbm_step(sim.handle, S)
        lbm.lbm_get_macros(sim.handle, *[t.data_ptr() for t in host_out], 0)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        for _ in range(segs):
            lbm.lbm_init_fields(sim.handle, n, *[t.numpy() for t in host_in])
            lbm.lbm_step(sim.handle, S)
            lbm.lbm_get_macros(sim.handle, *[t.data_ptr() for t in host_out], 0)
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t1
        # The same with one step per call (fields in, one step, macros out):
        # the cost of the host copies when nothing amortises them.
        calls = 20
        t2 = time.perf_counter()
        for _ in range(calls):
            lbm.lbm_init_fields(sim.handle, n, *[t.numpy() for t in host_in])
            lbm.lbm_step(sim.handle, 1)
            lbm.lbm_get_macros(sim.handle, *[t.data_ptr() for t in host_out], 0)
        torch.cuda.synchronize(dev)
        n1_s = time.perf_counter() - t2
        res["e2e"] = {"value": n * S * segs / e2e_s / 1e6, "unit": "MLUPS",
                      "h2d_bytes_per_step": 4 * 8 * n / S, "d2h_bytes_per_step": 4 * 8 * n / S,
                      "segment_steps": S, "segments": segs,
                      "one_step_per_call": {"value": n * calls / n1_s / 1e6, "unit": "MLUPS",
                                            "ms_per_call": n1_s / calls * 1e3, "calls": calls,
                                            "h2d_bytes_per_step": 4 * 8 * n, "d2h_bytes_per_step": 4 * 8 * n}}
    sim.close()
    return res


def run_large(args, local_rank, n=4096, kind="pulse"):
    """An n x n D2Q37 FP32 throughput grid: the pulse (CBC-RELAX on four
    sides, the 256^2 parity workload's recipe) or the benchmark's vortex
    workload (inflow | CBC-RELAX, periodic y) at that size.  Whole steps
    timed with CUDA events (5 GB of populations exceed L2, so no flush),
    then the bulk kernel's duration beside the band kernel through the
    timing hook, then both phases in sequence."""
    import torch
    import paper_2307_16766_gb300 as lbm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if kind == "pulse":
        cfg, fields = W.pulse_d2q37(n=n, storage="f32")
    else:
        cfg, fields = workload(n, n, "f32", 1)
    sim = lbm.Simulation(cfg, device=dev).init_fields(*fields)
    del fields
    stream = sim.stream
    sim.step(max(3, args.warmup))
    torch.cuda.synchronize(dev)
    K = max(1, min(args.steps, 40))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(K):
            sim.step(1)
            ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    step_ms = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(K)])
    KE = min(K, 20)
    kev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(KE)]
    with torch.cuda.stream(stream):
        for evs in kev:
            for e in evs:
                e.record(stream)
        for k in range(KE):
            lbm.lbm_set_kernel_events(sim.handle, [e.cuda_event for e in kev[k]])
            sim.step(1)
    torch.cuda.synchronize(dev)
    lbm.lbm_set_kernel_events(sim.handle, [])
    bulk_ms = np.array([kev[k][0].elapsed_time(kev[k][1]) for k in range(KE)])
    band_ms = np.array([kev[k][3].elapsed_time(kev[k][4]) for k in range(KE)])
    KB = min(K, 10)
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(KB)]
    with torch.cuda.stream(stream):
        for k in range(KB):
            pev[k][0].record(stream)
            sim.step_phase(0)
            pev[k][1].record(stream)
            sim.step_phase(1)
            pev[k][2].record(stream)
    torch.cuda.synchronize(dev)
    p_bulk = np.array([pev[k][0].elapsed_time(pev[k][1]) for k in range(KB)])
    p_band = np.array([pev[k][1].elapsed_time(pev[k][2]) for k in range(KB)])
    rho = sim.macros()[0]
    finite = bool(np.all(np.isfinite(rho)))
    sim.close()
    peak, peak_kind = measured_peaks()
    nodes, bn = n * n, bulk_nodes(cfg)
    step_s = float(step_ms.sum()) / 1e3
    return {"value": nodes * K / step_s / 1e6, "unit": "MLUPS", "steps": K,
            "ms_per_step": step_s / K * 1e3,
            "step_frac": 296.0 * nodes * K / step_s / 1e9 / peak,
            "bulk_ms": float(bulk_ms.mean()), "band_overlapped_ms": float(band_ms.mean()),
            "bulk_frac": 296.0 * bn / (float(bulk_ms.mean()) / 1e3) / 1e9 / peak,
            "phased_bulk_ms": float(p_bulk.mean()), "phased_band_ms": float(p_band.mean()),
            "peak_GBps": peak, "peak_kind": peak_kind, "finite": finite,
            "workload": cfg["name"] + ", tau 0.8, FP32 storage",
            "l2": "not flushed (populations exceed L2)"}


def run_batch(args, local_rank):
    """The batched coefficient sweep (96 uneven D2Q9/D2Q37 FP32 runs, CBC on
    all sides): every run stepped --batch-steps times through one Batch
    (persistent launches replayed as CUDA graphs), timed with CUDA events on
    the batch's stream; beside it the same runs stepped one after another
    as separate Simulations.  The batch's populations (about 2 GB) exceed
    L2, so no flush is needed between steps."""
    import torch
    import paper_2307_16766_gb300 as lbm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    runs = W.sweep_batch(96, storage="f32", steps=args.batch_steps)
    cfgs = [c for c, _ in runs]
    nodes = sum(c["nx"] * c["ny"] for c in cfgs)
    B = lbm.Batch(cfgs, device=dev)
    for r, (_, f) in enumerate(runs):
        B[r].init_fields(*f)
    B.step(max(3, args.warmup))                 # autotune, inflow-free graphs captured
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = args.batch_steps
    with torch.cuda.stream(B.stream):
        e0.record(B.stream)
        B.step(K)
        e1.record(B.stream)
    torch.cuda.synchronize(dev)
    batch_s = e0.elapsed_time(e1) / 1e3
    finite = all(bool(np.all(np.isfinite(B[r].macros()[0]))) for r in range(0, len(B), 8))
    ctas = {"D2Q9": B.ctas_per_sm("D2Q9", "f32"), "D2Q37": B.ctas_per_sm("D2Q37", "f32")}
    B.close()

    # the plain form: each run its own Simulation, stepped in turn
    KS = min(K, 100)
    sims = [lbm.Simulation(c, device=dev).init_fields(*f) for c, f in runs]
    for s_ in sims:
        s_.step(3)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for s_ in sims:
        s_.step(KS)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    seq_s = e0.elapsed_time(e1) / 1e3
    for s_ in sims:
        s_.close()
    q = {"D2Q9": 9, "D2Q37": 37}
    step_bytes = sum(2 * q[c["lattice"]] * 4 * c["nx"] * c["ny"] for c in cfgs)
    return {"value": nodes * K / batch_s / 1e6, "unit": "MLUPS", "runs": len(cfgs),
            "lattices": {k: sum(c["lattice"] == k for c in cfgs) for k in q},
            "nodes_per_step": nodes, "steps": K, "ms_per_step": batch_s / K * 1e3,
            "step_GBps": step_bytes * K / batch_s / 1e9, "ctas_per_sm": ctas,
            "sequential_value": nodes * KS / seq_s / 1e6, "sequential_steps": KS,
            "finite": finite,
            "workload": "96-run CBC coefficient sweep: D2Q9/D2Q37 by seeded coin, nx, ny ~ U{128..512}, "
                        "tau ~ U[0.55, 1], alpha_T, beta_P ~ U[0, 1], CBC-RELAX on four sides, mesoscopic viscous vector, "
                        "Gaussian pulses, FP32 storage"}


def run_gradient(args, local_rank):
    """Gradient of the pressure loss against a larger periodic reference
    with respect to the relaxation parameters on the D2Q37 512x256 FP32
    pulse with the mesoscopic viscous vector (alpha_V in play):
    --gradient-steps steps of the reverse-mode sweep (the checkpointed
    forward pass, then the backward pass that recomputes each 100-step
    segment and runs the adjoint kernels), timed with CUDA events on the
    solver's stream, beside the same number of ordinary steps of the same
    grid (L2-resident at this size, so neither is flushed).  The
    tangent-linear steps (three directions) are timed beside them."""
    import torch
    import paper_2307_16766_gb300 as lbm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    K = args.gradient_steps
    ck = 100
    cfg, f, rcfg, rf, (x0, y0) = W.gradient_pulse(steps=K)
    cfg = dict(cfg, viscous="meso", alpha_V=0.3)
    nx, ny = cfg["nx"], cfg["ny"]
    cs2 = W.CS2["D2Q37"]
    # reference pressure of the interior crop, every step
    ref = lbm.Simulation(rcfg, device=dev).init_fields(*rf)
    dP = torch.empty((K, ny, nx), dtype=torch.float64, device=dev)
    for k in range(K):
        ref.step(1)
        rho, _, _, T = ref.macros(device=True)
        dr = rho[y0:y0 + ny, x0:x0 + nx] - 1.0
        dT = T[y0:y0 + ny, x0:x0 + nx] - 1.0
        dP[k] = cs2 * (dr + dT + dr * dT)
    ref.close()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    # ordinary steps
    sim = lbm.Simulation(cfg, device=dev).init_fields(*f)
    sim.step(5)
    torch.cuda.synchronize(dev)
    ev[0].record(sim.stream)
    sim.step(K)
    ev[1].record(sim.stream)
    torch.cuda.synchronize(dev)
    fwd_s = ev[0].elapsed_time(ev[1]) / 1e3
    # reverse mode from the initial state: forward with checkpoints, backward
    sim.init_fields(*f)
    lbm.lbm_adj_begin(sim.handle, ck, K)
    torch.cuda.synchronize(dev)
    ev[0].record(sim.stream)
    J = lbm.lbm_adj_forward(sim.handle, K, dP.data_ptr(), ny * nx)
    ev[1].record(sim.stream)
    dJ = lbm.lbm_adj_backward(sim.handle)
    ev[2].record(sim.stream)
    torch.cuda.synchronize(dev)
    adj_f = ev[0].elapsed_time(ev[1]) / 1e3
    adj_b = ev[1].elapsed_time(ev[2]) / 1e3
    lbm.lbm_adj_end(sim.handle)
    # forward mode (tangent-linear), three directions, beside it
    sim.init_fields(*f)
    lbm.lbm_grad_begin(sim.handle)
    torch.cuda.synchronize(dev)
    ev[0].record(sim.stream)
    lbm.lbm_grad_step(sim.handle, K, dP.data_ptr(), ny * nx)
    ev[1].record(sim.stream)
    torch.cuda.synchronize(dev)
    tl_s = ev[0].elapsed_time(ev[1]) / 1e3
    Jt, dJt = lbm.lbm_grad_result(sim.handle)
    lbm.lbm_grad_end(sim.handle)
    sim.close()
    names = ("alpha_T", "beta_P", "P_inf", "alpha_V", "t_inf")
    return {"value": (adj_f + adj_b) / fwd_s, "unit": "gradient time / forward time (reverse mode, all parameters)",
            "steps": K, "checkpoint_every": ck,
            "forward_ms_per_step": fwd_s / K * 1e3,
            "adjoint_forward_ms_per_step": adj_f / K * 1e3, "adjoint_backward_ms_per_step": adj_b / K * 1e3,
            "J": J, "dJ": dict(zip(names, dJ)),
            "tangent": {"ratio": tl_s / fwd_s, "J": Jt, "dJ": {"alpha_T": dJt[0], "beta_P": dJt[1], "P_inf": dJt[2]},
                        "directions": 3},
            "mode": "reverse (adjoint) sweep, checkpoint every %d steps, recompute per segment" % ck,
            "workload": "D2Q37 %dx%d FP32 rho+T Gaussian pulse, CBC-RELAX on four sides, mesoscopic viscous "
                        "vector, alpha_T = beta_P = 0.5, alpha_V = 0.3, P_inf = c_s^2 rho0; loss against the "
                        "centre crop of a %dx%d periodic run, every step; gradient w.r.t. sigma (beta_P), beta "
                        "(alpha_T), alpha_V, P_inf (and t_inf)" % (nx, ny, rcfg["nx"], rcfg["ny"])}


def max_over_ranks(seconds, world):
    """The slowest rank's timed-region length (replicas run in lock step
    between the barriers; the job is as fast as its slowest GPU)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes, steps, world, seconds):
    """Lattice updates of all replicas per second / 1e6 (weak scaling)."""
    return nodes * steps * world / seconds / 1e6


def cpu_model():
    """The host CPU's name from /proc/cpuinfo (x86: model name; Arm: the
    implementer / part codes), else the machine type."""
    import platform
    info = {}
    try:
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                info.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if "model name" in info:
        return info["model name"]
    if "CPU part" in info:
        return "%s, CPU implementer %s part %s" % (platform.machine(), info.get("CPU implementer", "?"),
                                                   info["CPU part"])
    return platform.machine()


def _oracle_rate(cfg, fields, seconds):
    import oracle
    s = oracle.Sim(cfg).init(*fields)
    t = time.perf_counter()
    s.step(1)
    one = time.perf_counter() - t
    n = max(1, int(seconds / max(one, 1e-3)))
    t = time.perf_counter()
    s.step(n)
    dt = time.perf_counter() - t
    return cfg["nx"] * cfg["ny"] * n / dt / 1e6, n, dt


def cpu_baseline(cfg, fields, seconds=15.0, seconds_1t=6.0):
    """The FP64 oracle on this host: all threads (the baseline) and one
    thread, each on a bounded number of steps of the workload."""
    import oracle
    nproc = oracle.threads()
    mlups, n, dt = _oracle_rate(cfg, fields, seconds)
    oracle.set_threads(1)
    try:
        m1, n1, dt1 = _oracle_rate(cfg, fields, seconds_1t)
    finally:
        oracle.set_threads(nproc)
    return {"value": mlups, "unit": "MLUPS", "cores": nproc, "kind": "oracle",
            "cpu": cpu_model(), "single_thread_value": m1,
            "sample": "%d FP64 oracle steps of the %dx%d workload after one warm-up step (%.1f s) on %d "
                      "threads; %d steps (%.1f s) on 1 thread" % (n, cfg["nx"], cfg["ny"], dt, nproc, n1, dt1)}


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo" if args.impl == "reference" else "nccl")

    if args.impl == "reference":
        if rank == 0:
            cfg, fields = workload(args.nx, args.ny, "f64", args.steps)
            import oracle
            s = oracle.Sim(cfg).init(*fields)
            for _ in range(min(args.warmup, 1)):
                s.step(1)
            t = time.perf_counter()
            s.step(1)
            one = time.perf_counter() - t
            n = max(1, min(args.steps, int(120.0 / max(one, 1e-3))))
            t = time.perf_counter()
            s.step(n)
            dt = time.perf_counter() - t
            v = cfg["nx"] * cfg["ny"] * n / dt / 1e6
            line = {"metric": METRIC, "value": v, "unit": "MLUPS", "impl": "reference",
                    "n_gpus": args.gpus, "steps": n, "warmup": args.warmup,
                    "ms_per_step": dt / n * 1e3, "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                    "config": workload_config(cfg, {"l2": "n/a (CPU)"}),
                    "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(),
                                     "kind": "oracle", "cpu": cpu_model(),
                                     "sample": "%d of %d requested steps of the full grid" % (n, args.steps)},
                    "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                    "gpu_launches": 0}
            print(json.dumps(line))
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    res = run_gpu(args, rank, world, local_rank, args.storage, want_e2e=not args.no_e2e)
    fp64 = None
    if not args.no_fp64_leg and args.storage != "f64":
        a2 = argparse.Namespace(**vars(args))
        a2.steps = min(args.steps, 50)
        fp64 = run_gpu(a2, rank, world, local_rank, "f64", want_e2e=False)
    refl = None
    if not args.no_reference_leg and args.storage == "f32":
        a2 = argparse.Namespace(**vars(args))
        a2.steps = min(args.steps, 50)
        refl = run_gpu(a2, rank, world, local_rank, "f32", want_e2e=False, reference=True)
    fp16 = None
    if not args.no_fp16_leg and args.storage == "f32":
        a2 = argparse.Namespace(**vars(args))
        a2.steps = min(args.steps, 50)
        fp16 = run_gpu(a2, rank, world, local_rank, "f16", want_e2e=False)

    batch = None
    if not args.no_batch_leg and args.storage == "f32":
        batch = run_batch(args, local_rank)
    large = large_vortex = None
    if not args.no_large_leg and args.storage == "f32":
        large = run_large(args, local_rank)
        large_vortex = run_large(args, local_rank, kind="vortex")
    gradient = None
    if not args.no_gradient_leg and args.storage == "f32":
        gradient = run_gradient(args, local_rank)

    K = args.steps
    nodes = args.nx * args.ny
    step_s = max_over_ranks(res["step_ms_total"] / 1e3, world)
    value = whole_job_mlups(nodes, K, world, step_s)

    if rank == 0:
        peak, peak_kind = measured_peaks()
        Q, b = 37, BYTES_PER_VALUE[args.storage]
        # dominant kernel: the k_bulk launch, timed live on its own stream
        # while the band kernel runs beside it
        alg_bytes = 2 * Q * b * res["interior_nodes"]
        achieved = alg_bytes / (res["interior_ms_mean"] / 1e3) / 1e9
        traffic = bulk_traffic(args.storage, res["interior_nodes"])
        launches_per_step = 2            # bulk and band (inflow written once per buffer; no ZG sides)
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": res["step_ms_total"] / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "f64": "f64", "f16": "f16-storage/f32"}[args.storage],
            "data": "synthetic", "config": workload_config(res["cfg"]),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_bulk (stream+collide)", "peak_kind": peak_kind,
                         "bytes_per_launch": alg_bytes, "kernel_ms": res["interior_ms_mean"],
                         "band_overlapped_ms": res["boundary_overlapped_ms_mean"],
                         "phased_bulk_ms": res["bulk_ms_mean"],
                         "phased_boundary_ms": res["boundary_ms_mean"]},
            "e2e": res.get("e2e"),
            "gpu_launches": launches_per_step * K,
            "clocks": res["clocks"],
            "finite": res["finite"],
        }
        if fp64 is not None:
            line["fp64"] = {"value": nodes / (fp64["step_ms_total"] / 1e3 / min(K, 50)) / 1e6,
                            "unit": "MLUPS", "interior_ms": fp64["interior_ms_mean"],
                            "phased_bulk_ms": fp64["bulk_ms_mean"],
                            "phased_boundary_ms": fp64["boundary_ms_mean"],
                            "interior_GBps": 2 * Q * 8 * fp64["interior_nodes"] / (fp64["interior_ms_mean"] / 1e3) / 1e9,
                            "roofline": fp64_roofline(fp64["interior_nodes"], fp64["interior_ms_mean"])}
        if refl is not None:
            Kr = min(K, 50)
            line["reference_shift"] = {
                "value": nodes / (refl["step_ms_total"] / 1e3 / Kr) / 1e6, "unit": "MLUPS",
                "interior_ms": refl["interior_ms_mean"], "phased_bulk_ms": refl["bulk_ms_mean"],
                "phased_boundary_ms": refl["boundary_ms_mean"],
                "interior_GBps": 2 * Q * 4 * refl["interior_nodes"] / (refl["interior_ms_mean"] / 1e3) / 1e9,
                "what": "the same FP32 workload with the populations held relative to the stream's "
                        "equilibrium (u_ref = (U0, 0)): FP32 u error vs FP64 after 20000 steps 1.6e-7 "
                        "(plain shift 2.9e-5), tests/test_gpu_parity.py"}
        if fp16 is not None:
            line["fp16"] = {"value": nodes / (fp16["step_ms_total"] / 1e3 / min(K, 50)) / 1e6,
                            "unit": "MLUPS", "interior_ms": fp16["interior_ms_mean"],
                            "phased_bulk_ms": fp16["bulk_ms_mean"],
                            "phased_boundary_ms": fp16["boundary_ms_mean"],
                            "interior_GBps": 2 * Q * 2 * fp16["interior_nodes"] / (fp16["interior_ms_mean"] / 1e3) / 1e9,
                            "phased_bulk_GBps": 2 * Q * 2 * fp16["interior_nodes"] / (fp16["bulk_ms_mean"] / 1e3) / 1e9,
                            "storage": "shifted FP16 (g / w), FP32 arithmetic"}
        if batch is not None:
            line["batch"] = batch
        if large is not None:
            line["large"] = large
        if large_vortex is not None:
            line["large_vortex"] = large_vortex
        if gradient is not None:
            line["gradient"] = gradient
        if not args.no_cpu_baseline and world == 1:
            cfg, fields = workload(args.nx, args.ny, "f64", 1)
            line["cpu_baseline"] = cpu_baseline(cfg, fields)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
