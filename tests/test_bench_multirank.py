"""Multi-rank paths of bench.py on CPU (gloo, world size 2): the job's time
is the slowest rank's, its throughput the sum over replicas; the reference
arm under torchrun prints one line from rank 0 and exits 0 on every rank."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, seconds, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(seconds[rank], world)
    v = bench.whole_job_mlups(1000, 10, world, t)
    out.put((rank, t, v))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_throughput_gloo():
    world = 2
    seconds = [0.5, 2.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, seconds, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 2.0                          # the slowest rank's time on every rank
        assert v == pytest.approx(1000 * 10 * 2 / 2.0 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.whole_job_mlups(2000, 5, 1, 0.5) == pytest.approx(0.02)


def test_reference_arm_under_torchrun_two_ranks():
    """Rank 0 times the oracle and prints one JSON line; rank 1 exits 0."""
    import oracle
    oracle.lib()                     # build the oracle once, before two ranks need it
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--nx", "96", "--ny", "64"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
