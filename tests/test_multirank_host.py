"""The N > 1 launch path of bench.py on CPU: two gloo ranks exercise its
rendezvous, barrier and the max / sum reductions that turn per-rank step
times and byte counts into the whole-job line, and the reference arm's
rank-0-only rule (the other ranks exit without work)."""

import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    class A:
        gpus = world
    w, r, _ = bench.dist_setup(A())
    bench.barrier(w)
    mx = bench.max_over_ranks(w, 10.0 + r)       # per-rank step time -> the slowest rank
    sm = bench.sum_over_ranks(w, 1e9 * (r + 1))  # per-rank bytes -> whole-job bytes
    q.put((r, w, mx, sm))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert all(g[2] == 11.0 for g in got)
    assert all(g[3] == 3e9 for g in got)


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun with two ranks the reference arm prints one JSON line
    (rank 0) and every rank exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--rows", "4096", "--cols", "64",
           "--sketch-rows", "32", "--target-rank", "8", "--cpu-sample-cols", "16"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    import json
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
