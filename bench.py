#!/usr/bin/env python
"""Benchmark of the block-SRHT hot path on GB300.

One step = the whole hot path over one batch of synthetic input: the block
SRHT sketch B = Omega A (Sec. 2) followed by the rank-k randomized SVD of
Algorithm 1 (Sec. 3.1) on the tall-skinny workload n = 2^20, m = 4096,
A = G1 diag(i^-2) G2^T + 1e-4 N in FP32, p = 4 blocks, l = 512, k = 100.

Prints ONE JSON line (rank 0). ``value`` is the whole-step throughput in
GB/s of A: (n * m * sizeof(A)) / step time; the sketch kernel's own HBM
throughput and the per-stage times are reported beside it. A (16 GiB) is far
larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own replica on its own GPU (weak
scaling, no collective on the data path); the step time is the max over ranks.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "tall-skinny lowrank+noise n=2^20 m=4096 fp32 p=4 l=512 rank-100 rSVD"
METRIC = "ΩA sketch HBM GB/s (% peak); rSVD/Nyström time at stated error; p50/p99 latency"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    # Long aliases: under torchrun, options that prefix one of its own
    # (--n: --nnodes, --nproc-per-node) are taken as ambiguous by its parser.
    ap.add_argument("--n", "--rows", dest="n", type=int, default=1 << 20)
    ap.add_argument("--m", "--cols", dest="m", type=int, default=4096)
    ap.add_argument("--p", "--blocks", dest="p", type=int, default=4)
    ap.add_argument("--l", "--sketch-rows", dest="l", type=int, default=512)
    ap.add_argument("--k", "--target-rank", dest="k", type=int, default=100)
    ap.add_argument("--dtype", choices=["f32", "f64", "bf16", "f16"], default="f32")
    ap.add_argument("--mode", choices=["full", "sketch", "serve", "nystrom"], default="full",
                    help="full = sketch + rSVD (the benchmark step); sketch = sketch only; "
                         "serve = the mixed request stream through the serving loop; "
                         "nystrom = Algorithm 2 on the RBF kernel workload (n = --rows points)")
    ap.add_argument("--nystrom-ks", default="100,200,400", help="target ranks of the nystrom mode")
    ap.add_argument("--serve-requests", type=int, default=600,
                    help="requests of the serving stream (serve mode)")
    ap.add_argument("--serve-compare", type=int, default=120,
                    help="requests of the reduced stream timed on both the served path and the plain "
                         "FP64 one-at-a-time path (serve mode)")
    ap.add_argument("--serve-points", default="0.5,0.8,1.0",
                    help="serve mode: loads (fractions of the saturation throughput) of the Poisson runs")
    ap.add_argument("--serve-sat-requests", type=int, default=0,
                    help="serve mode: measure the saturation throughput on this many leading requests "
                         "(0: the whole stream)")
    ap.add_argument("--serve-window", type=int, default=96,
                    help="most requests in flight at once (client side, serve mode)")
    ap.add_argument("--variant", choices=["auto", "cudacore", "tensor", "gaussian"], default="auto",
                    help="sketch kernel: library choice, CUDA-core butterflies (K1), tensor cores (K2, 16-bit A), "
                         "or the Gaussian-embedding comparator of Sec. 4 (FP32)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the metric's other parts (FP64 sketch, small FP64 workload, 16-bit workload, "
                         "stated rSVD error, Nystrom, serving summary)")
    ap.add_argument("--serve-summary-requests", type=int, default=120)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-cols", type=int, default=64)
    ap.add_argument("--cpu-sample-rows", type=int, default=1 << 14)
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def torch_dtype(name):
    import torch
    return {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16, "f16": torch.float16}[name]


def make_input(args, rank):
    """The tall-skinny workload in the storage type of --dtype; the generator
    converts each row panel (no full-size FP32 temporary for 16-bit A)."""
    import synth
    dt = torch_dtype(args.dtype)
    return synth.lowrank_noise_device(args.n, args.m, seed=1236 + rank, dtype=dt)


# --------------------------------------------------------------- CPU oracle
def _oracle_sample(args):
    """The oracle's bounded sample of the workload and its step.

    full mode: Algorithm 1 as the oracle states it (dense-Omega sketch, LAPACK
    QR and SVD) on the first n_s rows of the same generator (n_s = min(n,
    2^14) by default), GB/s of those rows; every stage but the l x l SVD
    grows linearly with the rows, so this slightly flatters nothing but the
    oracle's fixed costs.  sketch mode: the dense-Omega sketch of an
    n x cols column slice (the sketch is column-separable)."""
    import numpy as np
    from oracle import bsrht as orc
    from oracle import lowrank as orl
    import synth

    elem = {"f32": 4, "f64": 8, "bf16": 2, "f16": 2}[args.dtype]
    if args.mode == "sketch":
        cols = args.cpu_sample_cols
        a = synth.lowrank_noise(args.n, cols, rank=min(1000, cols), seed=77).astype(np.float32)
        step = lambda s: orc.sketch_dense(a, args.p, args.l, seed=s)  # noqa: E731
        return step, args.n * cols * elem, (f"dense-Omega oracle sketch of an n={args.n} x {cols}-column slice "
                                            f"(p={args.p}, l={args.l}); GB/s of A")
    ns = min(args.n, args.cpu_sample_rows)
    a = synth.lowrank_noise(ns, args.m, rank=min(1000, args.m), seed=77).astype(np.float32).astype(np.float64)
    l = min(args.l, args.m, ns)
    k = min(args.k, l)
    step = lambda s: orl.rsvd(a, k, l, args.p, s)  # noqa: E731
    return step, ns * args.m * elem, (f"oracle Algorithm 1 (dense-Omega sketch + LAPACK QR/SVD, FP64) on "
                                      f"n={ns} x m={args.m} rows of the workload generator (p={args.p}, l={l}, "
                                      f"k={k}); GB/s of A rows")


def cpu_baseline(args, seconds_target=15.0):
    """The CPU oracle on a bounded sample of the same workload, in GB/s of A."""
    step, nbytes, sample = _oracle_sample(args)
    t0 = time.perf_counter()
    reps = 0
    while True:
        step(reps)
        reps += 1
        if time.perf_counter() - t0 > seconds_target or reps >= 3:
            break
    dt = (time.perf_counter() - t0) / reps
    gbs = nbytes / dt / 1e9
    return {"value": round(gbs, 4), "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{sample}; {reps} rep(s), {dt:.2f} s each"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    step, nbytes, sample = _oracle_sample(args)
    for w in range(args.warmup):
        step(w)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        step(s)
        times.append(time.perf_counter() - t0)
    dt = statistics.mean(times)
    gbs = nbytes / dt / 1e9
    workload = WORKLOAD if (args.mode == "full" and args.dtype == "f32" and args.n == 1 << 20 and args.m == 4096) \
        else f"n={args.n} m={args.m} {args.dtype} p={args.p} l={args.l} k={args.k} mode={args.mode}"
    line = {"metric": METRIC, "value": round(gbs, 4), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "sample": sample}, "impl": "reference",
            "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- our arm
# DRAM traffic of the dominant sketch kernel, one launch at the benchmark
# shape: dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture
# at n = 2^18 (the full-size capture would exceed the profiler's size
# limits), scaled to n = 2^20 by the rows processed (reads grow with n, the
# partial-sum writes do not).  Each record holds the SHA-256 of the kernel
# sources it was taken on; once those files change the record no longer
# describes the kernel and the line reports null (profiles/ holds the
# capture, its command and the hash).
TRAFFIC_RECORDS = {
    # FP32: the reads are A itself; the writes are the per-(CTA, panel)
    # partial sums, written once (they do not grow with n).
    ("f32", 1 << 20, 4096, 4, 512): {
        "kernel": "k_sketch_tma", "read_n2e18": 4295577600, "write_n2e18": 10937344, "write_scales": False,
        "sources": ("paper_2210_11295_gb300/csrc/sketch_tma.cu", "paper_2210_11295_gb300/csrc/tma.cuh",
                    "paper_2210_11295_gb300/csrc/f32x2.cuh", "paper_2210_11295_gb300/csrc/tmem.cuh"),
        "sha256": "ca6860d416ec01d8c929f0487f7bd6c01e8f56c165772ffdb2198846db92a4b4"},
    # FP64: besides A, the read-modify-write of the FP64 partial sums at
    # every flush of the integer sums (one per 32 chunks of a CTA), which
    # grows with n like the reads.
    ("f64", 1 << 20, 4096, 4, 512): {
        "kernel": "k_sketch_f64x", "read_n2e18": 8838070016, "write_n2e18": 266583552, "write_scales": True,
        "sources": ("paper_2210_11295_gb300/csrc/sketch_f64x.cu", "paper_2210_11295_gb300/csrc/tma.cuh"),
        "sha256": "13dd167a62728e7de4f5dafe612557852b4d179c5eab3a41148373abf2378615"},
}


def _sources_sha(paths):
    """SHA-256 of the files concatenated (what cat a b | sha256sum prints)."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def sketch_traffic(dtype, n, m, p, l, variant="auto"):
    """Recorded DRAM bytes of one launch of the dominant sketch kernel, or
    None (no record for this shape, or the kernel changed since)."""
    rec = TRAFFIC_RECORDS.get((dtype, n, m, p, l))
    if variant != "auto" or rec is None:
        return None
    if _sources_sha(rec["sources"]) != rec["sha256"]:
        return None
    return 4 * rec["read_n2e18"] + (4 if rec["write_scales"] else 1) * rec["write_n2e18"]


def gaussian_comparator(args, lib, a, sketch_ms, step_ms, mode, stream):
    """Times the Gaussian embedding (BSRHT_VARIANT_GAUSSIAN: Omega_G with
    N(0, 1/l) entries, B = Omega_G A on the tensor cores, 2 l n m flops) on
    the same A as the block SRHT sketch, and in full mode one rSVD with it.
    Sec. 4 of the paper reports the same approximation quality and a block
    SRHT up to 2.5x faster to apply (on CPU clusters); the quality side is in
    tests/test_gpu_gaussian.py."""
    import torch

    n, m = a.shape
    p, l, k = args.p, args.l, args.k
    g = lib.VARIANT_GAUSSIAN
    ws = torch.empty(max(lib.bsrht_sketch_workspace(n, m, p, l, a.dtype, variant=g), 1), dtype=torch.uint8,
                     device=a.device)
    out = torch.empty(l, m, device=a.device, dtype=torch.float32)
    lib.bsrht_sketch(a, p, l, 0, out=out, workspace=ws, variant=g)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    for i, (e0, e1) in enumerate(ev):
        e0.record(stream)
        lib.bsrht_sketch(a, p, l, 1 + i, out=out, workspace=ws, variant=g)
        e1.record(stream)
    torch.cuda.synchronize()
    g_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
    del ws, out
    res = {"kind": "Gaussian embedding (Sec. 4): Omega_G l x n with N(0, 1/l) entries (Philox, Box-Muller), "
                   "B = Omega_G A on tcgen05 (3xTF32, FP32 accuracy)",
           "sketch_ms": round(g_ms, 3), "bsrht_sketch_ms": round(sketch_ms, 3),
           "bsrht_speedup": round(g_ms / sketch_ms, 2),
           "gaussian_tflops": round(2.0 * l * n * m / (g_ms * 1e-3) / 1e12, 1)}
    if mode == "full":
        rws = torch.empty(max(lib.bsrht_rsvd_workspace(n, m, k, l, p, a.dtype, variant=g), 1), dtype=torch.uint8,
                          device=a.device)
        u = torch.empty(n, k, device=a.device, dtype=torch.float64)
        s = torch.empty(k, device=a.device, dtype=torch.float64)
        v = torch.empty(m, k, device=a.device, dtype=torch.float64)
        lib.bsrht_rsvd(a, k, l, p, 0, variant=g, workspace=rws, outs=(u, s, v))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lib.bsrht_rsvd(a, k, l, p, 1, variant=g, workspace=rws, outs=(u, s, v))
        e1.record(stream)
        torch.cuda.synchronize()
        res["rsvd_ms"] = round(e0.elapsed_time(e1), 3)
        res["bsrht_rsvd_ms"] = round(step_ms, 3)
        del rws, u, s, v
    torch.cuda.empty_cache()
    return res


def single_view_rsvd(args, lib, a, stream):
    """One bsrht_srsvd call (Algorithm 3, s = 2 l) on the benchmark's A after
    a warm-up call: time (CUDA events) and stage times."""
    import torch

    n, m = a.shape
    k, l, p = args.k, args.l, args.p
    s = min(2 * l, m, n)
    ws = torch.empty(max(lib.bsrht_srsvd_workspace(n, m, k, l, s, p, a.dtype), 1), dtype=torch.uint8, device=a.device)
    outs = (torch.empty(n, k, device=a.device, dtype=torch.float64), torch.empty(k, device=a.device, dtype=torch.float64),
            torch.empty(m, k, device=a.device, dtype=torch.float64))
    lib.bsrht_srsvd(a, k, l, s, p, 0, workspace=ws, outs=outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lib.bsrht_srsvd(a, k, l, s, p, 1, workspace=ws, outs=outs)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lib.bsrht_profile_enable(True)
    lib.bsrht_srsvd(a, k, l, s, p, 2, workspace=ws, outs=outs)
    torch.cuda.synchronize()
    stages = {}
    for name, t in lib.bsrht_profile_stages():  # stage names repeat (several sketches): sum them
        stages[name] = round(stages.get(name, 0.0) + t, 3)
    lib.bsrht_profile_enable(False)
    del ws, outs
    torch.cuda.empty_cache()
    return {"kind": "Algorithm 3 (single view): Omega, Phi, Psi block SRHTs, Gamma Gaussian, s = 2 l", "s": s,
            "ms": round(ms, 3), "stages_ms": stages}


# --------------------------------------------------------------- metric extras
# The rest of the benchmark's metric, measured after the timed steps on rank
# 0: the FP64 sketch (the paper's arithmetic), the small FP64 workload, the
# 16-bit workload with its per-dtype errors, the stated error of the rSVD,
# the kernel-matrix Nystrom workload and a short serving stream.  Each part
# reports its own CUDA-event times; the oracle is used only for the stated
# errors.
def _events_ms(stream, fn, reps):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)


def _kernel_ms(lib, fn, reps):
    """Mean of the library's own CUDA-event time of the sketch kernel."""
    lib.bsrht_profile_enable(True)
    ks = []
    for _ in range(reps):
        fn()
        st = dict(lib.bsrht_profile_stages())
        if "sketch_kernel" in st:
            ks.append(st["sketch_kernel"])
    lib.bsrht_profile_enable(False)
    return statistics.mean(ks) if ks else None


def _rel(a, b):
    import numpy as np
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def f64_sketch_object(lib, a32, p, l, peak, stream):
    """The sketch in FP64 at the full tall-skinny shape: the FP32 workload
    plus an FP64 perturbation of 1e-7 (full 53-bit significands)."""
    import numpy as np
    import torch
    from oracle import bsrht as orc
    n, m = a32.shape
    a = torch.empty(n, m, device=a32.device, dtype=torch.float64)
    gen = torch.Generator(device=a32.device)
    gen.manual_seed(1250)
    for r0 in range(0, n, 1 << 16):
        r1 = min(n, r0 + (1 << 16))
        a[r0:r1] = a32[r0:r1].double() + 1e-7 * torch.randn(r1 - r0, m, device=a32.device, dtype=torch.float64,
                                                             generator=gen)
    out = torch.empty(l, m, device=a.device, dtype=torch.float64)
    ws = torch.empty(max(lib.bsrht_sketch_workspace(n, m, p, l, torch.float64), 1), dtype=torch.uint8, device=a.device)
    run = lambda s: lib.bsrht_sketch(a, p, l, s, out=out, workspace=ws)  # noqa: E731
    for w in range(3):
        run(w)
    call_ms = _events_ms(stream, lambda: run(7), 5)
    k_ms = _kernel_ms(lib, lambda: run(8), 5) or call_ms
    run(9)
    torch.cuda.synchronize()
    cols = [0, 1, 15, 16, 1000, 2047, m - 16, m - 1]
    got = out[:, cols].cpu().numpy()
    ref = orc.sketch_fast(a[:, cols].cpu().numpy(), p, l, 9)
    nbytes = n * m * 8 + l * m * 8
    ach = nbytes / (k_ms * 1e-3) / 1e9
    del out, ws
    torch.cuda.empty_cache()
    # The whole rank-100 Algorithm 1 in FP64 on the same matrix: one warm-up
    # call, one timed call with its stages (the tall products run on the
    # FP64 units, 1.25 TFLOP/s nominal on this GPU).
    k = 100
    rws = torch.empty(max(lib.bsrht_rsvd_workspace(n, m, k, l, p, torch.float64), 1), dtype=torch.uint8,
                      device=a.device)
    outs = (torch.empty(n, k, device=a.device, dtype=torch.float64),
            torch.empty(k, device=a.device, dtype=torch.float64),
            torch.empty(m, k, device=a.device, dtype=torch.float64))
    lib.bsrht_rsvd(a, k, l, p, 0, workspace=rws, outs=outs)
    lib.bsrht_profile_enable(True)
    rs_ms = _events_ms(stream, lambda: lib.bsrht_rsvd(a, k, l, p, 1, workspace=rws, outs=outs), 1)
    rs_st = {name: round(v, 2) for name, v in lib.bsrht_profile_stages()}
    lib.bsrht_profile_enable(False)
    rs_s1 = float(outs[1][0].item())
    del a, rws, outs
    torch.cuda.empty_cache()
    return {"workload": f"tall-skinny lowrank+noise n={n} m={m} f64 p={p} l={l} (sketch)", "dtype": "f64",
            "kernel": "k_sketch_f64x (exact 64-bit integer Walsh-Hadamard transform, TMA-fed)",
            "ms": round(call_ms, 4), "kernel_ms": round(k_ms, 4), "gbs": round(nbytes / (call_ms * 1e-3) / 1e9, 2),
            "roofline": {"bound": "hbm", "achieved": round(ach, 2), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 4), "traffic": sketch_traffic("f64", n, m, p, l)},
            "parity": {"columns": cols, "rel_fro_vs_oracle": float(f"{_rel(got, ref):.3e}"), "tol": 1e-12},
            "rsvd_fp64": {"k": k, "ms": round(rs_ms, 1), "sigma_1": rs_s1, "stages_ms": rs_st,
                          "note": "tall products A Q and the tall QR on the FP64 units"}}


def p_sweep_object(lib, a, l, k, peak, stream):
    """The tall-skinny FP32 workload at p = 1, 4, 16, 64 blocks (the block
    count of eq. 2.3; r = n / p rows per Walsh-Hadamard transform): sketch
    call and kernel time with their HBM fraction, and the rank-k Algorithm 1
    step time, on the same resident A."""
    import torch
    n, m = a.shape
    rows = []
    for p in (1, 4, 16, 64):
        out = torch.empty(l, m, device=a.device, dtype=torch.float32)
        ws = torch.empty(max(lib.bsrht_sketch_workspace(n, m, p, l, a.dtype), 1), dtype=torch.uint8,
                         device=a.device)
        run = lambda s: lib.bsrht_sketch(a, p, l, s, out=out, workspace=ws)  # noqa: E731
        for w in range(3):
            run(w)
        call_ms = _events_ms(stream, lambda: run(7), 5)
        k_ms = _kernel_ms(lib, lambda: run(8), 5) or call_ms
        rws = torch.empty(max(lib.bsrht_rsvd_workspace(n, m, k, l, p, a.dtype), 1), dtype=torch.uint8,
                          device=a.device)
        outs = (torch.empty(n, k, device=a.device, dtype=torch.float64),
                torch.empty(k, device=a.device, dtype=torch.float64),
                torch.empty(m, k, device=a.device, dtype=torch.float64))
        rs = lambda s: lib.bsrht_rsvd(a, k, l, p, s, workspace=rws, outs=outs)  # noqa: E731
        rs(0)
        rsvd_ms = _events_ms(stream, lambda: rs(1), 2)
        nbytes = n * m * 4 + l * m * 4
        rows.append({"p": p, "sketch_ms": round(call_ms, 4), "kernel_ms": round(k_ms, 4),
                     "gbs": round(nbytes / (call_ms * 1e-3) / 1e9, 2),
                     "kernel_frac_of_measured_peak": round(nbytes / (k_ms * 1e-3) / 1e9 / peak, 4),
                     "rsvd_ms": round(rsvd_ms, 3)})
        del out, ws, rws, outs
        torch.cuda.empty_cache()
    return {"workload": f"tall-skinny lowrank+noise n={n} m={m} fp32 l={l} k={k}, p in 1, 4, 16, 64", "per_p": rows}


def config1_object(lib, stream):
    """The small FP64 workload: A = U diag(e^(-i/10)) V^T, n = 4096, m = 256,
    p = 4, l = 128, rank-20 Algorithm 1, against the oracle."""
    import numpy as np
    import torch
    import synth
    from oracle import lowrank as orl
    a_np, _ = synth.haar_spectrum(4096, 256, seed=1235)
    a = torch.from_numpy(a_np).cuda()
    k, l, p = 20, 128, 4
    for _ in range(3):
        lib.bsrht_rsvd(a, k, l, p, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 10
    for _ in range(reps):
        u, s, v = lib.bsrht_rsvd(a, k, l, p, 0)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / reps
    ur, sr, vr = orl.rsvd(a_np, k, l, p, 0)
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    approx, ref = (u * s) @ v.T, (ur * sr) @ vr.T
    return {"workload": "haar spectrum n=4096 m=256 f64 p=4 l=128 k=20 seed 0", "ms_per_call": round(ms, 3),
            "usvt_rel_err_vs_oracle": float(f"{_rel(approx, ref):.3e}"),
            "sigma_max_rel_err_vs_oracle": float(f"{np.max(np.abs(s - sr)) / sr[0]:.3e}"), "tol": 1e-12,
            "timing": "host wall clock per call (the call synchronizes on its status)"}


def config3_object(lib, peak, stream, sample_rows=1 << 15):
    """The 16-bit workload: n = 2^20, m = 8192 in BF16 and FP16 (FP32
    arithmetic), p = 8, l = 1024, rank 200: sketch with the CUDA-core (K1)
    and tensor-core (K2) kernels, one Algorithm 1 call (BF16), and on an
    n = 2^15 sample of the same generator the errors against the FP64 oracle
    -- on the same stored values (arithmetic error) and, for Omega A,
    against the FP32 source before rounding to 16 bits (storage included)."""
    import numpy as np
    import torch
    import synth
    from oracle import bsrht as orc
    from oracle import lowrank as orl
    n, m, p, l, k = 1 << 20, 8192, 8, 1024, 200
    res = {"workload": f"tall-skinny lowrank+noise n={n} m={m} p={p} l={l} k={k}, 16-bit storage"}
    for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        a = synth.lowrank_noise_device(n, m, seed=1237, dtype=dt)
        out = torch.empty(l, m, device=a.device, dtype=torch.float32)
        d = {}
        for vname, var in (("k1_cudacore", lib.VARIANT_AUTO), ("k2_tensor", lib.VARIANT_TENSOR)):
            ws = torch.empty(max(lib.bsrht_sketch_workspace(n, m, p, l, dt, variant=var), 1), dtype=torch.uint8,
                             device=a.device)
            run = lambda s: lib.bsrht_sketch(a, p, l, s, out=out, workspace=ws, variant=var)  # noqa: E731
            for w in range(2):
                run(w)
            call_ms = _events_ms(stream, lambda: run(5), 3)
            k_ms = _kernel_ms(lib, lambda: run(6), 3) or call_ms
            ach = (n * m * 2 + l * m * 4) / (k_ms * 1e-3) / 1e9
            d[vname] = {"ms": round(call_ms, 3), "kernel_ms": round(k_ms, 3), "gbs": round(ach, 1),
                        "frac_of_measured_peak": round(ach / peak, 4)}
            del ws
        if name == "bf16":
            rws = torch.empty(lib.bsrht_rsvd_workspace(n, m, k, l, p, dt), dtype=torch.uint8, device=a.device)
            outs = (torch.empty(n, k, device=a.device, dtype=torch.float64),
                    torch.empty(k, device=a.device, dtype=torch.float64),
                    torch.empty(m, k, device=a.device, dtype=torch.float64))
            lib.bsrht_rsvd(a, k, l, p, 0, workspace=rws, outs=outs)
            d["rsvd_ms"] = round(_events_ms(stream, lambda: lib.bsrht_rsvd(a, k, l, p, 1, workspace=rws, outs=outs),
                                            1), 3)
            del rws, outs
        del a, out
        torch.cuda.empty_cache()
        # Errors on the sample.
        a32 = synth.lowrank_noise_device(sample_rows, m, seed=1237, dtype=torch.float32)
        a_s = a32.to(dt)
        b = lib.bsrht_sketch(a_s, p, l, 1)
        u, s, v = lib.bsrht_rsvd(a_s, k, l, p, 1)
        torch.cuda.synchronize()
        a64 = a_s.double().cpu().numpy()
        src = a32.double().cpu().numpy()
        b = b.double().cpu().numpy()
        u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
        ur, sr, vr = orl.rsvd(a64, k, l, p, 1)
        e = float(np.linalg.norm(a64 - (u * s) @ v.T))
        e_ref = float(np.linalg.norm(a64 - (ur * sr) @ vr.T))
        d["errors_on_sample"] = {
            "rows": sample_rows,
            "sketch_rel_fro_vs_fp64_oracle_same_values": float(f"{_rel(b, orc.sketch_fast(a64, p, l, 1)):.3e}"),
            "sketch_rel_fro_vs_fp64_oracle_fp32_source": float(f"{_rel(b, orc.sketch_fast(src, p, l, 1)):.3e}"),
            "rank200_residual_rel_diff_vs_oracle": float(f"{abs(e - e_ref) / e_ref:.3e}"),
            "rank200_residual_rel": float(f"{e / np.linalg.norm(a64):.4e}"),
            "sigma_max_rel_err_vs_oracle": float(f"{np.max(np.abs(s - sr)) / sr[0]:.3e}")}
        del a32, a_s
        torch.cuda.empty_cache()
        res[name] = d
    return res


def rsvd_error_object(lib, a, u, s, v, args, sample_rows=1 << 16):
    """The stated error of the benchmark's rank-k approximation.  Full size:
    ||A V - U S||_F / ||S|| (zero in exact arithmetic for Algorithm 1) and the
    orthogonality of U and V.  On an n = 2^16 sample of the generator: the
    oracle's Algorithm 1, the Eckart-Young optimum ||A - [[A]]_k||_F
    (eigenvalues of A^T A on the GPU, in FP64) and sigma_{k+1}."""
    import numpy as np
    import torch
    import synth
    from oracle import lowrank as orl
    n, m = a.shape
    k, l, p = args.k, args.l, args.p
    av = torch.cat([(a[i:i + 65536].double() @ v) for i in range(0, n, 65536)])
    full = {"av_minus_us_rel": float(f"{(torch.linalg.norm(av - u * s) / torch.linalg.norm(s)).item():.3e}"),
            "u_orth": float(f"{torch.linalg.norm(u.T @ u - torch.eye(k, device=u.device, dtype=u.dtype)).item():.3e}"),
            "v_orth": float(f"{torch.linalg.norm(v.T @ v - torch.eye(k, device=v.device, dtype=v.dtype)).item():.3e}")}
    del av
    a_s = synth.lowrank_noise_device(sample_rows, m, seed=1236, dtype=torch.float32)
    us, ss, vs = lib.bsrht_rsvd(a_s, k, l, p, 0)
    gram = a_s.double().T @ a_s.double()
    sig = torch.sqrt(torch.clamp(torch.linalg.eigvalsh(gram), min=0.0)).flip(0).cpu().numpy()
    a64 = a_s.double().cpu().numpy()
    us, ss, vs = us.cpu().numpy(), ss.cpu().numpy(), vs.cpu().numpy()
    ur, sr, vr = orl.rsvd(a64, k, l, p, 0)
    e = float(np.linalg.norm(a64 - (us * ss) @ vs.T))
    e_ref = float(np.linalg.norm(a64 - (ur * sr) @ vr.T))
    opt = orl.best_rank_k_errors(sig, k)
    del a_s, gram
    torch.cuda.empty_cache()
    return {"full_size": full,
            "sample": {"rows": sample_rows, "residual_fro": float(f"{e:.6e}"), "oracle_residual_fro": float(f"{e_ref:.6e}"),
                       "rel_diff_vs_oracle": float(f"{abs(e - e_ref) / e_ref:.3e}"),
                       "sigma_max_rel_err_vs_oracle": float(f"{np.max(np.abs(ss - sr)) / sr[0]:.3e}"),
                       "eckart_young_fro": float(f"{opt['fro']:.6e}"), "ratio_to_optimum": round(e / opt["fro"], 5),
                       "sigma_k_plus_1": float(f"{opt['spectral']:.6e}")}}


def nystrom_object(lib, peak, stream, n=65536, p=8, l=600, ks=(100, 200, 400), sub=4096):
    """The kernel-matrix workload: A_ij = exp(-|xi - xj|^2 / (2 h^2)),
    x_i ~ U[0,1]^784, h the median pairwise distance, n = 65536 (FP32),
    p = 8, l = 600.  Per k: time of Algorithm 2 and the trace error
    tr(A) - sum(Lambda) (exact: the residual is PSD).  On the 4096-point
    subsample: the same against the oracle and the optimum sum_{i>k} lambda_i."""
    import numpy as np
    import torch
    import synth
    from oracle import lowrank as orl
    x = synth.rbf_points(n, 784, seed=1238)
    h = synth.rbf_bandwidth(x)
    xd = torch.from_numpy(x).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a = synth.rbf_kernel_device(xd, h, dtype=torch.float32)
    torch.cuda.synchronize()
    gen_ms = (time.perf_counter() - t0) * 1e3
    tr = float(torch.trace(a.double()).item())
    per_k = []
    for k in ks:
        ws = torch.empty(lib.bsrht_nystrom_workspace(n, k, l, p, torch.float32), dtype=torch.uint8, device="cuda")
        outs = (torch.empty(n, k, device="cuda", dtype=torch.float64), torch.empty(k, device="cuda", dtype=torch.float64))
        lib.bsrht_nystrom(a, k, l, p, 0, workspace=ws, outs=outs)
        ms = _events_ms(stream, lambda: lib.bsrht_nystrom(a, k, l, p, 1, workspace=ws, outs=outs), 3)
        lam = outs[1]
        per_k.append({"k": k, "ms": round(ms, 3), "trace_error_rel": float(f"{(tr - float(lam.sum())) / tr:.5e}")})
        del ws, outs
    out = torch.empty(l, n, device="cuda", dtype=torch.float32)
    sws = torch.empty(max(lib.bsrht_sketch_workspace(n, n, p, l, torch.float32), 1), dtype=torch.uint8, device="cuda")
    lib.bsrht_sketch(a, p, l, 0, out=out, workspace=sws)
    sk_ms = _events_ms(stream, lambda: lib.bsrht_sketch(a, p, l, 1, out=out, workspace=sws), 3)
    del a, out, sws
    torch.cuda.empty_cache()
    # Matrix-free: A formed a column panel at a time from the points and
    # sketched right away (bsrht_nystrom_rbf), k = ks[0].
    k0 = ks[0]
    fws = torch.empty(lib.bsrht_nystrom_rbf_workspace(n, 784, k0, l, p), dtype=torch.uint8, device="cuda")
    fouts = (torch.empty(n, k0, device="cuda", dtype=torch.float64), torch.empty(k0, device="cuda", dtype=torch.float64))
    lib.bsrht_nystrom_rbf(xd, h, k0, l, p, 0, workspace=fws, outs=fouts)
    mf_ms = _events_ms(stream, lambda: lib.bsrht_nystrom_rbf(xd, h, k0, l, p, 1, workspace=fws, outs=fouts), 3)
    matrix_free = {"k": k0, "ms": round(mf_ms, 3),
                   "trace_error_rel": float(f"{(tr - float(fouts[1].sum())) / tr:.5e}"),
                   "scratch_gb": round(fws.numel() / 1e9, 2), "stored_matrix_gb": round(n * n * 4 / 1e9, 2),
                   "stored_path_ms": per_k[0]["ms"], "generate_stored_matrix_ms": round(gen_ms, 1),
                   "note": "the stored path needs the n x n matrix formed first (generate_stored_matrix_ms, "
                           "torch); the matrix-free path forms it panel by panel inside the call"}
    del fws, fouts, xd
    torch.cuda.empty_cache()
    # The subsample against the oracle (FP32 arithmetic threshold on both sides).
    idx = np.sort(np.random.default_rng(1239).choice(n, size=sub, replace=False))
    a_sub = synth.rbf_kernel(x[idx], h).astype(np.float32)
    lam_all = np.linalg.eigvalsh(a_sub.astype(np.float64))[::-1]
    tr_s = float(np.trace(a_sub.astype(np.float64)))
    sub_rows = []
    for k in ks:
        _, lam_d = lib.bsrht_nystrom(torch.from_numpy(a_sub).cuda(), k, l, p, 0)
        torch.cuda.synchronize()
        _, lam_o, _ = orl.nystrom(a_sub.astype(np.float64), k, l, p, 0, unit_roundoff=2.0 ** -23)
        sub_rows.append({"k": k, "trace_error_rel": float(f"{(tr_s - float(lam_d.sum())) / tr_s:.5e}"),
                         "oracle_trace_error_rel": float(f"{(tr_s - float(lam_o.sum())) / tr_s:.5e}"),
                         "optimum_rel": float(f"{float(np.sum(lam_all[k:])) / tr_s:.5e}")})
    gbs = (n * n * 4 + l * n * 4) / (sk_ms * 1e-3) / 1e9
    return {"workload": f"RBF kernel n={n} (x ~ U[0,1]^784, median bandwidth h={h:.4f}) fp32 p={p} l={l}",
            "per_k": per_k, "sketch": {"ms": round(sk_ms, 3), "gbs": round(gbs, 1), "frac_of_measured_peak": round(gbs / peak, 4)},
            "matrix_free": matrix_free,
            "subsample": {"points": sub, "per_k": sub_rows}}


def serve_object(lib, requests=120, compare=40):
    """A short config-5 stream through the serving loop (the serve mode runs
    the long one): saturation throughput, Poisson arrivals at 0.5x of it
    with p50 / p99 latency, and a reduced stream (n <= 2^17, m <= 1024)
    served from FP32 storage against the plain FP64 one-request-at-a-time
    path: with Nystrom in FP64 arithmetic (equal accuracy) and, for
    comparison, in FP32 arithmetic."""
    import numpy as np
    import torch
    import synth
    reqs = synth.request_stream(requests, seed=1240, rate_hz=1.0)
    rng = np.random.default_rng(1242)
    dtypes = [torch.bfloat16 if rng.random() < 0.5 and r["kind"] != "nystrom" else torch.float32 for r in reqs]
    inputs = _ServeInputs()
    kw = dict(hbm_budget=24 << 30, executors=4, max_group=16)
    _serve_run(lib, inputs, reqs[:20], dtypes, math.inf, 96, **kw)
    sat_s, lat_sat, st_sat, _ = _serve_run(lib, inputs, reqs, dtypes, math.inf, 96, **kw)
    x_sat = len(reqs) / sat_s
    ms, lat, st, _ = _serve_run(lib, inputs, reqs, dtypes, 0.5 * x_sat, 96, **kw)
    small = [r for r in synth.request_stream(20 * compare, seed=1243, rate_hz=1.0, nystrom_max_log2n=14)
             if r["n"] <= 1 << 17 and (r["m"] <= 1024 or r["kind"] == "nystrom")][:compare]
    sdt = [torch.float32] * len(small)
    p_s, _, p_outs = _plain_run(lib, inputs, small, math.inf, keep_outputs=True)
    s_s, _, _, s_outs = _serve_run(lib, inputs, small, sdt, math.inf, len(small), keep_outputs=True, **kw)
    acc = _accuracy(lib, inputs, small, s_outs, p_outs, sdt)
    del s_outs
    s32_s, _, _, s32_outs = _serve_run(lib, inputs, small, sdt, math.inf, len(small), keep_outputs=True,
                                       nystrom_f64=False, **kw)
    acc32 = _accuracy(lib, inputs, small, s32_outs, p_outs, sdt)
    del inputs, s32_outs, p_outs
    torch.cuda.empty_cache()
    return {"stream": f"{len(reqs)} config-5 requests (sketch / rSVD / Nystrom, half BF16)",
            "saturation_req_s": round(x_sat, 2), "saturation_p50_ms": round(_pct(lat_sat, 50), 2),
            "saturation_p99_ms": round(_pct(lat_sat, 99), 2),
            "poisson_0.5x": {"rate_req_s": round(0.5 * x_sat, 2), "p50_ms": round(_pct(lat, 50), 2),
                             "p99_ms": round(_pct(lat, 99), 2), "makespan_s": round(ms, 2)},
            "grouped_requests": st_sat["grouped_requests"], "graph_launches": st_sat["graph_launches"],
            "vs_plain_fp64": {"requests": len(small), "closed_batch_speedup": round(p_s / s_s, 2),
                              "accuracy_worst": {kk: float(f"{vv:.3e}") for kk, vv in acc.items()},
                              "policy": "FP32 storage; sketch and rSVD in FP32 arithmetic, Nystrom in FP64 "
                                        "arithmetic (BSRHT_PREC_F64)",
                              "nystrom_in_fp32": {"closed_batch_speedup": round(p_s / s32_s, 2),
                                                  "accuracy_worst": {kk: float(f"{vv:.3e}")
                                                                     for kk, vv in acc32.items()}}}}


def _extra(name, fn, out):
    """Runs one extra measurement; a failure is recorded, not fatal."""
    t0 = time.perf_counter()
    try:
        out[name] = fn()
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    except Exception as e:  # noqa: BLE001 -- reported in the JSON line
        out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
    import paper_2210_11295_gb300 as lib

    dev = torch.device("cuda", torch.cuda.current_device())
    a = make_input(args, rank)
    torch.cuda.synchronize()
    n, m, p, l, k = args.n, args.m, args.p, args.l, args.k
    elem = a.element_size()
    stream = torch.cuda.current_stream()
    mode = args.mode
    if mode == "full":
        try:
            lib.bsrht_rsvd(a[:4096, :256].contiguous(), 4, 16, 1, 0)
        except lib.BsrhtError as e:
            if e.status != -95:
                raise
            mode = "sketch"
    out = torch.empty(l, m, device=dev, dtype=lib.sketch_out_dtype(a.dtype))
    ws = torch.empty(max(lib.bsrht_sketch_workspace(n, m, p, l, a.dtype), 1), dtype=torch.uint8, device=dev)
    if mode == "full":
        rws = torch.empty(max(lib.bsrht_rsvd_workspace(n, m, k, l, p, a.dtype), 1), dtype=torch.uint8, device=dev)
        u = torch.empty(n, k, device=dev, dtype=torch.float64)
        s = torch.empty(k, device=dev, dtype=torch.float64)
        v = torch.empty(m, k, device=dev, dtype=torch.float64)

    variant = {"auto": lib.VARIANT_AUTO, "cudacore": lib.VARIANT_CUDACORE, "tensor": lib.VARIANT_TENSOR,
               "gaussian": lib.VARIANT_GAUSSIAN}[args.variant]

    def step(seed):
        if mode == "full":
            lib.bsrht_rsvd(a, k, l, p, seed, variant=variant, workspace=rws, outs=(u, s, v))
        else:
            lib.bsrht_sketch(a, p, l, seed, out=out, workspace=ws, variant=variant)

    for w in range(args.warmup):
        step(w)
    torch.cuda.synchronize()

    # Sketch kernel alone, CUDA events on the launching stream (the roofline leg).
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        ev[i][0].record(stream)
        lib.bsrht_sketch(a, p, l, 1000 + i, out=out, workspace=ws, variant=variant)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    sketch_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
    # The dominant kernel alone (the roofline's denominator): the library's
    # CUDA events around it on the launching stream (stage "sketch_kernel";
    # the call also runs the sign tables and the block-sum reduce).
    kernel_ms = None
    lib.bsrht_profile_enable(True)
    kms = []
    for i in range(args.steps):
        lib.bsrht_sketch(a, p, l, 2000 + i, out=out, workspace=ws, variant=variant)
        st = dict(lib.bsrht_profile_stages())
        if "sketch_kernel" in st:
            kms.append(st["sketch_kernel"])
    lib.bsrht_profile_enable(False)
    if kms:
        kernel_ms = statistics.mean(kms)

    # The timed steps.
    launches0 = lib.bsrht_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    launches = lib.bsrht_kernel_launches() - launches0
    step_ms = t_start.elapsed_time(t_end) / args.steps
    step_ms = max_over_ranks(world, step_ms)

    # Per-stage times of one extra traced step (library CUDA events).
    stages = None
    if mode == "full":
        lib.bsrht_profile_enable(True)
        step(10_000)
        torch.cuda.synchronize()
        stages = {name: round(ms, 3) for name, ms in lib.bsrht_profile_stages()}
        lib.bsrht_profile_enable(False)

    # The comparator of Sec. 4: the Gaussian-embedding sketch (and one rSVD
    # with it) on the same A, FP32 data only.
    comparator = gaussian_comparator(args, lib, a, sketch_ms, step_ms, mode, stream) \
        if args.dtype == "f32" and args.variant == "auto" else None

    # Algorithm 3 (single-view RSVD) on the same A, s = 2 l: one call, with
    # its stages.
    single_view = single_view_rsvd(args, lib, a, stream) if mode == "full" and args.variant == "auto" else None

    # The metric's other parts (rank 0, the default tall-skinny FP32 run).
    extras = {}
    default_shape = (args.dtype, n, m, p, l, k, args.variant) == ("f32", 1 << 20, 4096, 4, 512, 100, "auto")
    if mode == "full" and default_shape and rank == 0 and not args.no_extras:
        peak_v = peaks()[0]
        _extra("rsvd_error", lambda: rsvd_error_object(lib, a, u, s, v, args), extras)
        _extra("p_sweep", lambda: p_sweep_object(lib, a, l, k, peak_v, stream), extras)
        _extra("f64", lambda: f64_sketch_object(lib, a, p, l, peak_v, stream), extras)
        _extra("config1_fp64", lambda: config1_object(lib, stream), extras)
        _extra("nystrom", lambda: nystrom_object(lib, peak_v, stream), extras)
        _extra("config3_16bit", lambda: config3_object(lib, peak_v, stream), extras)
        _extra("serve", lambda: serve_object(lib, args.serve_summary_requests), extras)

    # End to end through the C ABI from pinned host buffers.
    a_host = a.cpu().pin_memory()
    e2e_ms = None
    h2d = n * m * elem
    d2h = (n * k + k + m * k) * 8 if mode == "full" else l * m * out.element_size()
    if args.e2e_steps > 0:
        a_dev2 = torch.empty_like(a)
        if mode == "full":
            hu = torch.empty(n, k, dtype=torch.float64).pin_memory()
            hs = torch.empty(k, dtype=torch.float64).pin_memory()
            hv = torch.empty(m, k, dtype=torch.float64).pin_memory()
        else:
            hb = torch.empty(l, m, dtype=out.dtype).pin_memory()
        del a
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            a_dev2.copy_(a_host, non_blocking=True)
            if mode == "full":
                lib.bsrht_rsvd(a_dev2, k, l, p, i, variant=variant, workspace=rws, outs=(u, s, v))
                hu.copy_(u, non_blocking=True)
                hs.copy_(s, non_blocking=True)
                hv.copy_(v, non_blocking=True)
            else:
                lib.bsrht_sketch(a_dev2, p, l, i, out=out, workspace=ws, variant=variant)
                hb.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.e2e_steps
        e2e_ms = max_over_ranks(world, e2e_ms)

    total_bytes_all = sum_over_ranks(world, float(n * m * elem))
    value = total_bytes_all / (step_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    sketch_bytes = n * m * elem + l * m * out.element_size()
    achieved_call = sketch_bytes / (sketch_ms * 1e-3) / 1e9
    achieved = sketch_bytes / ((kernel_ms or sketch_ms) * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(step_ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32": "f32", "f64": "f64", "bf16": "f32", "f16": "f32"}[args.dtype],
        "data": "synthetic",
        "config": {"workload": WORKLOAD if (mode == "full" and args.dtype == "f32" and n == 1 << 20 and m == 4096)
                   else f"n={n} m={m} {args.dtype} p={p} l={l} k={k} mode={mode}",
                   "n": n, "m": m, "p": p, "l": l, "k": k, "storage": args.dtype, "step": mode,
                   "l2": "A is 16 GiB >> 129 MB L2: inputs larger than L2, no flush"},
        "sketch": {"ms": round(sketch_ms, 4), "gbs": round(achieved_call, 2),
                   "frac_of_measured_peak": round(achieved_call / peak, 4),
                   "kernel_ms": round(kernel_ms, 4) if kernel_ms else None},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": sketch_traffic(args.dtype, n, m, p, l, args.variant),
                     "kernel": ("k_sketch_chunked + k_sketch_reduce (one bsrht_sketch call)" if args.dtype == "f64"
                                else ("k_sketch_tc" if args.variant == "tensor" else "k_sketch_tma")
                                + " (its own CUDA events; the whole bsrht_sketch call, with the sign tables and "
                                  "the block-sum reduce, is sketch.ms)") if kernel_ms else
                               "one bsrht_sketch call",
                     "peak_kind": peak_kind},
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
        "e2e": {"value": round(total_bytes_all / (e2e_ms * 1e-3) / 1e9, 3) if e2e_ms else None, "unit": "GB/s",
                "ms_per_step": round(e2e_ms, 3) if e2e_ms else None,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
    }
    if stages:
        line["stages_ms"] = stages
    if comparator:
        line["gaussian_comparator"] = comparator
    if single_view:
        line["single_view_rsvd"] = single_view
    line.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------- serving
class _ServeInputs:
    """Resident A matrices of the serving stream: one FP32 matrix per size
    class (n, next power of two >= m) from the config-2 generator (rank
    min(1000, m_class / 2)), requests take its first m columns; BF16 and FP64
    copies on demand; one PSD n x n matrix per n for Nystrom requests."""

    def __init__(self):
        self.base = {}
        self.copies = {}

    def get(self, kind, n, m, dtype):
        import torch
        import synth
        if kind == "nystrom":
            key = ("psd", n)
            if key not in self.base:
                self.base[key] = synth.psd_lowrank_device(n, rank=min(1000, n // 2), seed=1241 + n)
        else:
            mc = 64
            while mc < m:
                mc *= 2
            key = (n, mc)
            if key not in self.base:
                self.base[key] = synth.lowrank_noise_device(n, mc, rank=min(1000, mc // 2), seed=1236 + n + mc)
        src = self.base[key]
        if dtype != torch.float32:
            ck = key + (dtype,)
            if ck not in self.copies:
                self.copies[ck] = src.to(dtype)
            src = self.copies[ck]
        return src if kind == "nystrom" else src[:, :m]

    def bytes(self):
        return sum(t.numel() * t.element_size() for t in list(self.base.values()) + list(self.copies.values()))


def _serve_outputs(req, dtype, lib):
    import torch
    n, m, l, k = req["n"], req["m"], req["l"], req["k"]
    if req["kind"] == "sketch":
        return (torch.empty(l, m, device="cuda", dtype=lib.sketch_out_dtype(dtype)),)
    if req["kind"] == "rsvd":
        return (torch.empty(n, k, device="cuda", dtype=torch.float64), torch.empty(k, device="cuda", dtype=torch.float64),
                torch.empty(m, k, device="cuda", dtype=torch.float64))
    return (torch.empty(n, k, device="cuda", dtype=torch.float64), torch.empty(k, device="cuda", dtype=torch.float64))


def _serve_run(lib, inputs, reqs, dtypes, rate, window, keep_outputs=False, nystrom_f64=True, **server_kw):
    """Feeds reqs (arrival times scaled to `rate` req/s; inf = all at once)
    to a fresh server, at most `window` in flight.  Returns (makespan s,
    latencies arrival->done ms, stats, outputs)."""
    import torch
    arrivals = [0.0] * len(reqs)
    if not math.isinf(rate):
        t0r = reqs[0]["t"]
        scale = (len(reqs) / rate) / max(reqs[-1]["t"] - t0r, 1e-9)
        arrivals = [(r["t"] - t0r) * scale for r in reqs]
    mats = [inputs.get(r["kind"], r["n"], r["m"], dt) for r, dt in zip(reqs, dtypes)]
    torch.cuda.synchronize()
    outs = [None] * len(reqs)
    tickets = [None] * len(reqs)
    lat = [None] * len(reqs)
    with lib.Server(**server_kw) as srv:
        inflight = []
        start = time.monotonic()
        for i, (r, a) in enumerate(zip(reqs, mats)):
            while len(inflight) >= window:
                j = inflight.pop(0)
                srv.wait(tickets[j], 3600.0)
                if not keep_outputs:
                    outs[j] = None
            delay = start + arrivals[i] - time.monotonic()
            if delay > 0:
                time.sleep(delay)
            o = _serve_outputs(r, dtypes[i], lib)
            if r["kind"] == "sketch":
                t = srv.submit_sketch(a, r["p"], r["l"], r["seed"], o[0])
            elif r["kind"] == "rsvd":
                t = srv.submit_rsvd(a, r["k"], r["l"], r["p"], r["seed"], o)
            else:
                # Nystrom on FP32 storage in FP64 arithmetic: an FP32 sketch
                # cannot resolve core directions below l 2^-23 of the
                # largest, which the FP64 path keeps (Remark 3.1's threshold).
                t = srv.submit_nystrom(a, r["k"], r["l"], r["p"], r["seed"], o,
                                       precision=lib.PREC_F64 if nystrom_f64 and a.dtype == torch.float32
                                       else lib.PREC_AUTO)
            tickets[i], outs[i] = t, o
            inflight.append(i)
        for j in inflight:
            srv.wait(tickets[j], 3600.0)
        end = max(srv.times(t)[1] for t in tickets)
        for i, t in enumerate(tickets):
            lat[i] = (srv.times(t)[1] - (start + arrivals[i])) * 1e3
        st = srv.stats()
        bad = [(i, srv.poll(t)[1]) for i, t in enumerate(tickets) if srv.poll(t)[1] != 0]
    if bad:
        detail = "; ".join(f"{reqs[i]} {dtypes[i]}: {lib.strerror(st)}" for i, st in bad[:8])
        raise RuntimeError(f"{len(bad)} served requests failed: {detail}")
    return end - start, lat, st, outs


def _plain_run(lib, inputs, reqs, rate, keep_outputs=False):
    """The plain path: FP64 inputs, one direct library call at a time on one
    stream, no grouping, graphs or tuning; requests queue behind each other."""
    import torch
    t0r = reqs[0]["t"]
    if math.isinf(rate):
        arrivals = [0.0] * len(reqs)
    else:
        scale = (len(reqs) / rate) / max(reqs[-1]["t"] - t0r, 1e-9)
        arrivals = [(r["t"] - t0r) * scale for r in reqs]
    mats = [inputs.get(r["kind"], r["n"], r["m"], torch.float64) for r in reqs]
    torch.cuda.synchronize()
    lat, outs = [], []
    start = time.monotonic()
    for r, a, arr in zip(reqs, mats, arrivals):
        delay = start + arr - time.monotonic()
        if delay > 0:
            time.sleep(delay)
        if r["kind"] == "sketch":
            o = (lib.bsrht_sketch(a, r["p"], r["l"], r["seed"]),)
        elif r["kind"] == "rsvd":
            o = lib.bsrht_rsvd(a, r["k"], r["l"], r["p"], r["seed"])
        else:
            o = lib.bsrht_nystrom(a, r["k"], r["l"], r["p"], r["seed"])
        torch.cuda.synchronize()
        lat.append((time.monotonic() - start - arr) * 1e3)
        outs.append(o if keep_outputs else None)
    return time.monotonic() - start, lat, outs


def _pct(v, q):
    v = sorted(v)
    rank = max(1, min(len(v), math.ceil(q / 100.0 * len(v))))
    return v[rank - 1]


def _accuracy(lib, inputs, reqs, outs_served, outs_plain, dtypes):
    """Per request: sketch -> relative Frobenius difference served vs plain;
    rSVD -> |err_served - err_plain| / err_plain of ||A - U S V^T||_F;
    Nystrom -> difference of tr(A) - sum(Lambda) (exact trace error, the
    residual is PSD) relative to tr(A).  Returns the worst of each kind."""
    import torch
    worst = {"sketch": 0.0, "rsvd": 0.0, "nystrom": 0.0}
    for r, so, po, dt in zip(reqs, outs_served, outs_plain, dtypes):
        a = inputs.get(r["kind"], r["n"], r["m"], torch.float64)
        if r["kind"] == "sketch":
            d = (torch.linalg.norm(so[0].double() - po[0]) / torch.linalg.norm(po[0])).item()
        elif r["kind"] == "rsvd":
            def err(o):
                u, s, v = o
                return torch.linalg.norm(a - (u * s) @ v.T).item()
            ep = err(po)
            d = abs(err(so) - ep) / max(ep, 1e-300)
        else:
            # Relative to tr(A): the stream's PSD matrices have rank below l,
            # so the FP64 trace error itself is at rounding level and cannot
            # serve as the scale.
            tr = torch.trace(a).item()
            ep = tr - po[1].sum().item()
            d = abs((tr - so[1].sum().item()) - ep) / max(abs(tr), 1e-300)
        worst[r["kind"]] = max(worst[r["kind"]], d)
    return worst


def run_serve(args):
    """Config-5 stream through the serving loop: Poisson arrivals at 0.5x,
    0.8x and 1.0x of the measured saturation throughput, p50 / p99 latency
    (arrival to completion) and throughput; then a reduced stream (n <= 2^17,
    m <= 1024, Nystrom n = 2^14) through both the served path and the plain FP64
    one-at-a-time path, with their accuracy compared request by request."""
    import numpy as np
    import torch
    import synth
    import paper_2210_11295_gb300 as lib

    torch.cuda.set_device(0)
    reqs = synth.request_stream(args.serve_requests, seed=1240, rate_hz=1.0)
    rng = np.random.default_rng(1242)
    dtypes = [torch.bfloat16 if rng.random() < 0.5 and r["kind"] != "nystrom" else torch.float32 for r in reqs]
    inputs = _ServeInputs()
    kw = dict(hbm_budget=24 << 30, executors=4, max_group=16)
    # Warm-up pass (graphs, tuning, allocator) on the first requests, then
    # saturation (on the whole stream, or on its leading requests).
    _serve_run(lib, inputs, reqs[: min(60, len(reqs))], dtypes, math.inf, args.serve_window, **kw)
    n_sat = len(reqs) if args.serve_sat_requests <= 0 else min(len(reqs), args.serve_sat_requests)
    sat_s, lat_sat, st_sat, _ = _serve_run(lib, inputs, reqs[:n_sat], dtypes[:n_sat], math.inf, args.serve_window,
                                           **kw)
    x_sat = n_sat / sat_s
    points = []
    for frac in (float(f) for f in args.serve_points.split(",") if f.strip()):
        ms, lat, st, _ = _serve_run(lib, inputs, reqs, dtypes, frac * x_sat, args.serve_window, **kw)
        points.append({"load": frac, "rate_req_s": round(frac * x_sat, 2), "makespan_s": round(ms, 3),
                       "throughput_req_s": round(len(reqs) / ms, 2), "p50_ms": round(_pct(lat, 50), 3),
                       "p99_ms": round(_pct(lat, 99), 3),
                       "grouped_launches": st["grouped_launches"], "grouped_requests": st["grouped_requests"],
                       "graph_launches": st["graph_launches"]})
    # Served vs plain FP64 one-at-a-time on the reduced stream.
    small = [r for r in synth.request_stream(20 * args.serve_compare, seed=1243, rate_hz=1.0, nystrom_max_log2n=14)
             if r["n"] <= 1 << 17 and (r["m"] <= 1024 or r["kind"] == "nystrom")][: args.serve_compare]
    sdt = [torch.float32] * len(small)
    p_s, p_lat, p_outs = _plain_run(lib, inputs, small, math.inf, keep_outputs=True)
    s_s, s_lat, s_st, s_outs = _serve_run(lib, inputs, small, sdt, math.inf, len(small), keep_outputs=True, **kw)
    acc = _accuracy(lib, inputs, small, s_outs, p_outs, sdt)
    rate = 0.8 * len(small) / p_s
    p2_s, p2_lat, _ = _plain_run(lib, inputs, small, rate)
    s2_s, s2_lat, _, _ = _serve_run(lib, inputs, small, sdt, rate, len(small), **kw)
    line = {
        "metric": "serving: throughput (req/s) and p50/p99 latency (arrival to completion, ms)",
        "value": round(x_sat, 3), "unit": "req/s", "n_gpus": 1, "higher_is_better": True,
        "data": "synthetic", "dtype": "f32/bf16 storage, FP32 sketch arithmetic, FP64 QR/SVD/Cholesky",
        "config": {"workload": f"Poisson stream of {len(reqs)} sketch/rSVD/Nystrom requests, n=2^U{{14..20}}, "
                               "m log-uniform [64,4096], p in {1,2,4,8,16}, l log-uniform [64,1024], "
                               "k=l//4, FP32 or BF16 (Nystrom: n<=2^15, FP32 PSD)",
                   "executors": kw["executors"], "max_group": kw["max_group"], "hbm_budget": kw["hbm_budget"],
                   "window": args.serve_window, "input_gb": round(inputs.bytes() / 1e9, 2)},
        "saturation": {"requests": n_sat, "makespan_s": round(sat_s, 3), "throughput_req_s": round(x_sat, 2),
                       "a_gb_per_s": round(sum(r["n"] * r["m"] * (2 if dt == torch.bfloat16 else 4)
                                               for r, dt in zip(reqs[:n_sat], dtypes[:n_sat])) / sat_s / 1e9, 2), "p50_ms": round(_pct(lat_sat, 50), 3),
                       "p99_ms": round(_pct(lat_sat, 99), 3), "grouped_launches": st_sat["grouped_launches"],
                       "grouped_requests": st_sat["grouped_requests"], "graph_launches": st_sat["graph_launches"],
                       "tuned_classes": st_sat["tuned_classes"]},
        "poisson": points,
        "vs_plain_fp64": {
            "stream": f"{len(small)} requests with n <= 2^17, m <= 1024, Nystrom n = 2^14 "
                      "(FP32 served, FP64 plain)",
            "closed_batch": {"served_req_s": round(len(small) / s_s, 2), "plain_req_s": round(len(small) / p_s, 2),
                             "speedup": round(p_s / s_s, 2),
                             "served_p50_ms": round(_pct(s_lat, 50), 3), "served_p99_ms": round(_pct(s_lat, 99), 3),
                             "plain_p50_ms": round(_pct(p_lat, 50), 3), "plain_p99_ms": round(_pct(p_lat, 99), 3)},
            "poisson_at_0.8x_plain": {"rate_req_s": round(rate, 2),
                                      "served_p50_ms": round(_pct(s2_lat, 50), 3),
                                      "served_p99_ms": round(_pct(s2_lat, 99), 3),
                                      "plain_p50_ms": round(_pct(p2_lat, 50), 3),
                                      "plain_p99_ms": round(_pct(p2_lat, 99), 3)},
            "accuracy_worst": {k: float(f"{v:.3e}") for k, v in acc.items()},
            "accuracy_note": "sketch: relative Frobenius difference to the FP64 result; rSVD: relative "
                             "difference of ||A - U S V^T||_F; Nystrom: difference of tr(A) - sum(Lambda), "
                             "relative to tr(A)"},
        "gpu_launches": int(lib.bsrht_kernel_launches()),
    }
    print(json.dumps(line), flush=True)


def run_nystrom(args):
    """Algorithm 2 on the kernel workload: A_ij = exp(-|xi - xj|^2 / (2 h^2)),
    x_i ~ U[0,1]^784, h = median pairwise distance (seeded 4096-point
    subsample), FP32 n x n; p, l from the command line (8, 600 for the
    65536-point case), every k of --nystrom-ks.  Reports the step time, the
    sketch kernel's HBM rate and the trace error tr(A) - sum(Lambda) (exact:
    the residual is PSD, Sec. 3.2)."""
    import torch
    import synth
    import paper_2210_11295_gb300 as lib

    torch.cuda.set_device(0)
    n, p, l = args.n, args.p, args.l
    x = synth.rbf_points(n, 784, seed=1238)
    h = synth.rbf_bandwidth(x)
    a = synth.rbf_kernel_device(torch.from_numpy(x).cuda(), h, dtype=torch.float32)
    del x
    torch.cuda.synchronize()
    tr = float(torch.trace(a.double()).item())
    stream = torch.cuda.current_stream()
    results = []
    for k in [int(v) for v in args.nystrom_ks.split(",")]:
        ws = torch.empty(lib.bsrht_nystrom_workspace(n, k, l, p, torch.float32), dtype=torch.uint8, device="cuda")
        u = torch.empty(n, k, device="cuda", dtype=torch.float64)
        lam = torch.empty(k, device="cuda", dtype=torch.float64)
        for w in range(args.warmup):
            lib.bsrht_nystrom(a, k, l, p, w, workspace=ws, outs=(u, lam))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            lib.bsrht_nystrom(a, k, l, p, 100 + i, workspace=ws, outs=(u, lam))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        lib.bsrht_profile_enable(True)
        lib.bsrht_nystrom(a, k, l, p, 7, workspace=ws, outs=(u, lam))
        torch.cuda.synchronize()
        stages = {name: round(t, 3) for name, t in lib.bsrht_profile_stages()}
        lib.bsrht_profile_enable(False)
        results.append({"k": k, "ms_per_step": round(ms, 3), "trace_error": tr - float(lam.sum().item()),
                        "trace_error_rel": (tr - float(lam.sum().item())) / tr, "stages_ms": stages})
    out = torch.empty(l, n, device="cuda", dtype=torch.float32)
    sws = torch.empty(max(lib.bsrht_sketch_workspace(n, n, p, l, torch.float32), 1), dtype=torch.uint8,
                      device="cuda")
    lib.bsrht_sketch(a, p, l, 0, out=out, workspace=sws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        lib.bsrht_sketch(a, p, l, i, out=out, workspace=sws)
    e1.record(stream)
    torch.cuda.synchronize()
    sk_ms = e0.elapsed_time(e1) / args.steps
    peak, peak_kind = peaks()
    gbs = (n * n * 4 + l * n * 4) / (sk_ms * 1e-3) / 1e9
    line = {"metric": "Nystrom (Algorithm 2) time at stated trace error; sketch A Omega^T HBM GB/s",
            "value": results[0]["ms_per_step"], "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"RBF kernel n={n} (x ~ U[0,1]^784, median bandwidth h={h:.4f}) fp32 p={p} l={l}",
                       "steps": args.steps, "warmup": args.warmup},
            "per_k": results,
            "sketch": {"ms": round(sk_ms, 4), "gbs": round(gbs, 2), "frac_of_measured_peak": round(gbs / peak, 4),
                       "peak_kind": peak_kind},
            "trace_A": tr}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.mode == "nystrom":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "nystrom mode has no CPU reference arm"}))
            return
        run_nystrom(args)
        return
    if args.mode == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "serve mode has no CPU reference arm"}))
            return
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
