"""Benchmark of the candidate-scoring hot path on the scale workload.

One step = one pass of the whole path over one batch of synthetic input:
draw S uniform directions (Philox, on the GPU), score them with the BF16
tensor-core kernel (GEMM1 projections -> sector rounding -> GEMM2 per-class
sums -> f), select the top 64, re-score those in FP64 and pick the winner.

Workload: n = 2^20, r = 4, K = 3, S = 2^16 directions per step per GPU;
V ~ CN(0,1) * diag(4, 2, 1, 0.5) in complex64 (seed 0); step s on rank g uses
direction seed 1 + s * world + g.  Metric: candidate*n evaluations per
second (S * n per step), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode bf16|fp32]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (same metric, unit and config).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate·n evals/s at n=2^20,r=4,K=3 (% roofline); samples to 0.999·best"
UNIT = "candidate*n evals/s"
N, R, K, S, TOP_M = 1 << 20, 4, 3, 1 << 16, 64
SCALES = (4.0, 2.0, 1.0, 0.5)
L2_FLUSH_BYTES = 512 << 20


def _config(mode: str, world: int):
    return {"workload": "scale: n=2^20, r=4, K=3, S=2^16 uniform directions per GPU per step; "
                        "V ~ CN(0,1) diag(4,2,1,0.5) complex64; top-64 FP64 rescore",
            "n": N, "r": R, "K": K, "S_per_gpu": S, "top_m": TOP_M,
            "mode": "BF16 tensor-core + FP64 rescore" if mode == "bf16" else "FP32 CUDA-core + FP64 rescore",
            "parallelism": "replicas over candidates (dp%d)" % world,
            "l2": "flushed before every timed step (512 MiB write, untimed)"}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p.get("bf16_tflops", 1900.0)), float(p.get("hbm_gbs", 6800.0)), "measured"
    return 1900.0, 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(seed: int, sample_S: int):
    """The FP64 oracle, as it stands, on the host cores: sample_S directions of
    the same workload over the full n."""
    import oracle
    from paper_2602_20376_gb300 import inputs
    cores = len(os.sched_getaffinity(0))
    V = inputs.factor(N, R, seed=0, scales=SCALES, dtype=np.complex64)
    C = oracle.sphere_sample(seed, sample_S, R).astype(np.complex64)
    oracle.score(V, K, C[:2], nthreads=cores)  # load + warm
    t0 = time.perf_counter()
    oracle.score(V, K, C, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": sample_S * N / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d directions x n=2^20 coordinates (FP64 C oracle, OpenMP over directions)" % sample_S,
            "seconds": dt}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample_S = args.ref_sample
    vals = []
    for step in range(args.warmup + args.steps):
        b = cpu_baseline(1 + step, sample_S)
        if step >= args.warmup:
            vals.append(b)
    secs = float(np.sum([v["seconds"] for v in vals]))
    value = len(vals) * sample_S * N / secs
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(vals), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(_config("bf16", 1), S_per_step=sample_S),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    global S
    S = args.candidates
    import torch
    import torch.distributed as dist

    from paper_2602_20376_gb300 import inputs, lrq

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lrq.load()
    mode = lrq.LRQ_MODE_BF16_TC if args.mode == "bf16" else lrq.LRQ_MODE_FP32

    V_host = torch.from_numpy(inputs.factor(N, R, seed=0, scales=SCALES, dtype=np.complex64)).pin_memory()
    V = V_host.to(dev)
    C = torch.empty((S, R), dtype=torch.complex64, device=dev)
    ws = lrq.workspace(lrq.lrq_sample_score_workspace_size(N, R, K, S, mode, TOP_M), dev)
    ws_r = lrq.workspace(lrq.lrq_rescore_workspace_size(N, R, TOP_M), dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    top_idx = torch.empty(TOP_M, dtype=torch.int64, device=dev)
    top_f = torch.empty(TOP_M, dtype=torch.float32, device=dev)
    f64 = torch.empty(TOP_M, dtype=torch.float64, device=dev)
    best = torch.empty(1, dtype=torch.int64, device=dev)
    best_f = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(s):
        seed = 1 + s * world + rank
        lrq.lrq_sample_score(V, K, C, True, seed, mode, TOP_M, None, top_idx, top_f, ws, status, stream)
        lrq.lrq_rescore(V, K, C, top_idx, f64, None, best, best_f, ws_r, status, stream)

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    lrq.check_status(status, "warm-up")

    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_stop = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    s_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    s_stop = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = lrq.lrq_kernel_launches()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            s_start[i].record(stream)
            lrq.lrq_set_timing_events(k_start[i], k_stop[i])
            step(args.warmup + i)
            lrq.lrq_set_timing_events(None, None)
            s_stop[i].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    launches = lrq.lrq_kernel_launches() - launches0
    lrq.check_status(status, "timed steps")
    step_ms = float(sum(a.elapsed_time(b) for a, b in zip(s_start, s_stop)))
    kern_ms = float(sum(a.elapsed_time(b) for a, b in zip(k_start, k_stop)))
    t_max = torch.tensor([step_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    step_ms = float(t_max.item())
    evals = float(world) * args.steps * S * N
    value = evals / (step_ms * 1e-3)

    # end to end through the C ABI with host buffers: V copied in from pinned
    # memory and the winner read back inside the timed region, every step
    res_host = torch.empty(TOP_M + 2, dtype=torch.float64).pin_memory()
    e_start = torch.cuda.Event(enable_timing=True)
    e_stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_start.record(stream)
    for i in range(args.steps):
        V.copy_(V_host, non_blocking=True)
        step(args.warmup + args.steps + i)
        res_host[:TOP_M].copy_(f64, non_blocking=True)
        res_host[TOP_M:TOP_M + 1].copy_(best_f, non_blocking=True)
        res_host[TOP_M + 1:].copy_(best.to(torch.float64), non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e_stop.record(stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    lrq.check_status(status, "e2e steps")
    e2e_val = float(world) * args.steps * S * N / e2e_s

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak_tf, _, peak_kind = _peaks()
    flops = 16.0 * R * N * S  # two complex r-contractions per evaluation (algorithmic)
    kern_avg_s = kern_ms * 1e-3 / args.steps
    achieved = flops / kern_avg_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.mode == "bf16" else "f32",
        "data": "synthetic", "config": _config(args.mode, world),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved / peak_tf, "traffic": args.traffic,
                     "kernel": "score_tc_kernel" if args.mode == "bf16" else "score_fp32_kernel",
                     "kernel_ms": kern_avg_s * 1e3, "peak_kind": peak_kind + " bf16 dense (burst)",
                     "flops_per_launch": flops},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": N * R * 8,
                "d2h_bytes_per_step": (TOP_M + 2) * 8},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "samples_to_best": None,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(1, args.cpu_sample)
        cb.pop("seconds")
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["bf16", "fp32"], default="bf16")
    ap.add_argument("--candidates", type=int, default=S,
                    help="directions per step per GPU (default 2^16; smaller only for profiling runs)")
    ap.add_argument("--cpu-sample", type=int, default=256)
    ap.add_argument("--ref-sample", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the scoring kernel from an ncu capture")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
