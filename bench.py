"""Benchmark of the candidate-scoring hot path on the scale workload.

One step = one pass of the whole path over one batch of synthetic input:
draw S uniform directions (Philox, on the GPU), score them with the
tensor-core kernel (F16 GEMM1 projections -> sector rounding -> FP8 GEMM2
per-class sums -> f) against the instance's operands (packed once by
lrq_prepare), select the top 64, re-score those in FP64 and pick the
winner.  The end-to-end leg copies V in from host memory, prepares it and
reads the winner back inside its timed region, every step.

Workload: n = 2^20, r = 4, K = 3, S = 2^16 directions per step per GPU;
V ~ CN(0,1) * diag(4, 2, 1, 0.5) in complex64 (seed 0); step s on rank g uses
direction seed 1 + s * world + g.  Metric: candidate*n evaluations per
second (S * n per step), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode tc|fp32]
                  [--workload scale|exact|maxcut|batched|learned|rank1|hybrid] [--sampler uniform|null]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (same metric, unit and config).

The default line (workload "scale") also carries "samples_to_best": the
learned proposal's median S_u / S_l on 256 held-out angular-synchronisation
instances (n = 4096, K = 8, r = 4), trained on the GPU in the same run, with
the fixed direction e_1 as a second baseline, at the workload's sigma and in
a high-noise regime ("hard").
The other workloads print one line each for the remaining paths:
  exact    n = 12, r = 2, K = 3: vertex enumeration + 4096 sampled directions
  maxcut   planted 3-partition SBM, n = 10^6: Laplacian truncation (r = 3),
           2^17 tensor-core-scored candidates, FP64 rescore, exact cut count
           (--sampler null: null-vector directions instead of uniform ones)
  batched  512 instances, n log-uniform in [64, 8192], r in 2..6,
           K in {2, 3, 4, 8}: one graph-captured persistent launch; also
           the same launch with an exact sub-batch (--exact-subbatch)
  learned  the learned proposal at a larger training set
  rank1    SBM n = 10^6: rank-2 Laplacian truncation, the two-eigenvector
           rounding vector q = u1 + i u2, exact rank-1 sweep (Algorithm 1)
           and the best exact cut along it
  hybrid   rank1, then greedy local search from the sweep's best-cut state
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
            "mode": ("tensor-core (F16 signs, FP8 hi+lo class sums) + FP64 rescore" if mode == "tc"
                     else "FP32 CUDA-core + FP64 rescore"),
            "parallelism": "replicas over candidates (dp%d)" % world,
            "prepared_v": "V's operands packed once (lrq_prepare) before the device-timed steps, which score "
                          "fresh directions against them; the e2e steps copy V in and prepare it every step",
            "l2": "flushed before every timed step (512 MiB write, untimed)"}


# DRAM bytes (read + write) of one score_tc_kernel launch of the default scale
# workload (n = 2^20, r = 4, K = 3, S = 2^16, tensor-core mode), from a one-pass
# ncu capture of the launch after the L2 flush: reads are one pass over the
# packed coordinate tiles and the directions (candidate tiles that reuse a
# coordinate tile find it in L2), writes the FP64 partial sums (S x 2r doubles
# per coordinate chunk).  Measured with
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none \
#       -k regex:score_tc -s 1 -c 1 python bench.py --steps 1 --warmup 1 --no-cpu-baseline --no-learned
# (one pass): 72.20 MB read + 10.41 MB written.  It must be taken again whenever
# the kernel changes, and set to None (reported as null) until it has been.
SCALE_TRAFFIC_BYTES = 72.20e6 + 10.41e6


def _traffic(args):
    if args.traffic is not None:
        return args.traffic
    if args.mode == "tc" and args.candidates == S and args.workload == "scale":
        return SCALE_TRAFFIC_BYTES  # None until measured for the current kernel
    return None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p.get("bf16_tflops", 1900.0)), float(p.get("hbm_gbs", 6800.0)), "measured"
    return 1900.0, 6800.0, "fallback"


def _sm_max_mhz():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh).get("sm_max_mhz", 2070.0))
    return 2070.0


N_SM = 152
FP8_OVER_BF16 = 2.0  # nominal dense fp8 / bf16 tensor rate (4.5 / 2.25 PFLOP/s)


def tc_roofline(flops, kern_s, bf16_peak, kind):
    """Roofline of the tensor-core kernel against the dtype-weighted peak: of
    the 16 r flops of an evaluation, GEMM1's 8 r run in F16 (the measured
    dense BF16 rate, which F16 shares) and GEMM2's 8 r in FP8 E4M3 (nominally
    twice that rate), so the pair's peak is 1 / (0.5 / P + 0.5 / (2 P)) =
    4/3 P.  The fraction on the plain BF16 basis is kept beside it."""
    achieved = flops / kern_s / 1e12
    peak = bf16_peak / (0.5 + 0.5 / FP8_OVER_BF16)
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_kind": "%s dense bf16 burst %.1f TFLOP/s for GEMM1's F16 half, x%.0f (nominal fp8/bf16) for "
                         "GEMM2's FP8 half: dtype-weighted" % (kind, bf16_peak, FP8_OVER_BF16),
            "frac_bf16_basis": achieved / bf16_peak}


_FP32_PEAK = None


def fp32_peak_measured():
    """Measured FP32 CUDA-core peak: a cuBLAS SGEMM (TF32 off) of 8192^3,
    best of 5 after 3 warm-ups, in TFLOP/s -- the FP32 counterpart of the
    cuBLAS BF16 figure of the measured peaks.  Cached per process."""
    global _FP32_PEAK
    if _FP32_PEAK is None:
        import torch
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        try:
            n = 8192
            a = torch.randn((n, n), device="cuda", dtype=torch.float32)
            b = torch.randn((n, n), device="cuda", dtype=torch.float32)
            c = torch.empty_like(a)
            for _ in range(3):
                torch.matmul(a, b, out=c)
            best = None
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            _FP32_PEAK = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b, c
        finally:
            torch.backends.cuda.matmul.allow_tf32 = old
    return _FP32_PEAK


def fp32_roofline(flops, kern_s):
    """Roofline of an FP32 CUDA-core kernel (bound by FP32 issue), against the
    algorithmic 16 r flops per evaluation: the peak is the measured FP32
    SGEMM rate; the unit-count figure (152 SMs x 128 FP32 lanes x 2 flops x
    the maximum SM clock) is given beside it."""
    achieved = flops / kern_s / 1e12
    derived = N_SM * 128 * 2 * _sm_max_mhz() * 1e6 / 1e12
    peak = fp32_peak_measured()
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_kind": "measured: cuBLAS FP32 SGEMM 8192^3, TF32 off (of measured)",
            "peak_derived": derived, "frac_derived": achieved / derived,
            "peak_derived_kind": "%d SMs x 128 FP32 lanes x 2 flops x %.0f MHz" % (N_SM, _sm_max_mhz())}


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


def cpu_baseline(seed: int, sample_S: int, threads: int = 0):
    """The FP64 oracle, as it stands, on the host cores (all of them, or
    `threads`): sample_S directions of the same workload over the full n."""
    import oracle
    from paper_2602_20376_gb300 import inputs
    cores = threads or len(os.sched_getaffinity(0))
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
            "config": dict(_config("tc", 1), S_per_step=sample_S),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def score_error(V, C, ws, ws_r, mode, stream, sample=1024, seed=7):
    """The tensor-core mode's per-candidate error on the scale workload: one
    more (untimed) scoring of S directions, then FP64 re-scoring of a fixed
    random sample of them (lrq_rescore, equal to the FP64 oracle to 1e-9):
    max and median of |f_tc - f_64| / f_64."""
    import torch
    from paper_2602_20376_gb300 import lrq
    dev = V.device
    Sn = C.shape[0]
    scores = torch.empty(Sn, dtype=torch.float32, device=dev)
    top_idx = torch.empty(TOP_M, dtype=torch.int64, device=dev)
    top_f = torch.empty(TOP_M, dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    lrq.lrq_sample_score(V, K, C, True, 987654321, mode, TOP_M, scores, top_idx, top_f, ws, status, stream)
    m = min(sample, Sn)
    idx = torch.from_numpy(np.random.default_rng(seed).choice(Sn, m, replace=False).astype(np.int64)).to(dev)
    f64 = torch.empty(m, dtype=torch.float64, device=dev)
    best = torch.empty(1, dtype=torch.int64, device=dev)
    best_f = torch.empty(1, dtype=torch.float64, device=dev)
    wsr = lrq.workspace(lrq.lrq_rescore_workspace_size(V.shape[0], V.shape[1], m), dev)
    lrq.lrq_rescore(V, K, C, idx, f64, None, best, best_f, wsr, status, stream)
    torch.cuda.synchronize()
    lrq.check_status(status, "score error sample")
    ref = f64.cpu().numpy()
    rel = np.abs(scores[idx].double().cpu().numpy() - ref) / ref
    return {"max_rel": float(rel.max()), "median_rel": float(np.median(rel)), "sample": int(m),
            "reference": "FP64 re-scoring (lrq_rescore) of a fixed random sample of the S directions"}


def run_ours(args):
    global S
    S = args.candidates
    import torch
    import torch.distributed as dist

    from paper_2602_20376_gb300 import inputs, lrq, multi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lrq.load()
    mode = lrq.LRQ_MODE_TC if args.mode == "tc" else lrq.LRQ_MODE_FP32

    V_host = torch.from_numpy(inputs.factor(N, R, seed=0, scales=SCALES, dtype=np.complex64)).pin_memory()
    V = V_host.to(dev)
    C = torch.empty((S, R), dtype=torch.complex64, device=dev)
    ws = lrq.workspace(lrq.lrq_sample_score_workspace_size(N, R, K, S, mode, TOP_M), dev)
    ws_r = lrq.workspace(lrq.lrq_rescore_workspace_size(N, R, TOP_M), dev)
    prep = lrq.PreparedInstance(N, R, K, mode=mode, device=dev)
    ws_p = lrq.workspace(prep.workspace_size(S, TOP_M), dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    top_idx = torch.empty(TOP_M, dtype=torch.int64, device=dev)
    top_f = torch.empty(TOP_M, dtype=torch.float32, device=dev)
    f64 = torch.empty(TOP_M, dtype=torch.float64, device=dev)
    best = torch.empty(1, dtype=torch.int64, device=dev)
    best_f = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(s):
        seed = multi.direction_seed(s, world, rank)
        prep.score_into(C, True, seed, TOP_M, None, top_idx, top_f, ws_p, status, stream)
        lrq.lrq_rescore(V, K, C, top_idx, f64, None, best, best_f, ws_r, status, stream)

    prep.prepare(V, stream)
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
    step_ms = multi.max_over_ranks(step_ms, device=dev)
    # the only exchange of the path: each rank's winner of its last step
    win_f, win_rank, win_idx = multi.merge_best(float(best_f.item()), int(best.item()), device=dev)
    evals = float(world) * args.steps * S * N
    value = evals / (step_ms * 1e-3)

    # end to end through the C ABI with host buffers: V copied in from pinned
    # memory and the winner read back inside the timed region, every step
    res_host = torch.empty(TOP_M + 2, dtype=torch.float64).pin_memory()
    e_start = torch.cuda.Event(enable_timing=True)
    e_stop = torch.cuda.Event(enable_timing=True)
    for i in range(min(args.warmup, 2)):  # untimed: the host-buffer path once warmed up
        V.copy_(V_host, non_blocking=True)
        prep.prepare(V, stream)
        step(args.warmup + i)
        res_host[:TOP_M].copy_(f64, non_blocking=True)
        res_host[TOP_M:TOP_M + 1].copy_(best_f, non_blocking=True)
        res_host[TOP_M + 1:].copy_(best.to(torch.float64), non_blocking=True)
        torch.cuda.current_stream().synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_start.record(stream)
    for i in range(args.steps):
        V.copy_(V_host, non_blocking=True)
        prep.prepare(V, stream)
        step(args.warmup + args.steps + i)
        res_host[:TOP_M].copy_(f64, non_blocking=True)
        res_host[TOP_M:TOP_M + 1].copy_(best_f, non_blocking=True)
        res_host[TOP_M + 1:].copy_(best.to(torch.float64), non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e_stop.record(stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    lrq.check_status(status, "e2e steps")
    lrq.check_status(prep.dev_status, "lrq_prepare")
    e2e_val = float(world) * args.steps * S * N / e2e_s

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak_tf, _, peak_kind = _peaks()
    flops = 16.0 * R * N * S  # two complex r-contractions per evaluation (algorithmic)
    kern_avg_s = kern_ms * 1e-3 / args.steps
    if args.mode == "tc":
        roof = tc_roofline(flops, kern_avg_s, peak_tf, peak_kind)
    else:
        roof = fp32_roofline(flops, kern_avg_s)
    roof.update({"traffic": _traffic(args), "kernel": "score_tc_kernel" if args.mode == "tc" else "score_fp32_kernel",
                 "kernel_ms": kern_avg_s * 1e3, "flops_per_launch": flops})
    tc_err = score_error(V, C, ws, ws_r, mode, stream) if args.mode == "tc" else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16+e4m3" if args.mode == "tc" else "f32",
        "data": "synthetic", "config": _config(args.mode, world),
        "roofline": roof,
        "tc_error": tc_err,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": N * R * 8,
                "d2h_bytes_per_step": (TOP_M + 2) * 8},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "samples_to_best": None,
        "winner": {"f": win_f, "rank": win_rank, "candidate": win_idx},
    }
    if world == 1 and not args.no_learned:
        stb = learned_gain(dev, args.learned_n, args.learned_train, args.learned_eval, args.learned_steps)
        stb["hard"] = learned_gain(dev, args.learned_n, args.learned_train, args.learned_eval, args.learned_steps,
                                   hard=True)
        line["samples_to_best"] = stb
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(1, args.cpu_sample)
        cb.pop("seconds")
        one = cpu_baseline(2, max(4, args.cpu_sample // 16), threads=1)
        one.pop("seconds")
        cb["single_thread"] = one
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()



# ---------------------------------------------------------------------------
# the other workloads (one GPU; one JSON line each)
# ---------------------------------------------------------------------------
def _events(torch, k):
    return [torch.cuda.Event(enable_timing=True) for _ in range(k)]


def _line(metric, value, unit, args, ms, config, **extra):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "data": "synthetic", "config": config}
    out.update(extra)
    print(json.dumps(out), flush=True)


def learned_gain(dev, n, ntrain, neval, steps, hard=False):
    """Samples to 0.999 of the best of 2^16 uniform directions: the learned
    stream (16 mixture modes, then vMF draws; trained here on the GPU)
    against uniform sampling and against the fixed direction e_1 followed by
    uniform sampling.  hard=True draws sigma from the regime where the noise
    is comparable to the planted signal."""
    import torch

    from paper_2602_20376_gb300 import proposal as P
    sig = P.sigma_hard(n) if hard else P.SIGMA_EASY
    base = 2 * 10 ** 6 if hard else 10 ** 6
    t0 = time.perf_counter()
    V, lam = P.truncate_instances(n, range(base, base + ntrain + neval), device=dev, sigma_range=sig)
    Vg, feat = P.features(V, lam)
    targets = P.training_targets(Vg[:ntrain], P.K_ANGSYNC, 1 << 14, 555)
    model = P.Proposal(feat.shape[1], seed=0, device=dev)
    model.fit_standardizer(feat[:ntrain])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = P.train(model, feat[:ntrain], targets, steps, 64, 1e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    rows = P.evaluate(model, Vg[ntrain:], feat[ntrain:], P.K_ANGSYNC, 1 << 16, 777)
    med = lambda xs: sorted(xs)[len(xs) // 2]  # noqa: E731
    fin = lambda x: x if x != float("inf") else None  # noqa: E731
    return {"median_ratio": P.median_gain(rows), "median_ratio_vs_e1": P.median_gain(rows, baseline=3),
            "median_ratio_draws_only": P.median_gain([(r[0], r[1], r[4]) for r in rows]),
            "median_S_uniform": fin(med([r[1] for r in rows])), "median_S_learned": fin(med([r[2] for r in rows])),
            "median_S_e1_then_uniform": fin(med([r[3] for r in rows])),
            "reached_within_16": {"learned": P.reached_within(rows, 2, 16), "e1_then_uniform":
                                  P.reached_within(rows, 3, 16), "uniform": P.reached_within(rows, 1, 16)},
            "e1_reached": P.reached_within(rows, 3, 1),
            "level": 0.999, "S_max": 1 << 16,
            "reached": sum(1 for r in rows if r[2] != float("inf")), "instances": len(rows),
            "workload": "angular synchronisation Q = x x^H + sigma W, x on A_8^n, sigma ~ U[%g, %g], n=%d, "
                        "rank-4 truncation, K=8; %d training instances (top 1%% of 2^14 uniform directions "
                        "each), %d held-out" % (sig[0], sig[1], n, ntrain, neval),
            "train_steps": steps, "loss_first10": float(losses[:10].mean()), "loss_last10": float(losses[-10:].mean()),
            "data_s": t1 - t0, "train_s": t2 - t1,
            "kernels": "tcgen05 BF16 MLP fwd/bwd (mlp_gemm_tc_kernel), vMF NLL, Adam, vMF modes and sampler"}


def run_learned(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2602_20376_gb300 import lrq
    lrq.load()
    dev = torch.device("cuda", 0)
    ntrain, neval, steps = max(args.learned_train, 512), max(args.learned_eval, 256), max(args.learned_steps, 800)
    res = learned_gain(dev, args.learned_n, ntrain, neval, steps)
    res["hard"] = learned_gain(dev, args.learned_n, ntrain, neval, steps, hard=True)
    _line("median S_u/S_l to 0.999*best (learned vs uniform proposals)", res["median_ratio"], "x", args, None,
          {"workload": res["workload"]}, dtype="bf16", samples_to_best=res)


def run_exact(args):
    import torch

    from paper_2602_20376_gb300 import inputs, lrq
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    lrq.load()
    V64 = torch.from_numpy(inputs.factor(12, 2, seed=0)).to(dev)
    V32 = V64.to(torch.complex64)
    SS = 4096

    def step(i):
        out = lrq.enumerate_exact(V64, 3)
        smp = lrq.sample_score(V32, 3, S=SS, seed=1 + i, mode=lrq.LRQ_MODE_FP32, top_m=4)
        rs = lrq.rescore(V32, 3, smp["C"], smp["top_idx"])
        return out, rs

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    a, b = _events(torch, args.steps), _events(torch, args.steps)
    l0 = lrq.lrq_kernel_launches()
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            a[i].record()
            out, rs = step(args.warmup + i)
            b[i].record()
        torch.cuda.synchronize()
    ms = sum(x.elapsed_time(y) for x, y in zip(a, b)) / args.steps
    f_exact = float(out["f"].item())
    f_samp = float(rs["best_f"].item())
    # enumeration throughput on a larger arrangement: n = 64, r = 2, K = 3
    Vb = torch.from_numpy(inputs.factor(64, 2, seed=26, scales=(2.0, 1.0))).to(dev)
    lrq.enumerate_exact(Vb, 3)
    torch.cuda.synchronize()
    e0, e1 = _events(torch, 2)
    e0.record()
    big = lrq.enumerate_exact(Vb, 3)
    e1.record()
    torch.cuda.synchronize()
    big_ms = e0.elapsed_time(e1)
    sets = int(big["n_sets"].item())
    _line("exact rank-2 solves/s (n=12, r=2, K=3: vertex enumeration + 4096 sampled directions)", 1e3 / ms,
          "solves/s", args, ms, {"workload": "exact small instance: n=12, r=2, K=3, V ~ CN(0,1) complex128 seed 0; "
                                 "7164 index sets; S=4096 FP32 samples + top-4 FP64 rescore"},
          dtype="f64", gpu_launches=int(lrq.lrq_kernel_launches() - l0), clocks=clk.summary(),
          exact={"f_enumeration": f_exact, "f_best_of_4096": f_samp, "ratio": f_samp / f_exact,
                 "index_sets": int(out["n_sets"].item())},
          enumerate_n64={"index_sets": sets, "ms": big_ms, "sets_per_s": sets / (big_ms * 1e-3)})


def run_maxcut(args):
    import torch

    from paper_2602_20376_gb300 import inputs, lrq
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    lrq.load()
    n, SS, m = 1_000_000, 1 << 17, 64
    rowptr, colidx, labels = inputs.sbm_graph(n, 4.0, 8.0, seed=1)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colidx).to(dev)
    Q = lrq.laplacian_matrix(rp, ci)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    tr = lrq.truncate(Q, 3, max_iter=1000, seed=0, want_c128=False)
    t1.record()
    torch.cuda.synchronize()
    trunc_ms = t0.elapsed_time(t1)
    V = tr["V32"]
    lam = tr["lam"].cpu().numpy().tolist()
    cut = torch.zeros(1, dtype=torch.int64, device=dev)
    planted = torch.from_numpy(np.asarray(labels, dtype=np.uint8)).to(dev)
    lrq.lrq_cut_count(rp, ci, planted, cut)
    torch.cuda.synchronize()
    planted_cut = int(cut.item())
    ws = lrq.workspace(lrq.lrq_sample_score_workspace_size(n, 3, 3, SS, lrq.LRQ_MODE_TC, m), dev)
    wsr = lrq.workspace(lrq.lrq_rescore_workspace_size(n, 3, m), dev)

    null = args.sampler == "null"
    Cn = torch.empty((SS, 3), dtype=torch.complex64, device=dev)
    draws = torch.zeros(1, dtype=torch.int64, device=dev)
    nst = torch.zeros(1, dtype=torch.int32, device=dev)

    def step(i):
        if null:  # the null-vector sampler (randomised Algorithm 2) in place of the uniform sphere
            lrq.lrq_sample_null_directions(V, 3, 1 + i, SS, Cn, draws, nst)
            out = lrq.sample_score(V, 3, C=Cn, mode=lrq.LRQ_MODE_TC, top_m=m, ws=ws)
        else:
            out = lrq.sample_score(V, 3, C=None, S=SS, seed=1 + i, mode=lrq.LRQ_MODE_TC, top_m=m, ws=ws)
        rs = lrq.rescore(V, 3, out["C"], out["top_idx"], want_z=True, ws=wsr)
        row = torch.nonzero(out["top_idx"] == rs["best"]).flatten()[0]  # z rows follow top_idx
        lrq.lrq_cut_count(rp, ci, rs["z"][row], cut)
        return rs

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    a, b = _events(torch, args.steps), _events(torch, args.steps)
    l0 = lrq.lrq_kernel_launches()
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            a[i].record()
            rs = step(args.warmup + i)
            b[i].record()
        torch.cuda.synchronize()
    ms = sum(x.elapsed_time(y) for x, y in zip(a, b)) / args.steps
    edges = int(rowptr[-1]) // 2
    extra = {}
    if null:
        lrq.check_status(nst, "lrq_sample_null_directions")
        extra = {"sampler": "null-vector", "draws_last_step": int(draws.item()),
                 "rejected_fraction": 1.0 - SS / int(draws.item())}
    _line("Max-3-Cut candidate*n evals/s (SBM n=10^6, S=2^17, r=3)", SS * n / (ms * 1e-3), UNIT, args, ms,
          {"workload": "planted 3-partition SBM n=10^6, p_in n=4, p_out n=8 (seed 1), unit weights, CSR int32; "
                       "rank-3 FP64 Lanczos truncation of L; S=2^17 tensor-core-scored candidates (%s), "
                       "top-64 FP64 rescore, exact cut of the winner" % ("null-vector sampler" if null else "uniform sphere"),
           "edges": edges},
          dtype="f16+e4m3", gpu_launches=int(lrq.lrq_kernel_launches() - l0), clocks=clk.summary(),
          maxcut={"cut": int(cut.item()), "planted_cut": planted_cut, "edges": edges,
                  "cut_fraction": int(cut.item()) / edges, "best_f": float(rs["best_f"].item()),
                  "lambda": lam, "truncate_ms": trunc_ms, "lanczos_steps": tr["iters"], **extra})


def run_batched(args):
    import torch

    from paper_2602_20376_gb300 import inputs, lrq
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    lrq.load()
    g = inputs.rng(4)
    P, SS = 512, 8192
    probs, evals = [], 0
    tg = torch.Generator(device=dev)
    t_prep = time.perf_counter()
    for p in range(P):
        n = int(np.exp(g.uniform(np.log(64), np.log(8192))))
        r = int(g.integers(2, 7))
        Kp = int(g.choice([2, 3, 4, 8]))
        tg.manual_seed(1000 + p)
        V0 = torch.randn((n, r), generator=tg, device=dev, dtype=torch.complex128)
        Q = V0 @ V0.conj().T
        nrm = torch.linalg.eigvalsh(V0.conj().T @ V0)[-1].item()  # ||V V^H||_2
        G = torch.randn((n, n), generator=tg, device=dev, dtype=torch.complex128)
        H = 0.5 * (G + G.conj().T)
        hn = 2.0 * np.sqrt(n) * np.sqrt(0.5)  # semicircle edge of H: ||H||_2 ~ 2 sqrt(n / 2)
        Q += (0.05 * nrm / hn) * H
        del G, H
        tr = lrq.truncate(lrq.dense_matrix(Q), r, tol=1e-8, seed=p, want_c128=False)
        del Q
        probs.append(dict(V=tr["V32"], K=Kp, S=SS, seed=77 + p))
        evals += n * SS
    torch.cuda.synchronize()
    t_prep = time.perf_counter() - t_prep
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = lrq.BatchedPlan(probs, top_m=4, stream=stream)
        t_at = time.perf_counter()
        plan.autotune()
        t_at = time.perf_counter() - t_at
        plan.capture()
        for _ in range(args.warmup):
            plan.replay()
        stream.synchronize()
        a, b = _events(torch, args.steps), _events(torch, args.steps)
        ka, kb = _events(torch, args.steps), _events(torch, args.steps)
        l0 = lrq.lrq_kernel_launches()
        with ClockSampler(0) as clk:
            for i in range(args.steps):
                a[i].record(stream)
                plan.replay()
                b[i].record(stream)
            stream.synchronize()
        launches = lrq.lrq_kernel_launches() - l0
        # the persistent kernel alone (timing hook), outside the graph
        for i in range(args.steps):
            lrq.lrq_set_timing_events(ka[i], kb[i])
            plan.run()
            lrq.lrq_set_timing_events(None, None)
        stream.synchronize()
        lrq.check_status(plan.status, "batched")
    ms = sum(x.elapsed_time(y) for x, y in zip(a, b)) / args.steps
    kms = sum(x.elapsed_time(y) for x, y in zip(ka, kb)) / args.steps
    mixed = _mixed_subbatch(torch, lrq, probs, g, tg, dev, args) if args.exact_subbatch > 0 else None
    tiles = {}
    for p in range(P):
        tiles[plan.tile(p)] = tiles.get(plan.tile(p), 0) + 1
    flops = 16.0 * sum(q["V"].shape[0] * q["V"].shape[1] * SS for q in probs)
    _line("batched candidate*n evals/s (512 instances, one graph-captured persistent launch)", evals / (ms * 1e-3),
          UNIT, args, ms,
          {"workload": "512 instances: n = floor(exp(U[ln 64, ln 8192])), r ~ U{2..6}, K ~ U{2,3,4,8}, "
                       "Q = V V^H + sigma H (sigma = 0.05 ||V V^H||_2, H GUE-like scaled to ||H||_2 ~ 1), "
                       "FP64 Lanczos truncation to r; S=8192 drawn directions each, FP32 scoring, top-4 FP64 "
                       "rescore", "total_evals": evals},
          dtype="f32", gpu_launches=int(launches), clocks=clk.summary(),
          roofline=dict(fp32_roofline(flops, kms * 1e-3), traffic=None, kernel="batched_score_kernel",
                        kernel_ms=kms),
          batched={"prep_s": t_prep, "autotune_s": t_at, "tiles": tiles, "mixed": mixed})
    plan.close()


def _mixed_subbatch(torch, lrq, probs, g, tg, dev, args):
    """The labelled exact sub-batch: problems with n ~ U{8..48}, r = 2,
    K ~ U{2,3,4,8} (same instance recipe, truncated to r = 2) added to the 512
    sampled ones and solved by vertex enumeration in the same graph-captured
    persistent launch; returns the mixed launch's time and its size."""
    from paper_2602_20376_gb300 import lrq as L
    ex, sets = [], 0
    for p in range(args.exact_subbatch):
        n = int(g.integers(8, 49))
        Kp = int(g.choice([2, 3, 4, 8]))
        tg.manual_seed(5000 + p)
        V0 = torch.randn((n, 2), generator=tg, device=dev, dtype=torch.complex128)
        Q = V0 @ V0.conj().T
        nrm = torch.linalg.eigvalsh(V0.conj().T @ V0)[-1].item()
        G = torch.randn((n, n), generator=tg, device=dev, dtype=torch.complex128)
        Q += (0.05 * nrm / (2.0 * np.sqrt(n) * np.sqrt(0.5))) * 0.5 * (G + G.conj().T)
        tr = L.truncate(L.dense_matrix(Q), 2, tol=1e-10, seed=p, want_c128=False)
        ex.append(dict(V=tr["V32"], K=Kp, exact=True))
        BK = Kp // 2 if Kp % 2 == 0 else Kp
        N = n * BK
        sets += N * (N - 1) * (N - 2) // 6 + N
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = lrq.BatchedPlan(probs + ex, top_m=4, stream=stream)
        plan.capture()
        for _ in range(args.warmup):
            plan.replay()
        stream.synchronize()
        a, b = _events(torch, args.steps), _events(torch, args.steps)
        for i in range(args.steps):
            a[i].record(stream)
            plan.replay()
            b[i].record(stream)
        stream.synchronize()
        lrq.check_status(plan.status, "mixed batched")
    ms = sum(x.elapsed_time(y) for x, y in zip(a, b)) / args.steps
    plan.close()
    return {"ms_per_step": ms, "exact_problems": len(ex), "index_sets": sets,
            "workload": "exact sub-batch: n ~ U{8..48}, r = 2, K ~ U{2,3,4,8}, solved by vertex enumeration "
                        "(Algorithm 2) in the same launch as the 512 sampled instances"}


def run_rank1(args, hybrid=False):
    """Rank-1 Max-3-Cut at n = 10^6: rank-2 truncation, the two-eigenvector
    rounding vector, the exact sweep with every state's cut; with hybrid,
    greedy local search from the sweep's best-cut state."""
    import torch

    from paper_2602_20376_gb300 import inputs, lrq
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    lrq.load()
    n = 1_000_000
    rowptr, colidx, _ = inputs.sbm_graph(n, 4.0, 8.0, seed=1)
    rp = torch.from_numpy(rowptr).to(dev)
    ci = torch.from_numpy(colidx).to(dev)
    Q = lrq.laplacian_matrix(rp, ci)

    def step(ev=None):
        if ev:
            ev[0].record()
        tr = lrq.truncate(Q, 2, max_iter=1000, seed=0, want_c64=False)
        if ev:
            ev[1].record()
        q = lrq.two_eigvec_q(tr["V"], tr["lam"])
        out = lrq.rank1_sweep(q, 3, rp, ci)
        if ev:
            ev[2].record()
        gr = lrq.greedy_cut(rp, ci, 3, out["zcut"]) if hybrid else None
        if ev:
            ev[3].record()
        return tr, out, gr

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    l0 = lrq.lrq_kernel_launches()
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            tr, out, gr = step(evs[i])
        torch.cuda.synchronize()
    phase = lambda a, b: sum(e[a].elapsed_time(e[b]) for e in evs) / args.steps
    ms, trunc_ms, sweep_ms = phase(0, 3), phase(0, 1), phase(1, 2)
    edges = int(rowptr[-1]) // 2
    cut = int(out["cut"].item())
    info = {"f": float(out["f"].item()), "best_cut_along_sweep": cut, "edges": edges, "cut_fraction": cut / edges,
            "lambda": [float(x) for x in tr["lam"].cpu()], "truncate_ms": trunc_ms, "sweep_ms": sweep_ms,
            "lanczos_steps": tr["iters"],
            "paper_context": "the paper's rank-1 solver (ARPACK eigensolve + sweep with incremental scoring) takes "
                             "about 70 min on one CPU at n = 10^6 on a 5-regular graph (App., rank-1 at scale)"}
    what = "rank-2 FP64 Lanczos truncation of L, two-eigenvector rounding vector q = u1 + i u2, exact rank-1 " \
           "sweep (K=3), every sweep state's exact cut"
    if hybrid:
        hc = int(gr["cut"].item())
        info.update(hybrid_cut=hc, hybrid_cut_fraction=hc / edges, greedy_ms=phase(2, 3), greedy_rounds=gr["rounds"],
                    greedy_moves=gr["moves"], greedy_converged=gr["converged"])
        metric = "hybrid Max-3-Cut solves/s (SBM n=10^6: truncation + rank-1 sweep + greedy from its best cut)"
        what += ", then greedy local search to a local optimum"
    else:
        metric = "rank-1 Max-3-Cut solves/s (SBM n=10^6: truncation + exact sweep + best cut along it)"
    _line(metric, 1e3 / ms, "solves/s", args, ms,
          {"workload": "planted 3-partition SBM n=10^6, p_in n=4, p_out n=8 (seed 1); " + what, "edges": edges},
          dtype="f64", gpu_launches=int(lrq.lrq_kernel_launches() - l0), clocks=clk.summary(),
          **{"hybrid" if hybrid else "rank1": info})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["tc", "fp32", "bf16"], default="tc",
                    help="tc: tensor-core mode (F16 projections, FP8 hi + lo class sums); fp32: CUDA-core "
                         "mode; bf16: deprecated alias of tc")
    ap.add_argument("--candidates", type=int, default=S,
                    help="directions per step per GPU (default 2^16; smaller only for profiling runs)")
    ap.add_argument("--cpu-sample", type=int, default=256)
    ap.add_argument("--ref-sample", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the scoring kernel from an ncu capture")
    ap.add_argument("--workload", choices=["scale", "exact", "maxcut", "batched", "learned", "rank1", "hybrid"],
                    default="scale")
    ap.add_argument("--sampler", choices=["uniform", "null"], default="uniform",
                    help="direction sampler of the maxcut workload")
    ap.add_argument("--no-learned", action="store_true", help="leave samples_to_best out of the default line")
    ap.add_argument("--exact-subbatch", type=int, default=32,
                    help="exact problems (S = 0) added to the batched workload's mixed launch")
    ap.add_argument("--learned-n", type=int, default=4096)
    ap.add_argument("--learned-train", type=int, default=256)
    ap.add_argument("--learned-eval", type=int, default=256)
    ap.add_argument("--learned-steps", type=int, default=800)
    args = ap.parse_args()
    if args.mode == "bf16":
        args.mode = "tc"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "scale":
        run_ours(args)
    else:
        {"exact": run_exact, "maxcut": run_maxcut, "batched": run_batched, "learned": run_learned,
         "rank1": run_rank1, "hybrid": lambda a: run_rank1(a, hybrid=True)}[args.workload](args)


if __name__ == "__main__":
    main()
