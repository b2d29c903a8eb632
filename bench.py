#!/usr/bin/env python
"""Benchmark of the batched C2C FFT with fused two-sided ABFT.

One step = the size sweep: float32 and float64, forward and inverse, N = 2^3
.. 2^24, each call transforming 2^28 complex elements (2 GiB complex64 /
4 GiB complex128 in, the same out), with the whole hot path on (checksum
encode, transform, group check, correction kernel: ft_mode CORRECT).
Reported value: aggregate GB/s = (bytes in + bytes out) / time over the step.
The plain sweep (ABFT off) is timed the same way for the overhead figure.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU under torch.distributed.run; each rank runs
the same per-GPU workload on its own data (transforms are independent, no
exchange), value = bytes of all ranks / max time over ranks.
`--impl reference` times the CPU oracle on a bounded sample of the same sweep.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched C2C FFT GB/s & GFLOP/s (5N·log2N) vs HBM roofline; ABFT overhead %"
ELEMENTS = 1 << 28
SIZES = [1 << k for k in range(3, 25)]
DTYPES = [("float32", 8), ("float64", 16)]
DIRECTIONS = ["forward", "inverse"]
WORKLOAD = ("size sweep: f32+f64, forward+inverse, N=2^3..2^24, 2^28 complex elements per call, "
            "two-sided ABFT on (correct mode)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sizes", default="", help="comma list of log2 N (default: the full sweep)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged-batch comparison")
    ap.add_argument("--no-filter", action="store_true", help="skip the spectral-filter comparison")
    ap.add_argument("--study", action="store_true",
                    help="add the ABFT threshold (ROC) and group-size studies (about a minute)")
    ap.add_argument("--no-campaign", action="store_true", help="skip the fault-injection campaign (config 3)")
    ap.add_argument("--campaign-launches", type=int, default=400,
                    help="CORRECT-mode launches per (dtype, N) of the fault-injection campaign")
    ap.add_argument("--campaign-sizes", default="8,9,10,11,12,13,14,15,16,17,18,19,20",
                    help="comma list of log2 N of the fault-injection campaign")
    ap.add_argument("--no-config1", action="store_true", help="skip the N=256 x 4096 float32 timing (config 1)")
    ap.add_argument("--no-float-pairs", action="store_true",
                    help="skip the float64 sweep in float-pair arithmetic (FT off) against the FP64-pipe kernels")
    return ap.parse_args()


def configs(args):
    ks = [int(v) for v in args.sizes.split(",")] if args.sizes else [int(math.log2(n)) for n in SIZES]
    return [(dt, eb, d, 1 << k) for dt, eb in DTYPES for d in DIRECTIONS for k in ks]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "turbofft_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_HEADERS = ("tf_device.cuh", "tf_dd.cuh", "tf_types.h", "tf_dft_constants.h", "tf_instantiate.cuh", "tf_registry.h")


def src_hash(key=None):
    """Hash of the device code one kernel is built from: the shared kernel
    headers and, for a key like float64_col_n2048_ft, its translation unit."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2412_05824_gb300", "csrc")
    files = list(KERNEL_HEADERS)
    if key:
        dt, kind = key.split("_")[:2]
        files.append("tf_k_%s_%s.cu" % ("f32" if dt == "float32" else "f64", kind))
        if kind == "cl":
            files += ["tf_cluster.cuh", "tf_instantiate_cl.cuh"]
    for f in files:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(key):
    """Traffic per launch from a committed ncu summary, if it was taken on
    the current kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    ent = t.get(key)
    if ent and ent.get("src_hash") == src_hash(key):
        return ent.get("traffic_bytes_per_launch")
    return None


# ---------------------------------------------------------------------------
# multi-rank plumbing: one process per GPU, each rank a replica with its own
# seeded data (transforms are independent; no data-path collective)
# ---------------------------------------------------------------------------
def dist_env():
    """(world, rank, local_rank) from the torch.distributed.run environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(rank: int) -> int:
    """Seed of a rank's synthetic input: distinct data on every replica."""
    return 2 + 1000 * rank


def max_over_ranks(v: float, world: int, device=None) -> float:
    """Largest value over the ranks (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(bytes_per_rank_step: float, steps: int, max_ms: float, world: int) -> float:
    """Whole-job throughput: bytes moved by all ranks over the slowest rank's time."""
    return world * bytes_per_rank_step * steps / (max_ms * 1e-3) / 1e9


# ---------------------------------------------------------------------------
# the CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(args, sample_elems=1 << 22):
    import numpy as np

    import oracle
    import synth_signals as ss

    total_bytes = 0.0
    total_s = 0.0
    for dt, eb, d, n in configs(args):
        batch = max(1, sample_elems // n)
        x = ss.uniform_complex(2, batch, n, np.float32 if dt == "float32" else np.float64)
        t0 = time.perf_counter()
        oracle.fft(x, inverse=(d == "inverse"))
        total_s += time.perf_counter() - t0
        total_bytes += 2.0 * batch * n * eb
    return total_bytes / total_s / 1e9, total_s, oracle.last_threads()


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.lib()
    for _ in range(args.warmup):
        oracle_sample(args, 1 << 18)
    vals, secs = [], []
    threads = 1
    for _ in range(args.steps):
        v, s, threads = oracle_sample(args, 1 << 20)
        vals.append(v)
        secs.append(s)
    value = statistics.mean(vals)
    sample = ("oracle (float64 radix-2, OpenMP over the batch) on 2^20 elements per sweep "
              "configuration instead of 2^28; GB/s by the same byte formula")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * statistics.mean(secs), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "elements_per_call": ELEMENTS, "parallelism": "replicas"},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# secondary workloads: ragged batch and differentiable spectral filter, each
# against the plain fixed-size form on the same GPU
# ---------------------------------------------------------------------------
RAGGED_COUNT, RAGGED_LOG_LO, RAGGED_LOG_HI, RAGGED_SEED = 20000, 6, 16, 2024


def time_calls(fn, warmup, reps, stream):
    """Mean ms of fn() over `reps` calls (CUDA events on `stream`)."""
    import torch
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(reps):
        fn()
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / reps


def bench_ragged(args, dev, stream, rank, peaks):
    """20,000 complex64 transforms, sizes log-uniform in 2^6..2^16 (seeded),
    packed back to back: ragged plan (one CUDA graph, autotuned shapes, ABFT
    on) against one plain launch per size on the same transforms laid out
    contiguously by size."""
    import numpy as np
    import torch

    import paper_2412_05824_gb300 as tfl
    import synth_signals as ss

    sizes = ss.ragged_sizes(RAGGED_SEED, RAGGED_COUNT, RAGGED_LOG_LO, RAGGED_LOG_HI)
    offsets, extent = ss.ragged_offsets(sizes)
    x = ss.uniform_complex_torch(rank_seed(rank) + 100, 1, extent, "float32", device=dev).view(-1)
    y = torch.empty_like(x)
    # one launch of the persistent ragged kernel (the default), and the graph
    # of per-size kernels with autotuned shapes
    rag = {"correct": tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct"),
           "off": tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "off")}
    tfl.set_ragged_single_launch(False)
    tfl.set_autotune(True)
    t0 = time.perf_counter()
    try:
        rag_graph = {"correct": tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct"),
                     "off": tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "off")}
    finally:
        tune_s = time.perf_counter() - t0
        tfl.set_autotune(False)
        tfl.set_ragged_single_launch(True)

    # the same transforms, contiguous per size (gathered once on the device)
    order = np.argsort(sizes, kind="stable")
    ssz = sizes[order]
    starts_sorted = np.concatenate([[0], np.cumsum(ssz)[:-1]])
    delta = torch.from_numpy(offsets[order] - starts_sorted).to(dev)
    idx = torch.repeat_interleave(delta, torch.from_numpy(ssz).to(dev)) + torch.arange(extent, device=dev)
    xs = x[idx]
    ys = torch.empty_like(xs)
    groups = []
    for n in np.unique(ssz):
        first = int(np.searchsorted(ssz, n))
        cnt = int(np.sum(ssz == n))
        groups.append((int(n), cnt, int(starts_sorted[first])))
    per = {ft: [(tfl.Plan(n, c, "complex64", "forward", ft), o) for n, c, o in groups] for ft in ("off", "correct")}
    sp = stream.cuda_stream

    def run_per(ft):
        for pl, o in per[ft]:
            st = pl.exec_ptr(xs.data_ptr() + 8 * o, ys.data_ptr() + 8 * o, sp)
            if st != tfl.SUCCESS:
                raise RuntimeError("per-size exec failed: %d" % st)

    def run_rag(pl):
        def f():
            st = pl.exec_ptr(x.data_ptr(), y.data_ptr(), sp)
            if st != tfl.SUCCESS:
                raise RuntimeError("ragged exec failed: %d" % st)
        return f

    reps = max(args.steps, 5)
    ms = {"ragged_ft": time_calls(run_rag(rag["correct"]), args.warmup, reps, stream),
          "ragged_plain": time_calls(run_rag(rag["off"]), args.warmup, reps, stream),
          "ragged_ft_graph_autotuned": time_calls(run_rag(rag_graph["correct"]), args.warmup, reps, stream),
          "ragged_plain_graph_autotuned": time_calls(run_rag(rag_graph["off"]), args.warmup, reps, stream),
          "per_size_plain": time_calls(lambda: run_per("off"), args.warmup, reps, stream),
          "per_size_ft": time_calls(lambda: run_per("correct"), args.warmup, reps, stream)}
    rep_ft = rag["correct"].report()
    # same transforms, same accuracy: ragged ABFT output against the per-size plain output
    rag["correct"].exec_ptr(x.data_ptr(), y.data_ptr(), sp)
    run_per("off")
    torch.cuda.synchronize()
    diff = float(torch.linalg.vector_norm(y[idx] - ys) / torch.linalg.vector_norm(ys))
    nbytes = 16.0 * extent
    members = rag_graph["correct"].members()
    single = rag["correct"].info()["single_launch"] == 1
    out = {"workload": "%d complex64 forward transforms, sizes 2^%d..2^%d log-uniform (seed %d), packed, "
                       "uniform[-1,1) data" % (RAGGED_COUNT, RAGGED_LOG_LO, RAGGED_LOG_HI, RAGGED_SEED),
           "elements": extent, "bytes_per_exec": nbytes, "reps": reps,
           "gbs": {k: round(nbytes / (v * 1e-3) / 1e9, 1) for k, v in ms.items()},
           "ms": {k: round(v, 4) for k, v in ms.items()},
           "hbm_frac_ragged_ft": round(nbytes / (ms["ragged_ft"] * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
           "abft_overhead_pct": round(100.0 * (ms["ragged_ft"] / ms["ragged_plain"] - 1.0), 2),
           "vs_per_size_plain": round(ms["per_size_plain"] / ms["ragged_ft"], 4),
           "plain_vs_per_size_plain": round(ms["per_size_plain"] / ms["ragged_plain"], 4),
           "single_launch": single,
           "graph_autotune_s": round(tune_s, 2),
           "shapes": [[m["n"], m["batch"], m["radix"][0], m["block"][0], m["per_block"][0]] for m in members],
           "shapes_columns": ["n", "count", "radix_pass0", "threads_pass0", "per_block_pass0"],
           "graph_launches_per_exec": 1,
           "kernel_launches_per_exec": 1 if single else sum(2 * m["num_passes"] for m in members),
           "kernel_launches_per_exec_graph_form": sum(2 * m["num_passes"] for m in members),
           "rel_l2_vs_per_size_plain": diff,
           "detected_last_exec": rep_ft["detected"]}
    for pl in list(rag.values()) + list(rag_graph.values()) + [q for v in per.values() for q, _ in v]:
        pl.close()
    del x, y, xs, ys, idx
    torch.cuda.empty_cache()
    return out


def bench_filter(args, dev, stream):
    """Differentiable spectral filter y = iFFT(W * FFT(x)), x [64, 128, 4096]
    complex64, loss = sum |y|^2, forward + backward: through the autograd
    Functions (ABFT on / off) against the same four transforms issued as
    plain fixed-size execs with the chain rule written out."""
    import torch

    import paper_2412_05824_gb300 as tfl
    from paper_2412_05824_gb300 import autograd as ag
    import synth_signals as ss

    B, C, N = 64, 128, 4096
    x0 = ss.uniform_complex_torch(7, B * C, N, "float32", device=dev).view(B, C, N)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    w0 = torch.complex(torch.randn(C, N, generator=g, device=dev), torch.randn(C, N, generator=g, device=dev))
    w0 = w0 * (N ** -0.5 / 2 ** 0.5)

    def autograd_step(ft):
        def f():
            x = x0.detach().requires_grad_(True)
            w = w0.detach().requires_grad_(True)
            loss = ag.spectral_filter(x, w, ft).abs().pow(2).sum()
            loss.backward()
            return x.grad, w.grad
        return f

    plans = {d: tfl.Plan(N, B * C, "complex64", d, "off") for d in ("forward", "inverse", "forward_scaled",
                                                                   "inverse_unscaled")}

    def plain_step():
        X = plans["forward"].exec(x0.view(B * C, N)).view(B, C, N)
        Z = X * w0
        Y = plans["inverse"].exec(Z.view(B * C, N)).view(B, C, N)
        gY = 2.0 * Y
        gZ = plans["forward_scaled"].exec(gY.view(B * C, N)).view(B, C, N)
        gw = (X.conj() * gZ).sum(0)
        gX = w0.conj() * gZ
        gx = plans["inverse_unscaled"].exec(gX.view(B * C, N)).view(B, C, N)
        return gx, gw

    def torch_step():
        x = x0.detach().requires_grad_(True)
        w = w0.detach().requires_grad_(True)
        loss = torch.fft.ifft(torch.fft.fft(x) * w).abs().pow(2).sum()
        loss.backward()
        return x.grad, w.grad

    reps = max(args.steps, 5)
    ms = {"autograd_ft": time_calls(autograd_step("correct"), args.warmup, reps, stream),
          "autograd_plain": time_calls(autograd_step("off"), args.warmup, reps, stream),
          "plain_fixed_size": time_calls(plain_step, args.warmup, reps, stream),
          "torch_fft_context": time_calls(torch_step, args.warmup, reps, stream)}
    gx_a, gw_a = autograd_step("correct")()
    gx_p, gw_p = plain_step()
    gx_t, gw_t = torch_step()

    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    out = {"workload": "x [64,128,4096] complex64 uniform[-1,1), W [128,4096] complex normal (std 1/64), "
                       "loss = sum|iFFT(W*FFT(x))|^2, forward + backward",
           "ms": {k: round(v, 4) for k, v in ms.items()},
           "autograd_overhead_vs_plain_pct": round(100.0 * (ms["autograd_plain"] / ms["plain_fixed_size"] - 1.0), 2),
           "abft_overhead_pct": round(100.0 * (ms["autograd_ft"] / ms["autograd_plain"] - 1.0), 2),
           "transforms_per_step": 4,
           "rel_l2_grad_x_autograd_vs_plain": rel(gx_a, gx_p),
           "rel_l2_grad_w_autograd_vs_plain": rel(gw_a, gw_p),
           "rel_l2_grad_x_vs_torch_fft": rel(gx_a, gx_t),
           "note": "torch_fft_context is the same step through torch.fft, for context only"}
    for pl in plans.values():
        pl.close()
    ag._plans.clear()
    return out


CAMPAIGN_ELEMENTS = 1 << 26


def bench_campaign(args, peaks):
    """Config 3: ABFT on, float32 and float64, N = 2^8..2^20, 2^26 elements
    per launch; 1 in every 100 launches carries one seeded bit flip (Sec. 5.3
    protocol).  Per (dtype, N): false alarms over the clean launches,
    detections / corrections / escapes of the injected faults, and the time of
    clean and injected runs against the plain path."""
    from paper_2412_05824_gb300 import abft_study

    rows = []
    t0 = time.perf_counter()
    for dt in ("complex64", "complex128"):
        for k in [int(v) for v in args.campaign_sizes.split(",") if v]:
            r = abft_study.campaign(1 << k, dt, elements=CAMPAIGN_ELEMENTS, launches=args.campaign_launches,
                                    every=100, timing_launches=200 if dt == "complex64" else 100)
            rows.append(r)
    tot = {key: sum(r[key] for r in rows) for key in ("clean_launches", "false_alarm_launches",
                                                      "false_alarm_groups", "faults", "breaking", "detected",
                                                      "detected_breaking", "located_right", "corrected",
                                                      "uncorrectable")}
    escapes = [dict(e, n=r["n"], dtype=r["dtype"]) for r in rows for e in r["escapes"]]
    cols = ["dtype", "log2N", "clean_launches", "false_alarm_launches", "faults", "breaking", "detected",
            "corrected", "uncorrectable", "escapes", "ms_plain", "ms_ft_clean", "ms_ft_injected",
            "overhead_pct_vs_plain", "injected_overhead_pct_vs_clean"]
    table = [[r["dtype"][7:], int(math.log2(r["n"])), r["clean_launches"], r["false_alarm_launches"], r["faults"],
              r["breaking"], r["detected"], r["corrected"], r["uncorrectable"], len(r["escapes"]), r["ms_plain"],
              r["ms_ft_clean"], r["ms_ft_injected"], r["overhead_pct_vs_plain"], r["injected_overhead_pct_vs_clean"]]
             for r in rows]
    per_dt = {}
    for dt in ("complex64", "complex128"):
        rr = [r for r in rows if r["dtype"] == dt]
        if rr:
            tp, tc, ti = (sum(r[k] for r in rr) for k in ("ms_plain", "ms_ft_clean", "ms_ft_injected"))
            per_dt[dt] = {"overhead_pct_vs_plain": round(100.0 * (tc / tp - 1.0), 2),
                          "injected_overhead_pct_vs_clean": round(100.0 * (ti / tc - 1.0), 2),
                          "injected_overhead_pct_vs_plain": round(100.0 * (ti / tp - 1.0), 2)}
    return {"workload": "ABFT on (correct), float32 + float64, N=2^8..2^20, %d elements per launch, "
                        "uniform[-1,1) (seed 3), 1 in 100 launches with one seeded bit flip (seed 4): "
                        "exponent bit 30/62 or mantissa bit 10-20/40-50" % CAMPAIGN_ELEMENTS,
            "launches_per_config": args.campaign_launches, "totals": tot,
            "detection_rate_breaking": (tot["detected_breaking"] / tot["breaking"]) if tot["breaking"] else None,
            "correction_rate_detected": (tot["corrected"] / tot["detected"]) if tot["detected"] else None,
            "escapes": escapes, "per_dtype_time": per_dt,
            "all_within_bar_after": all(r["all_within_bar_after"] for r in rows),
            "columns": cols, "rows": table, "seconds": round(time.perf_counter() - t0, 1),
            "bar_reference": "breaking / within bar measured per transform against the GPU's own clean "
                             "plain-path output"}


def bench_float_pairs(args, stream, peaks, x, y, workspace, sizes):
    """float64 sweep with ABFT off: the float-pair plans (float64 data,
    float arithmetic) against the FP64-pipe plans, same buffers, forward and
    inverse, 2^28 elements per call."""
    import paper_2412_05824_gb300 as tfl

    rows = []
    tot = {"fp64": 0.0, "pairs": 0.0}
    nbytes = 2.0 * ELEMENTS * 16
    for d in DIRECTIONS:
        for n in sizes:
            ms = {}
            for arith, structure in (("fp64", "default"), ("pairs", "float_pairs")):
                p = tfl.Plan(n, ELEMENTS // n, "complex128", d, "off", structure=structure)
                p.set_workspace(workspace)

                def f():
                    st = p.exec_ptr(x.data_ptr(), y.data_ptr(), stream.cuda_stream)
                    if st != tfl.SUCCESS:
                        raise RuntimeError("exec failed: %d" % st)
                ms[arith] = time_calls(f, args.warmup, max(args.steps, 3), stream)
                tot[arith] += ms[arith]
                p.close()
            rows.append([d[:3], int(math.log2(n)), round(nbytes / (ms["fp64"] * 1e-3) / 1e9, 1),
                         round(nbytes / (ms["pairs"] * 1e-3) / 1e9, 1), round(ms["fp64"] / ms["pairs"], 3),
                         round(nbytes / (ms["pairs"] * 1e-3) / 1e9 / peaks["hbm_gbs"], 3)])
    nall = nbytes * len(rows)
    return {"workload": "float64 C2C, ABFT off, N=2^%d..2^%d, forward + inverse, 2^28 elements per call"
                        % (int(math.log2(sizes[0])), int(math.log2(sizes[-1]))),
            "columns": ["dir", "log2N", "fp64_GBs", "float_pairs_GBs", "speedup", "float_pairs_hbm_frac"],
            "rows": rows,
            "sweep_gbs": {k: round(nall / (v * 1e-3) / 1e9, 1) for k, v in tot.items()},
            "speedup": round(tot["fp64"] / tot["pairs"], 3)}


def bench_config1(args, dev, stream, peaks):
    """Config 1: plain float32 forward, N = 256, batch 4096 (8 MiB in, 8 MiB
    out).  The working set fits in L2, so it is timed two ways: over a
    rotating pool of input/output pairs larger than 4x the L2 (every launch
    reads and writes HBM), and on one pair (L2-resident).  Median of >= 100
    launches, each bracketed by CUDA events, plus the mean of back-to-back
    launches."""
    import torch

    import paper_2412_05824_gb300 as tfl
    import synth_signals as ss

    n, batch = 256, 4096
    nbytes = 2.0 * n * batch * 8
    pool_n = 34  # 34 x 16 MiB = 570 MB > 4 x 129 MB L2
    xs = [ss.uniform_complex_torch(1 + i, batch, n, "float32", device=dev) for i in range(pool_n)]
    ys = [torch.empty_like(v) for v in xs]
    pl = tfl.Plan(n, batch, "complex64", "forward", "off")
    sp = stream.cuda_stream
    reps = max(100, 4 * pool_n)

    def per_launch(rotate):
        ts = []
        for _ in range(5):
            pl.exec_ptr(xs[0].data_ptr(), ys[0].data_ptr(), sp)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i, (a, b) in enumerate(evs):
            k = i % pool_n if rotate else 0
            a.record(stream)
            pl.exec_ptr(xs[k].data_ptr(), ys[k].data_ptr(), sp)
            b.record(stream)
        torch.cuda.synchronize()
        ts = [a.elapsed_time(b) for a, b in evs]
        return statistics.median(ts)

    def back_to_back(rotate):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(reps):
            k = i % pool_n if rotate else 0
            pl.exec_ptr(xs[k].data_ptr(), ys[k].data_ptr(), sp)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms = {"hbm_rotating_median": per_launch(True), "l2_resident_median": per_launch(False),
          "hbm_rotating_back_to_back": back_to_back(True), "l2_resident_back_to_back": back_to_back(False)}
    pl.close()
    del xs, ys
    torch.cuda.empty_cache()
    ideal_us = nbytes / (peaks["hbm_gbs"] * 1e9) * 1e6
    return {"workload": "plain float32 forward C2C, N=256, batch 4096, uniform[-1,1) (seeds 1..%d)" % pool_n,
            "bytes_in_out": nbytes, "reps": reps, "pool": "%d input/output pairs (%.0f MB > 4x L2)"
            % (pool_n, pool_n * nbytes / 1e6),
            "us": {k: round(1e3 * v, 3) for k, v in ms.items()},
            "gbs": {k: round(nbytes / (v * 1e-3) / 1e9, 1) for k, v in ms.items()},
            "hbm_frac": {k: round(nbytes / (v * 1e-3) / 1e9 / peaks["hbm_gbs"], 4) for k, v in ms.items()},
            "ideal_us_at_hbm_peak": round(ideal_us, 3)}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2412_05824_gb300 as tfl
    import synth_signals as ss

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfgs = configs(args)
    peaks, peak_src = measured_peaks()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # inputs resident in HBM (seeded, per rank), one buffer per dtype
    bufs = {}
    for dt, eb in DTYPES:
        x = ss.uniform_complex_torch(rank_seed(rank), 1, ELEMENTS, dt, device=dev)
        bufs[dt] = (x, torch.empty_like(x))
    workspace = torch.empty(ELEMENTS, dtype=torch.complex128, device=dev)  # two-pass intermediate

    def make_plans(ft):
        plans = {}
        for dt, eb, d, n in cfgs:
            p = tfl.Plan(n, ELEMENTS // n, "complex64" if dt == "float32" else "complex128", d, ft)
            p.set_workspace(workspace)
            plans[(dt, d, n)] = p
        return plans

    plans_ft = make_plans("correct")
    plans_plain = make_plans("off")
    stream = torch.cuda.current_stream(dev)

    def step(plans, record=None):
        evs = []
        for dt, eb, d, n in cfgs:
            x, y = bufs[dt]
            p = plans[(dt, d, n)]
            if record is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                evs.append(e)
            st = p.exec_ptr(x.data_ptr(), y.data_ptr(), stream.cuda_stream)
            if st != tfl.SUCCESS:
                raise RuntimeError("exec failed: %d" % st)
        if record is not None:
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            evs.append(e)
            record.append(evs)

    step_bytes = sum(2.0 * ELEMENTS * eb for dt, eb, d, n in cfgs)

    def timed(plans, sampler=None):
        for _ in range(args.warmup):
            step(plans)
        barrier()
        rec = []
        if sampler:
            sampler.start()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(plans, rec)
        t1.record(stream)
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = t0.elapsed_time(t1)
        per_cfg = [statistics.mean(r[i].elapsed_time(r[i + 1]) for r in rec) for i in range(len(cfgs))]
        return ms, per_cfg, clocks

    sampler = ClockSampler(local) if rank == 0 else None
    ms_ft, per_ft, clocks = timed(plans_ft, sampler)
    ms_plain, per_plain, _ = timed(plans_plain)
    # fault-tolerance outcome of the last exec of every plan: a clean run
    fa = sum(plans_ft[(dt, d, n)].report()["detected"] for dt, eb, d, n in cfgs)

    ms_ft = max_over_ranks(ms_ft, world, dev)
    ms_plain = max_over_ranks(ms_plain, world, dev)
    value = aggregate_gbs(step_bytes, args.steps, ms_ft, world)
    value_plain = aggregate_gbs(step_bytes, args.steps, ms_plain, world)

    # dominant kernel: the kernel with the largest share of one profiled step
    # (CUDA events on the exec's stream around every launch), then its
    # average duration over those launches
    kernel_ms, kernel_launch = {}, {}
    step_kernel_total = 0.0
    for dt2, eb2, d2, n2 in cfgs:
        pl = plans_ft[(dt2, d2, n2)]
        pl.set_profiling(True)
        x2, y2 = bufs[dt2]
        pl.exec_ptr(x2.data_ptr(), y2.data_ptr(), stream.cuda_stream)
        inf = pl.info()
        for (ps, corr, msk) in pl.kernel_times():
            kind = "fix" if corr else ("sp" if inf["num_passes"] == 1 else ("col" if ps == 0 else "row"))
            sub = inf["sub_n"][ps]
            if inf["cluster"] and not corr:
                kind, sub = "cl", n2  # both phases in one cluster kernel
            key = "%s_%s_n%d_ft" % (dt2, kind, sub)
            kernel_ms[key] = kernel_ms.get(key, 0.0) + msk
            kernel_launch.setdefault(key, []).append((msk, eb2, sub))
            step_kernel_total += msk
        pl.set_profiling(False)
    kname = max((k for k in kernel_ms if not k.split("_")[1] == "fix"), key=lambda k: kernel_ms[k])
    launches = kernel_launch[kname]
    kms = statistics.mean(m for m, _, _ in launches)
    eb = launches[0][1]
    ns_dom = launches[0][2]
    dt = kname.split("_")[0]
    fix_ms = statistics.mean([m for k, v in kernel_launch.items() if "_fix_" in k for m, _, _ in v] or [0.0])
    bytes_launch = 2.0 * ELEMENTS * eb
    flops_launch = 5.0 * ELEMENTS * math.log2(ns_dom)
    share = kernel_ms[kname] / step_kernel_total
    fp64_peak = None
    try:
        fp64_peak = tfl.fma_peak("complex128", 1.0, stream)
    except Exception:
        fp64_peak = None
    if dt == "float32":
        ach = bytes_launch / (kms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": ncu_traffic(kname),
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        if fp64_peak:
            peak_tf, psrc = fp64_peak, ("measured in this run: turbofft_fma_peak(F64), double FMA loop over "
                                        "every SM, 1 s of ~50 ms launches, best launch")
        else:
            peak_tf, psrc = 1.25, "fallback: FP64 nominal 1.25 TFLOP/s (recipe unit counts)"
        ach = flops_launch / (kms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak_tf, 4), "unit": "TFLOP/s",
                "frac": round(ach / peak_tf, 4), "traffic": ncu_traffic(kname),
                "peak_source": psrc,
                "hbm_gbs_achieved": round(bytes_launch / (kms * 1e-3) / 1e9, 1),
                "hbm_frac": round(bytes_launch / (kms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
    roof.update({"kernel": kname, "share_of_step": round(share, 4), "launches_per_step": len(launches),
                 "kernel_ms": round(kms, 4), "correction_kernel_ms": round(fix_ms, 4),
                 "algorithmic_bytes_per_launch": bytes_launch, "algorithmic_flops_per_launch": flops_launch})

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        host = {}
        for dt2, eb2 in DTYPES:
            hx = bufs[dt2][0].cpu().pin_memory()
            host[dt2] = (hx, torch.empty_like(hx).pin_memory())
        for _ in range(1):
            for dt2, eb2, d2, n2 in cfgs:
                hx, hy = host[dt2]
                plans_ft[(dt2, d2, n2)].exec_host(hx, hy)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for dt2, eb2, d2, n2 in cfgs:
                hx, hy = host[dt2]
                plans_ft[(dt2, d2, n2)].exec_host(hx, hy)
        barrier()
        el = max_over_ranks(time.perf_counter() - t0, world, dev)
        h2d = sum(ELEMENTS * eb2 for dt2, eb2, d2, n2 in cfgs)
        e2e = {"value": round(world * step_bytes * args.steps / el / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
               "note": "turbofft_exec_host: pinned host in/out, H2D + transform + D2H pipelined in chunks"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, s, th = oracle_sample(args, 1 << 19)
        cpu = {"value": round(v, 4), "unit": "GB/s", "cores": th, "kind": "oracle",
               "sample": "oracle (float64 radix-2, OpenMP) on 2^19 elements per sweep configuration "
                         "(%.1f s of CPU work); GB/s by the same byte formula" % s}

    ragged = bench_ragged(args, dev, stream, rank, peaks) if not args.no_ragged else None
    config1 = bench_config1(args, dev, stream, peaks) if not args.no_config1 else None
    f64_sizes = sorted({n for dt2, eb2, d2, n in cfgs if dt2 == "float64"})
    float_pairs = (bench_float_pairs(args, stream, peaks, bufs["float64"][0], bufs["float64"][1], workspace,
                                     f64_sizes) if (not args.no_float_pairs and f64_sizes) else None)
    campaign = bench_campaign(args, peaks) if (not args.no_campaign and rank == 0) else None
    sfilter = bench_filter(args, dev, stream) if not args.no_filter else None
    study = None
    if args.study and rank == 0:
        from paper_2412_05824_gb300 import abft_study
        # ROC at several lengths (signals per length scaled so each exec
        # stays small), and the ABFT level / group-size ablation
        roc_cases = [(256, 2000), (1024, 2000), (4096, 1000), (1 << 16, 128)]
        study = {"roc": [abft_study.roc(n, b, dt) for n, b in roc_cases for dt in ("complex64", "complex128")],
                 "group_size": [abft_study.ablation(n, dt) for n, dt in
                                ((8, "complex64"), (16, "complex64"), (32, "complex64"), (8, "complex128"),
                                 (16, "complex128"), (1024, "complex64"), (4096, "complex64"),
                                 (1024, "complex128"))]}

    launches_per_step = 0
    for dt2, eb2, d2, n2 in cfgs:
        inf2 = plans_ft[(dt2, d2, n2)].info()
        # cluster: kernel + correction; whole-transform checks: two passes,
        # check, two recompute kernels; else a kernel and a correction per pass
        launches_per_step += 2 if inf2["cluster"] else (5 if inf2["transform_checks"] else inf2["num_passes"] * 2)
    sweep = []
    for i, (dt2, eb2, d2, n2) in enumerate(cfgs):
        b = 2.0 * ELEMENTS * eb2
        inf2 = plans_ft[(dt2, d2, n2)].info()
        sweep.append([dt2[5:], d2[:3], int(math.log2(n2)), round(b / (per_ft[i] * 1e-3) / 1e9, 1),
                      round(b / (per_plain[i] * 1e-3) / 1e9, 1),
                      round(5.0 * ELEMENTS * math.log2(n2) / (per_ft[i] * 1e-3) / 1e9, 1),
                      round(b / (per_ft[i] * 1e-3) / 1e9 / peaks["hbm_gbs"], 3),
                      "cl%d" % inf2["cluster"] if inf2["cluster"] else "x".join(
                          str(inf2["sub_n"][q]) for q in range(inf2["num_passes"]))])
    per_dtype = {}
    for dt2, eb2 in DTYPES:
        idx = [i for i, c in enumerate(cfgs) if c[0] == dt2]
        if idx:
            b = sum(2.0 * ELEMENTS * eb2 for _ in idx)
            per_dtype[dt2] = {"ft_gbs": round(b / (sum(per_ft[i] for i in idx) * 1e-3) / 1e9, 1),
                              "plain_gbs": round(b / (sum(per_plain[i] for i in idx) * 1e-3) / 1e9, 1)}
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_ft / args.steps, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "elements_per_call": ELEMENTS,
                           "sizes": "2^%d..2^%d" % (int(math.log2(cfgs[0][3])), int(math.log2(cfgs[-1][3]))),
                           "ft_mode": "correct", "l2": "inputs 2-4 GiB per call, larger than the 129 MB L2",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps,
                "clocks": clocks,
                "plain_value": round(value_plain, 2),
                "abft_overhead_pct": round(100.0 * (ms_ft / ms_plain - 1.0), 2),
                "false_alarms_last_step": fa,
                "per_dtype": per_dtype,
                "sweep_columns": ["dtype", "dir", "log2N", "ft_GBs", "plain_GBs", "ft_GFLOPs", "ft_hbm_frac",
                                  "passes"],
                "sweep": sweep,
                "ragged": ragged,
                "spectral_filter": sfilter,
                "config1": config1,
                "float64_float_pairs": float_pairs,
                "ft_campaign": campaign,
                "fp64_fma_peak_tflops": round(fp64_peak, 4) if fp64_peak else None}
        if study is not None:
            line["abft_study"] = study
        print(json.dumps(line), flush=True)
    for pl in list(plans_ft.values()) + list(plans_plain.values()):
        pl.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
