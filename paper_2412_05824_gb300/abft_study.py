"""Threshold and group-size studies of the fused two-sided ABFT, run through
the C ABI (argument marshalling and bookkeeping only; every transform and
check runs in the library's kernels).

roc():       detection and false-alarm rates as the detection threshold is
             scaled (the delta sweep of Sec. 5.3.1, Fig. 19): normal-distributed
             signals, one seeded bit flip per faulty exec (Sec. 5.3.1 protocol),
             DETECT mode.  A fault counts as detected when the faulty exec
             flags more groups than the clean exec at the same threshold.
             Faults are also classed by whether they break the accuracy bar
             (relative L2 error of the faulty transform above 2e-6 log2 N for
             complex64, 5e-15 log2 N for complex128).
ablation():  time of the transform with checksums for 1..16 transactions per
             checksum group against the plain transform (the thread-block
             group-size study of Sec. 4.3, Figs. 16-17).
"""
from __future__ import annotations

import math

import numpy as np


def _bar(dtype: str, n: int) -> float:
    return (2e-6 if dtype == "complex64" else 5e-15) * max(1, int(math.log2(n)))


def _normal_device(seed: int, batch: int, n: int, dtype: str):
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    rdt = torch.float32 if dtype == "complex64" else torch.float64
    re = torch.randn(batch, n, generator=g, device="cuda", dtype=rdt)
    im = torch.randn(batch, n, generator=g, device="cuda", dtype=rdt)
    return torch.complex(re, im).contiguous()


def roc(n: int = 1024, batch: int = 2000, dtype: str = "complex64", faults: int = 1000,
        scales=(0.0625, 0.125, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0), seed: int = 7) -> dict:
    """Rates per threshold scale; see the module docstring."""
    import torch

    import paper_2412_05824_gb300 as tfl

    x = _normal_device(seed, batch, n, dtype)
    off = tfl.Plan(n, batch, dtype, "forward", "off")
    ref = off.exec(x)
    det = tfl.Plan(n, batch, dtype, "forward", "detect")
    info = det.info()
    rng = np.random.default_rng(seed)
    hi_bits = 32 if dtype == "complex64" else 64
    sites = []
    for _ in range(faults):
        p = int(rng.integers(0, info["num_passes"]))
        sites.append((int(rng.integers(0, batch)), p, int(rng.integers(0, info["stages"][p] + 1)),
                      int(rng.integers(0, n)), int(rng.integers(0, 2)), int(rng.integers(0, hi_bits))))
    bar = _bar(dtype, n)
    # which faults break the accuracy bar (threshold-independent: plain plan)
    breaking = []
    for (tr, p, st, el, comp, bit) in sites:
        off.inject(tr, p, st, el, comp, bit)
        y = off.exec(x)
        d = torch.linalg.vector_norm(y[tr] - ref[tr]) / torch.linalg.vector_norm(ref[tr])
        breaking.append(not bool(torch.isfinite(d)) or float(d) > bar)
    rows = []
    out = torch.empty_like(ref)
    for s in scales:
        det.set_threshold_scale(float(s))
        det.exec(x, out)
        clean = det.report()
        flagged = []
        for (tr, p, st, el, comp, bit) in sites:
            det.inject(tr, p, st, el, comp, bit)
            det.exec(x, out)
            flagged.append(det.report()["detected"] > clean["detected"])
        nb = sum(breaking)
        rows.append({
            "threshold_scale": s,
            "false_alarm_rate": clean["detected"] / max(1, clean["groups_checked"]),
            "detection_rate": sum(flagged) / len(sites),
            "detection_rate_breaking": (sum(f for f, b in zip(flagged, breaking) if b) / nb) if nb else None,
            "missed_breaking": sum(1 for f, b in zip(flagged, breaking) if b and not f),
        })
    det.set_threshold_scale(1.0)
    off.close()
    det.close()
    return {"n": n, "batch": batch, "dtype": dtype, "faults": faults, "breaking_faults": sum(breaking),
            "signals": "complex normal (seeded torch generator)", "rows": rows}


def ablation(n: int, dtype: str = "complex64", elements: int = 1 << 26, groups=(1, 2, 4, 8, 16),
             reps: int = 10) -> dict:
    """ms per exec for each transactions-per-group setting against ABFT off."""
    import torch

    import paper_2412_05824_gb300 as tfl
    import synth_signals as ss

    batch = max(1, elements // n)
    x = ss.uniform_complex_torch(3, batch, n, "float32" if dtype == "complex64" else "float64")
    y = torch.empty_like(x)
    s = torch.cuda.current_stream()

    def timed(plan):
        for _ in range(3):
            plan.exec_ptr(x.data_ptr(), y.data_ptr(), s.cuda_stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(reps):
            plan.exec_ptr(x.data_ptr(), y.data_ptr(), s.cuda_stream)
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    plain = tfl.Plan(n, batch, dtype, "forward", "off")
    base = timed(plain)
    plain.close()
    ft = tfl.Plan(n, batch, dtype, "forward", "correct")
    rows = []
    for t in groups:
        ft.set_group_transactions(t)
        ms = timed(ft)
        rows.append({"transactions": t, "ms": round(ms, 4), "overhead_pct": round(100.0 * (ms / base - 1.0), 2),
                     "detected": ft.report()["detected"]})
    ft.close()
    return {"n": n, "dtype": dtype, "batch": batch, "plain_ms": round(base, 4), "rows": rows}
