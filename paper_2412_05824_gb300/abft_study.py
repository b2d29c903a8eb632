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
             group-size study of Sec. 4.3, Figs. 16-17), with the
             thread-level checks of Sec. 4.2.1 beside them where one thread
             holds a whole transform.
campaign():  the fault-injection campaign of Sec. 5.3: a run of launches in
             CORRECT mode on uniform[-1,1) signals in which 1 of every 100
             launches carries one seeded bit flip (an exponent bit, 30 / 62,
             or a mantissa bit, 10-20 / 40-50, of one seeded value at a
             seeded stage).  Counts false alarms over the clean launches,
             detections, corrections and escapes (faults that go undetected
             although, left alone, they push their transform past the
             accuracy bar), and times the clean, injected and plain runs.
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
             reps: int = 10, thread_level: bool = True) -> dict:
    """ms per exec for each transactions-per-group setting (thread-block
    level, TB-T) and, where the length allows it, for thread-level checks,
    against ABFT off."""
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
    rows = []
    if thread_level:
        # thread-level ABFT (Sec. 4.2.1) where one thread holds a whole
        # transform (its own one-thread shape), against the same plain
        # baseline as the block-level rows: the default plain shape
        try:
            tl = tfl.Plan(n, batch, dtype, "forward", "correct_thread")
        except tfl.TurboFFTError:
            tl = None
        if tl is not None:
            ms = timed(tl)
            rows.append({"transactions": "thread", "ms": round(ms, 4),
                         "overhead_pct": round(100.0 * (ms / base - 1.0), 2), "detected": tl.report()["detected"],
                         "shape": "one thread per transform (radix %d)" % tl.info()["radix"][0]})
            tl.close()
    ft = tfl.Plan(n, batch, dtype, "forward", "correct")
    for t in groups:
        ft.set_group_transactions(t)
        ms = timed(ft)
        rows.append({"transactions": t, "ms": round(ms, 4), "overhead_pct": round(100.0 * (ms / base - 1.0), 2),
                     "detected": ft.report()["detected"],
                     "shape": "%d threads per transform" % (n // ft.info()["radix"][0])})
    ft.close()
    return {"n": n, "dtype": dtype, "batch": batch, "plain_ms": round(base, 4), "rows": rows}


def _rel_per_transform(a, b):
    """Relative L2 distance of every row of a from the same row of b
    (absolute where the row of b is zero; non-finite rows give inf)."""
    import torch

    num = torch.linalg.vector_norm(a - b, dim=-1)
    den = torch.linalg.vector_norm(b, dim=-1)
    r = torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)), num)
    return torch.nan_to_num(r, nan=float("inf"))


def campaign(n: int, dtype: str = "complex64", elements: int = 1 << 26, launches: int = 400, every: int = 100,
             timing_launches: int = 200, data_seed: int = 3, site_seed: int = 4) -> dict:
    """Fault-injection campaign (Sec. 5.3) for one (dtype, n); see the module
    docstring.

    `launches` execs of a CORRECT plan, each followed by a report read; exec
    i carries a fault when i % every == every - 1.  Over the clean execs the
    false alarms are counted.  For each faulty exec: detected, located on the
    injected transform, corrected, uncorrectable; the corrected transform's
    distance from the clean output; and the same fault on a plain (ABFT off)
    plan, whose distance from the clean output says whether the fault breaks
    the accuracy bar.  The bar is taken against the GPU's own clean output of
    the plain plan (the fault-free result the checks must restore).  Timing:
    `timing_launches` back-to-back execs each of the plain plan, the CORRECT
    plan on clean launches and the CORRECT plan with 1-in-`every` injection,
    CUDA events on the current stream."""
    import torch

    import paper_2412_05824_gb300 as tfl
    import synth_signals as ss

    real = "float32" if dtype == "complex64" else "float64"
    batch = max(1, elements // n)
    x = ss.uniform_complex_torch(data_seed, batch, n, real)
    y = torch.empty_like(x)
    yref = torch.empty_like(x)
    yoff = torch.empty_like(x)
    ft = tfl.Plan(n, batch, dtype, "forward", "correct")
    off = tfl.Plan(n, batch, dtype, "forward", "off")
    off.exec(x, yref)
    info = ft.info()
    bar = _bar(dtype, n)
    exp_bit = 30 if dtype == "complex64" else 62
    man_bits = (10, 20) if dtype == "complex64" else (40, 50)
    rng = np.random.default_rng([site_seed, n, 0 if dtype == "complex64" else 1])

    def draw():
        p = int(rng.integers(0, info["num_passes"]))
        kind = "exponent" if rng.integers(0, 2) == 0 else "mantissa"
        bit = exp_bit if kind == "exponent" else int(rng.integers(man_bits[0], man_bits[1] + 1))
        return (int(rng.integers(0, batch)), p, int(rng.integers(0, info["stages"][p] + 1)),
                int(rng.integers(0, n)), int(rng.integers(0, 2)), bit), kind

    clean_launches = false_alarm_launches = false_alarm_groups = 0
    faults = []
    max_clean_ratio = 0.0
    for i in range(launches):
        if i % every == every - 1:
            site, kind = draw()
            ft.inject(*site)
            ft.exec(x, y)
            rep = ft.report()
            tr = site[0]
            err_all = _rel_per_transform(y, yref)
            err_fixed = float(err_all[tr])
            others = float(torch.max(torch.cat([err_all[:tr], err_all[tr + 1:]]))) if batch > 1 else 0.0
            off.inject(*site)
            off.exec(x, yoff)
            err_left = float(_rel_per_transform(yoff[tr:tr + 1], yref[tr:tr + 1])[0])
            breaking = not (err_left <= bar)
            detected = rep["detected"] > 0
            faults.append({"site": list(site[:5]), "bit": site[5], "kind": kind, "breaking": breaking,
                           "detected": detected, "located_right": detected and rep["first_transform"] == tr,
                           "corrected": rep["corrected"], "uncorrectable": rep["uncorrectable"],
                           "err_uncorrected": err_left, "err_after": err_fixed, "err_others": others,
                           "within_bar_after": err_fixed <= bar and others <= bar})
        else:
            ft.exec(x, y)
            rep = ft.report()
            clean_launches += 1
            false_alarm_groups += rep["detected"]
            false_alarm_launches += 1 if rep["detected"] else 0
            max_clean_ratio = max(max_clean_ratio, rep["max_clean_ratio"])
    s = torch.cuda.current_stream()

    def timed(plan, inject):
        for _ in range(3):
            plan.exec_ptr(x.data_ptr(), y.data_ptr(), s.cuda_stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        for i in range(timing_launches):
            if inject and i % every == every - 1:
                site, _ = draw()
                plan.inject(*site)
            plan.exec_ptr(x.data_ptr(), y.data_ptr(), s.cuda_stream)
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / timing_launches

    ms_plain = timed(off, False)
    ms_clean = timed(ft, False)
    ms_inj = timed(ft, True)
    nf = len(faults)
    nb = sum(f["breaking"] for f in faults)
    out = {
        "n": n, "dtype": dtype, "batch": batch, "elements": batch * n, "launches": launches, "every": every,
        "clean_launches": clean_launches, "false_alarm_launches": false_alarm_launches,
        "false_alarm_groups": false_alarm_groups,
        "max_clean_ratio": max_clean_ratio,
        "faults": nf, "breaking": nb,
        "detected": sum(f["detected"] for f in faults),
        "detected_breaking": sum(f["detected"] for f in faults if f["breaking"]),
        "located_right": sum(f["located_right"] for f in faults),
        "corrected": sum(1 for f in faults if f["detected"] and f["corrected"] >= 1 and f["uncorrectable"] == 0),
        "uncorrectable": sum(1 for f in faults if f["uncorrectable"]),
        "escapes": [f for f in faults if f["breaking"] and not f["detected"]],
        "all_within_bar_after": all(f["within_bar_after"] for f in faults if f["detected"] or not f["breaking"]),
        "ms_plain": round(ms_plain, 4), "ms_ft_clean": round(ms_clean, 4), "ms_ft_injected": round(ms_inj, 4),
        "overhead_pct_vs_plain": round(100.0 * (ms_clean / ms_plain - 1.0), 2),
        "injected_overhead_pct_vs_clean": round(100.0 * (ms_inj / ms_clean - 1.0), 2),
        "injected_overhead_pct_vs_plain": round(100.0 * (ms_inj / ms_plain - 1.0), 2),
        "timing_launches": timing_launches,
    }
    ft.close()
    off.close()
    del x, y, yref, yoff
    torch.cuda.empty_cache()
    return out
