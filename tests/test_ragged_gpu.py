"""Ragged batches of mixed power-of-two sizes (one plan; one launch of the
persistent ragged kernel for float32 lengths up to 2^16, else one CUDA graph
of per-size kernels).

Parity of every transform of a ragged batch with the CPU oracle (relative L2
per transform <= 2e-6 log2 N for complex64, 5e-15 log2 N for complex128),
bit-identity with the per-size plans the ragged plan is made of, fault
injection through global transform indices, graph re-capture on new
pointers, the autotuner, and the full-size workload (20,000 transforms with
sizes log-uniform in 2^6..2^16) on sampled transforms.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402

RDT = {"c64": np.float32, "c128": np.float64}
CDT = {"c64": "complex64", "c128": "complex128"}


def layout(seed, count, lo=6, hi=16, max_gap=64):
    sizes = ss.ragged_sizes(seed, count, lo, hi)
    offsets, extent = ss.ragged_offsets(sizes, seed + 1, max_gap)
    return sizes, offsets, extent


def packed_input(seed, extent, dt):
    return ss.uniform_complex(seed, 1, extent, RDT[dt])[0]


def expected_rows(x, sizes, offsets, direction="forward"):
    """{size: (indices, oracle output [count, size])}"""
    out = {}
    for n in np.unique(sizes):
        idx = np.nonzero(sizes == n)[0]
        rows = np.stack([x[offsets[i]:offsets[i] + n] for i in idx])
        if direction == "forward":
            ref = oracle.fft(rows)
        else:
            ref = oracle.fft(rows, inverse=True, scaled=(direction == "inverse"))
        out[int(n)] = (idx, ref)
    return out


def check_against_oracle(y, x, sizes, offsets, dt, direction="forward"):
    worst = 0.0
    for n, (idx, ref) in expected_rows(x, sizes, offsets, direction).items():
        got = np.stack([y[offsets[i]:offsets[i] + n] for i in idx])
        err = oracle.rel_l2(got, ref)
        tol = oracle.tolerance(RDT[dt], n)
        assert np.all(np.isfinite(got)), n
        assert float(np.max(err)) <= tol, (n, float(np.max(err)), tol)
        worst = max(worst, float(np.max(err)) / tol)
    return worst


def run_ragged(plan, x, fill=np.nan):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.full_like(xd, complex(fill, fill))
    plan.exec(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def gap_mask(sizes, offsets, extent):
    m = np.ones(extent, dtype=bool)
    for n, o in zip(sizes, offsets):
        m[o:o + n] = False
    return m


@pytest.mark.parametrize("dt,direction,ft", [
    ("c64", "forward", "off"),
    ("c64", "forward", "correct"),
    ("c64", "inverse", "correct"),
    ("c64", "inverse_unscaled", "detect"),
    ("c128", "forward", "correct"),
    ("c128", "inverse", "off"),
])
def test_ragged_matches_oracle(dt, direction, ft):
    sizes, offsets, extent = layout(21, 160)
    x = packed_input(5, extent, dt)
    plan = tfl.RaggedPlan(sizes, offsets, CDT[dt], direction, ft)
    y = run_ragged(plan, x)
    check_against_oracle(y, x, sizes, offsets, dt, direction)
    # gaps between transforms are never written
    assert np.all(np.isnan(y[gap_mask(sizes, offsets, extent)].real))
    if ft != "off":
        rep = plan.report()
        assert rep["detected"] == 0 and rep["uncorrectable"] == 0 and rep["status"] == tfl.SUCCESS, rep
        assert rep["groups_checked"] > 0
    plan.close()


@pytest.mark.parametrize("ft", ["off", "correct"])
def test_ragged_equals_per_size_plans_bitwise(ft):
    """Graph form: each member runs the same kernel as the plain plan of its
    size and count; only the addressing differs, so the bits agree."""
    tfl.set_autotune(False)
    sizes, offsets, extent = layout(33, 120, 3, 16)
    x = packed_input(8, extent, "c64")
    tfl.set_ragged_single_launch(False)
    try:
        plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", ft)
    finally:
        tfl.set_ragged_single_launch(True)
    assert plan.info()["single_launch"] == 0
    y = run_ragged(plan, x)
    for n in np.unique(sizes):
        idx = np.nonzero(sizes == n)[0]
        rows = np.stack([x[offsets[i]:offsets[i] + n] for i in idx])
        p = tfl.Plan(int(n), len(idx), "complex64", "forward", ft)
        ref = p.exec(torch.from_numpy(rows).cuda()).cpu().numpy()
        p.close()
        got = np.stack([y[offsets[i]:offsets[i] + n] for i in idx])
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), int(n)
    plan.close()


def test_ragged_info_and_members():
    sizes, offsets, extent = layout(4, 90, 3, 18)
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct")
    info = plan.info()
    distinct, counts = np.unique(sizes, return_counts=True)
    assert info["num_members"] == len(distinct) and info["batch"] == len(sizes) and info["n"] == 0
    for k, m in enumerate(plan.members()):
        assert m["n"] == distinct[k] and m["batch"] == counts[k]
        assert m["sub_n"][0] * m["sub_n"][1] == distinct[k]
    plan.close()


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_ragged_injection_located_by_global_index(dt):
    sizes, offsets, extent = layout(12, 100)
    x = packed_input(13, extent, dt)
    plan = tfl.RaggedPlan(sizes, offsets, CDT[dt], "forward", "correct")
    bit = 30 if dt == "c64" else 62
    # one single-pass and one two-pass transform, several stages
    targets = [int(np.nonzero(sizes == 256)[0][3]), int(np.nonzero(sizes == 65536)[0][1])]
    for tr in targets:
        members = {m["n"]: m for m in plan.members()}
        m = members[int(sizes[tr])]
        for pass_ in range(m["num_passes"]):
            for stage in (0, 1, m["stages"][pass_]):
                elem = int(sizes[tr]) // 3 + stage
                plan.inject(tr, pass_, stage, elem, stage % 2, bit)
                y = run_ragged(plan, x)
                rep = plan.report()
                assert rep["detected"] >= 1 and rep["corrected"] >= 1, (tr, pass_, stage, rep)
                assert rep["uncorrectable"] == 0 and rep["status"] == tfl.SUCCESS, rep
                assert rep["first_transform"] == tr, (tr, rep)
                check_against_oracle(y, x, sizes, offsets, dt)
    # the next exec goes through the captured graph again and is clean
    y = run_ragged(plan, x)
    rep = plan.report()
    assert rep["detected"] == 0 and rep["corrected"] == 0, rep
    check_against_oracle(y, x, sizes, offsets, dt)
    plan.close()


def test_ragged_detect_mode_reports_uncorrectable():
    sizes, offsets, extent = layout(14, 60)
    x = packed_input(15, extent, "c64")
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "detect")
    tr = int(np.argmax(sizes))
    plan.inject(tr, 0, 1, 5, 0, 30)
    run_ragged(plan, x)
    rep = plan.report()
    assert rep["detected"] >= 1 and rep["status"] == tfl.FT_UNCORRECTABLE and rep["first_transform"] == tr
    plan.close()


def test_ragged_inject_rejects_bad_sites():
    sizes, offsets, extent = layout(16, 20)
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct")
    with pytest.raises(tfl.TurboFFTError):
        plan.inject(len(sizes), 0, 0, 0, 0, 3)  # transform out of range
    with pytest.raises(tfl.TurboFFTError):
        plan.inject(0, 0, 0, int(sizes[0]), 0, 3)  # element beyond that transform's length
    plan.close()


def test_ragged_new_pointers_recapture():
    sizes, offsets, extent = layout(17, 80)
    x1 = packed_input(18, extent, "c64")
    x2 = packed_input(19, extent, "c64")
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct")
    for x in (x1, x2, x1):
        y = run_ragged(plan, x)  # fresh buffers each time
        check_against_oracle(y, x, sizes, offsets, "c64")
    # same buffers twice: the graph is replayed
    xd = torch.from_numpy(x2).cuda()
    yd = torch.empty_like(xd)
    for _ in range(2):
        yd.zero_()
        plan.exec(xd, yd)
        torch.cuda.synchronize()
        check_against_oracle(yd.cpu().numpy(), x2, sizes, offsets, "c64")
    plan.close()


def test_ragged_threshold_change_reaches_the_graph():
    sizes, offsets, extent = layout(20, 40)
    x = packed_input(22, extent, "c64")
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "detect")
    run_ragged(plan, x)
    assert plan.report()["detected"] == 0
    plan.set_threshold_scale(1e-6)  # far below clean rounding: every group trips
    run_ragged(plan, x)
    assert plan.report()["detected"] > 0
    plan.set_threshold_scale(1.0)
    run_ragged(plan, x)
    assert plan.report()["detected"] == 0
    plan.close()


def test_ragged_exec_host():
    sizes, offsets, extent = layout(23, 70)
    x = packed_input(24, extent, "c64")
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct")
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.full_like(xh, complex(np.nan, np.nan)).pin_memory()
    plan.exec_host(xh, yh)
    y = yh.numpy()
    check_against_oracle(y, x, sizes, offsets, "c64")
    assert plan.report()["detected"] == 0
    plan.close()


def test_ragged_unsupported_calls():
    sizes, offsets, extent = layout(25, 10)
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "off")
    L = tfl.lib()
    buf = torch.empty(1 << 20, dtype=torch.complex64, device="cuda")
    assert L.turbofft_set_workspace(plan.handle, buf.data_ptr(), 8 << 20) == tfl.UNSUPPORTED
    assert L.turbofft_set_profiling(plan.handle, 1) == tfl.UNSUPPORTED
    xd = torch.zeros(extent, dtype=torch.complex64, device="cuda")
    yd = torch.empty_like(xd)
    s = torch.cuda.current_stream().cuda_stream
    assert L.turbofft_exec_static_scratch(plan.handle, xd.data_ptr(), yd.data_ptr(), s) == tfl.UNSUPPORTED
    # overlapping in/out over the packed span
    assert L.turbofft_exec(plan.handle, xd.data_ptr(), xd.data_ptr() + 16, s) == tfl.UNSUPPORTED
    i = tfl.PlanInfo()
    assert L.turbofft_plan_get_member_info(plan.handle, 99, ctypes.byref(i)) == tfl.INVALID_VALUE
    p1 = tfl.Plan(64, 4)
    assert L.turbofft_plan_get_member_info(p1.handle, 0, ctypes.byref(i)) == tfl.INVALID_VALUE
    p1.close()
    plan.close()


def test_autotune_ragged_and_plain():
    sizes, offsets, extent = layout(26, 200)
    x = packed_input(27, extent, "c64")
    tfl.set_autotune(True)
    try:
        plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct")
        plain = tfl.Plan(1024, 301, "complex64", "forward", "correct")
    finally:
        tfl.set_autotune(False)
    assert plan.info()["autotuned"] == 1
    assert all(m["autotuned"] == 1 for m in plan.members())
    y = run_ragged(plan, x)
    check_against_oracle(y, x, sizes, offsets, "c64")
    assert plan.report()["detected"] == 0
    info = plain.info()
    assert info["autotuned"] == 1
    assert info["block"][0] == info["sub_n"][0] // info["radix"][0] * info["per_block"][0]
    xb = ss.uniform_complex(28, 301, 1024, np.float32)
    yb = plain.exec(torch.from_numpy(xb).cuda()).cpu().numpy()
    assert float(np.max(oracle.rel_l2(yb, oracle.fft(xb)))) <= oracle.tolerance(np.float32, 1024)
    assert plain.report()["detected"] == 0
    plain.close()
    plan.close()


def test_ragged_full_size_sampled():
    """The benchmarked workload: 20,000 complex64 transforms, sizes
    log-uniform in 2^6..2^16, packed back to back, ABFT on, one graph;
    sampled transforms of every size checked against the oracle."""
    seed_sizes, seed_data = 2024, 4
    sizes = ss.ragged_sizes(seed_sizes, 20000, 6, 16)
    offsets, extent = ss.ragged_offsets(sizes)
    xd = ss.uniform_complex_torch(seed_data, 1, extent, "float32").view(-1)
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct")
    yd = plan.exec(xd)
    yd = plan.exec(xd)  # graph replay
    torch.cuda.synchronize()
    rep = plan.report()
    assert rep["detected"] == 0 and rep["status"] == tfl.SUCCESS and rep["groups_checked"] > 0, rep
    for n in np.unique(sizes):
        idx = np.nonzero(sizes == n)[0]
        pick = idx[[0, len(idx) // 2, len(idx) - 1]]
        for i in pick:
            o = int(offsets[i])
            xr = ss.uniform_complex(seed_data, 1, int(n), np.float32, first_element=o)
            assert np.array_equal(xr[0], xd[o:o + n].cpu().numpy())
            ref = oracle.fft(xr)
            got = yd[o:o + n].cpu().numpy()[None]
            assert float(oracle.rel_l2(got, ref)[0]) <= oracle.tolerance(np.float32, int(n)), (int(n), int(i))
    plan.close()


def test_autotune_structure_choice_stays_correct():
    """With autotuning on, a float32 2^14 plan times its split and cluster
    structures and keeps the faster; either way the result is the transform."""
    n, batch = 1 << 14, 40
    x = ss.uniform_complex(29, batch, n, np.float32)
    tfl.set_autotune(True)
    try:
        plans = [tfl.Plan(n, batch, "complex64", "forward", ft) for ft in ("off", "correct")]
    finally:
        tfl.set_autotune(False)
    for p in plans:
        assert p.info()["autotuned"] == 1
        y = p.exec(torch.from_numpy(x).cuda()).cpu().numpy()
        assert float(np.max(oracle.rel_l2(y, oracle.fft(x)))) <= oracle.tolerance(np.float32, n)
        p.close()


@pytest.mark.parametrize("ft", ["off", "correct", "detect"])
@pytest.mark.parametrize("direction", ["forward", "inverse"])
def test_single_launch_matches_graph_form(ft, direction):
    """One launch of the persistent kernel against the graph of per-size
    kernels: bit for bit where both use the same radix (every length but
    8192, which the single launch runs as two passes 64 x 128), within the
    bar of the oracle everywhere; gaps untouched; no false alarm."""
    sizes, offsets, extent = layout(41, 300, 3, 16, max_gap=32)
    x = packed_input(9, extent, "c64")
    one = tfl.RaggedPlan(sizes, offsets, "complex64", direction, ft)
    assert one.info()["single_launch"] == 1
    tfl.set_ragged_single_launch(False)
    try:
        graph = tfl.RaggedPlan(sizes, offsets, "complex64", direction, ft)
    finally:
        tfl.set_ragged_single_launch(True)
    y1 = run_ragged(one, x)
    y2 = run_ragged(graph, x)
    check_against_oracle(y1, x, sizes, offsets, "c64", direction)
    assert np.all(np.isnan(y1[gap_mask(sizes, offsets, extent)].real))
    for n, o in zip(sizes, offsets):
        if n != 8192:
            assert np.array_equal(y1[o:o + n].view(np.uint64), y2[o:o + n].view(np.uint64)), int(n)
    if ft != "off":
        rep = one.report()
        assert rep["detected"] == 0 and rep["status"] == tfl.SUCCESS and rep["groups_checked"] > 0, rep
    # repeated execs (the captured launch) give the same bits
    y3 = run_ragged(one, x)
    assert np.array_equal(np.nan_to_num(y1).view(np.uint64), np.nan_to_num(y3).view(np.uint64))
    one.close()
    graph.close()


def test_single_launch_injection_and_correction():
    """Faults injected into a single-launch exec (one seeded bit per exec, in
    every pass of every length class) are detected on the right global
    transform and corrected inside the same launch."""
    sizes, offsets, extent = layout(52, 200, 3, 16)
    x = packed_input(10, extent, "c64")
    plan = tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct")
    assert plan.info()["single_launch"] == 1
    ref = run_ragged(plan, x)
    members = {m["n"]: m for m in plan.members()}
    rng = np.random.default_rng(52)
    seen = set()
    for tr in rng.permutation(len(sizes))[:40]:
        n = int(sizes[tr])
        m = members[n]
        p = int(rng.integers(0, m["num_passes"]))
        st = int(rng.integers(0, m["stages"][p] + 1))
        plan.inject(int(tr), p, st, int(rng.integers(0, n)), int(rng.integers(0, 2)), 30)
        y = run_ragged(plan, x)
        rep = plan.report()
        assert rep["detected"] >= 1 and rep["corrected"] >= 1 and rep["uncorrectable"] == 0, (n, p, st, rep)
        assert rep["first_transform"] == tr
        check_against_oracle(y, x, sizes, offsets, "c64")
        seen.add((n, p))
    assert len(seen) >= 8
    # the next exec is clean again (the captured launch holds no site)
    y = run_ragged(plan, x)
    assert plan.report()["detected"] == 0
    assert np.array_equal(y.view(np.uint64), ref.view(np.uint64))
    plan.close()


def test_single_launch_applies_only_where_it_can():
    sizes, offsets, extent = layout(7, 40, 3, 16)
    assert tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "off").info()["single_launch"] == 1
    # float64, the register-sums mode and lengths above 2^16 keep the graph
    assert tfl.RaggedPlan(sizes, offsets, "complex128", "forward", "off").info()["single_launch"] == 0
    assert tfl.RaggedPlan(sizes, offsets, "complex64", "forward", "correct_registers").info()["single_launch"] == 0
    big = list(sizes) + [1 << 17]
    offs = list(offsets) + [int(extent + (extent & 1))]
    assert tfl.RaggedPlan(big, offs, "complex64", "forward", "off").info()["single_launch"] == 0
