"""Online two-sided ABFT on the GPU: clean runs raise no alarm; injected bit
flips (Sec. 5.3.1 protocol: one seeded bit of one seeded value of one
signal) that break the accuracy bar are detected, located on the right
transform and corrected back within the bar (CORRECT mode), or reported
(DETECT mode).  Every fault here is a data bit flip in a register made by the
kernel's own injection hook; nothing faults or stalls the GPU."""
import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402

DT = {"c64": np.float32, "c128": np.float64}


def breaks(err, tol) -> bool:
    """True unless every transform is within the bar (NaN/Inf count as breaking)."""
    return not (float(np.max(err)) <= tol)


class Runner:
    def __init__(self, n, batch, dt, direction="forward", seed=11):
        self.n, self.batch, self.dt = n, batch, dt
        self.x = ss.uniform_complex(seed, batch, n, DT[dt])
        self.xd = torch.from_numpy(self.x).cuda()
        self.direction = direction
        if direction == "forward":
            self.ref = oracle.fft(self.x)
        else:
            self.ref = oracle.fft(self.x, inverse=True, scaled=direction == "inverse")
        self.tol = oracle.tolerance(DT[dt], n)
        self.plans = {m: tfl.Plan(n, batch, "complex64" if dt == "c64" else "complex128", direction, m)
                      for m in ("off", "detect", "correct", "correct_registers")}

    def run(self, mode, site=None, bit=None):
        p = self.plans[mode]
        if site is not None:
            p.inject(*site, bit)
        y = p.exec(self.xd)
        torch.cuda.synchronize()
        rep = p.report() if mode != "off" else None
        yn = y.cpu().numpy()
        with np.errstate(all="ignore"):
            err = oracle.rel_l2(yn, self.ref)
        return yn, err, rep

    def stages(self, pass_):
        return self.plans["correct"].info()["stages"][pass_]

    def passes(self):
        return self.plans["correct"].info()["num_passes"]


CONFIGS = [("c64", 256, 203), ("c64", 4096, 21), ("c64", 1 << 17, 3),
           ("c128", 512, 67), ("c128", 1 << 14, 5)]


@pytest.mark.parametrize("dt,n,batch", CONFIGS)
def test_clean_runs_no_alarm(dt, n, batch):
    r = Runner(n, batch, dt)
    worst = 0.0
    for _ in range(20):
        _, err, rep = r.run("correct")
        assert rep["detected"] == 0 and rep["uncorrectable"] == 0 and rep["status"] == tfl.SUCCESS
        assert float(np.max(err)) <= r.tol
        worst = max(worst, rep["max_clean_ratio"])
    assert 0 < worst < 0.8, worst


def _sites(r, rng, count, bits):
    out = []
    for _ in range(count):
        p = int(rng.integers(0, r.passes()))
        out.append((int(rng.integers(0, r.batch)), p, int(rng.integers(0, r.stages(p) + 1)),
                    int(rng.integers(0, r.n)), int(rng.integers(0, 2)), int(rng.choice(bits))))
    return out


@pytest.mark.parametrize("dt,n,batch", CONFIGS)
def test_exponent_flips_detected_and_corrected(dt, n, batch):
    r = Runner(n, batch, dt)
    rng = np.random.default_rng(n + batch)
    bit = 30 if dt == "c64" else 62
    for (tr, p, st, el, comp, b) in _sites(r, rng, 12, [bit]):
        y, err, rep = r.run("correct", (tr, p, st, el, comp), b)
        # an exponent flip of a value |v| < 2 overflows or blows up: always caught
        _, err_off, _ = r.run("off", (tr, p, st, el, comp), b)
        if not breaks(err_off, r.tol):
            continue  # a flip that stays within the accuracy bar needs no correction
        assert rep["detected"] >= 1 and rep["corrected"] >= 1, (tr, p, st, el, comp, rep)
        assert rep["first_transform"] == tr
        assert rep["uncorrectable"] == 0 and rep["status"] == tfl.SUCCESS
        assert float(np.max(err)) <= r.tol, (tr, p, st, el, comp, float(np.max(err)))


@pytest.mark.parametrize("dt,n,batch", CONFIGS)
def test_mantissa_flips(dt, n, batch):
    r = Runner(n, batch, dt)
    rng = np.random.default_rng(3 * n + batch)
    bits = list(range(10, 21)) if dt == "c64" else list(range(40, 51))
    escapes = []
    for (tr, p, st, el, comp, b) in _sites(r, rng, 24, bits):
        _, err_off, _ = r.run("off", (tr, p, st, el, comp), b)
        y, err, rep = r.run("correct", (tr, p, st, el, comp), b)
        breaking = breaks(err_off, r.tol)
        if rep["detected"]:
            assert rep["first_transform"] == tr
            assert rep["corrected"] >= 1 and rep["uncorrectable"] == 0, rep
            assert float(np.max(err)) <= r.tol
        elif breaking:
            # a fault left undetected although it breaks the bar: recorded
            # with its site (the bar is 0 such escapes)
            escapes.append(((tr, p, st, el, comp, b), float(np.max(err_off)) / r.tol))
        else:
            assert float(np.max(err)) <= r.tol
    assert escapes == [], escapes


@pytest.mark.parametrize("dt,n,batch", [("c64", 512, 50), ("c64", 1 << 15, 5), ("c128", 1024, 11)])
def test_register_sums_mode_matches(dt, n, batch):
    """Right-side sums kept in registers (the paper's thread-level
    accumulation): the same detections and corrections."""
    r = Runner(n, batch, dt)
    rng = np.random.default_rng(7 * n)
    bit = 30 if dt == "c64" else 62
    for (tr, p, st, el, comp, b) in _sites(r, rng, 8, [bit] + list(range(16, 21))):
        _, err_off, _ = r.run("off", (tr, p, st, el, comp), b)
        y1, err1, rep1 = r.run("correct", (tr, p, st, el, comp), b)
        y2, err2, rep2 = r.run("correct_registers", (tr, p, st, el, comp), b)
        assert rep1["detected"] == rep2["detected"]
        assert rep1["corrected"] == rep2["corrected"] and rep1["uncorrectable"] == rep2["uncorrectable"] == 0
        if rep1["detected"]:
            assert rep1["first_transform"] == rep2["first_transform"] == tr
        assert float(np.max(err1)) <= r.tol and float(np.max(err2)) <= r.tol
    for _ in range(5):
        _, err, rep = r.run("correct_registers")
        assert rep["detected"] == 0 and float(np.max(err)) <= r.tol


@pytest.mark.parametrize("dt,n,batch", [("c64", 1024, 40), ("c64", 1 << 18, 2), ("c128", 2048, 9)])
def test_detect_mode_reports_without_correcting(dt, n, batch):
    r = Runner(n, batch, dt)
    bit = 30 if dt == "c64" else 62
    site = (batch // 2, 0, 0, 5, 0)
    _, err_off, _ = r.run("off", site, bit)
    assert breaks(err_off, r.tol)
    y, err, rep = r.run("detect", site, bit)
    assert rep["detected"] >= 1 and rep["corrected"] == 0
    assert rep["status"] == tfl.FT_UNCORRECTABLE
    assert rep["first_transform"] == batch // 2
    assert breaks(err, r.tol)


@pytest.mark.parametrize("direction", ["inverse", "inverse_unscaled"])
def test_inverse_direction_correction(direction):
    r = Runner(2048, 30, "c64", direction)
    for site in [(4, 0, 0, 100, 0), (17, 0, 1, 2047, 1), (29, 0, r.stages(0), 7, 0)]:
        y, err, rep = r.run("correct", site, 30)
        _, err_off, _ = r.run("off", site, 30)
        if breaks(err_off, r.tol):
            assert rep["corrected"] >= 1 and rep["first_transform"] == site[0]
        assert float(np.max(err)) <= r.tol


def test_two_pass_every_stage_both_passes():
    r = Runner(1 << 16, 4, "c64")
    assert r.passes() == 2
    for p in range(2):
        for st in range(r.stages(p) + 1):
            site = (2, p, st, (12345 * (st + 1)) % r.n, st % 2)
            y, err, rep = r.run("correct", site, 30)
            _, err_off, _ = r.run("off", site, 30)
            if breaks(err_off, r.tol):
                assert rep["corrected"] >= 1 and rep["first_transform"] == 2, (p, st, rep)
                assert rep["first_pass"] == p
            assert float(np.max(err)) <= r.tol, (p, st)


def test_threshold_scale_knob():
    """A threshold far below the rounding noise makes clean groups alarm;
    the library must then refuse to 'correct' (several signals flagged) and
    leave the correct output untouched."""
    r = Runner(1024, 64, "c64")
    p = r.plans["correct"]
    p.set_threshold_scale(1e-4)
    y, err, rep = r.run("correct")
    assert rep["detected"] > 0
    assert float(np.max(err)) <= r.tol
    p.set_threshold_scale(1.0)
    y, err, rep = r.run("correct")
    assert rep["detected"] == 0


def test_injection_is_one_shot():
    r = Runner(512, 16, "c64")
    r.run("correct", (3, 0, 1, 9, 0), 30)
    _, err, rep = r.run("correct")
    assert rep["detected"] == 0 and float(np.max(err)) <= r.tol


def test_inject_rejects_bad_sites():
    p = tfl.Plan(256, 4, "complex64", "forward", "correct")
    for site, bit in [((4, 0, 0, 0, 0), 3), ((0, 1, 0, 0, 0), 3), ((0, 0, 99, 0, 0), 3),
                      ((0, 0, 0, 256, 0), 3), ((0, 0, 0, 0, 2), 3), ((0, 0, 0, 0, 0), 32)]:
        with pytest.raises(tfl.TurboFFTError):
            p.inject(*site, bit)


def test_exec_host_reports_and_corrects():
    n, batch = 2048, 64
    x = ss.uniform_complex(12, batch, n, np.float32)
    plan = tfl.Plan(n, batch, "complex64", "forward", "correct")
    xh = torch.from_numpy(x).pin_memory()
    plan.inject(50, 0, 1, 77, 1, 30)
    y = plan.exec_host(xh)
    rep = plan.report()
    assert rep["corrected"] >= 1 and rep["first_transform"] == 50
    assert float(np.max(oracle.rel_l2(y.numpy(), oracle.fft(x)))) <= oracle.tolerance(np.float32, n)


@pytest.mark.parametrize("n,batch", [(1 << 13, 37), (1 << 16, 9), (1 << 20, 3)])
def test_float64_two_pass_checks_whole_transforms(n, batch):
    """float64 two-pass plans check whole transforms: v.x in the column pass,
    e.y in the row pass, compared after it (one check per transform); a
    fault in either pass is found on its transform and recomputed."""
    r = Runner(n, batch, "c128")
    assert r.plans["correct"].info()["transform_checks"] == 1
    assert r.plans["correct_registers"].info()["transform_checks"] == 0  # per-pass groups
    _, err, rep = r.run("correct")
    assert rep["detected"] == 0 and rep["groups_checked"] == batch
    assert 0 < rep["max_clean_ratio"] < 0.8
    assert float(np.max(err)) <= r.tol
    rng = np.random.default_rng(n + 5)
    for k in range(6):
        p = k % 2
        st = int(rng.integers(0, r.stages(p) + 1))
        tr, el, comp = int(rng.integers(0, batch)), int(rng.integers(0, n)), int(rng.integers(0, 2))
        y, err, rep = r.run("correct", (tr, p, st, el, comp), 62)
        assert rep["detected"] == 1 and rep["corrected"] == 1 and rep["recomputed"] == 1, (p, st, rep)
        assert rep["first_transform"] == tr and rep["first_pass"] == 1 and rep["uncorrectable"] == 0
        assert float(np.max(err)) <= r.tol
        # detect mode: reported on the transform, not corrected
        _, err_d, rep_d = r.run("detect", (tr, p, st, el, comp), 62)
        assert rep_d["detected"] == 1 and rep_d["located"] == 1 and rep_d["first_transform"] == tr
        assert not (float(np.max(err_d)) <= r.tol)


def test_float64_whole_transform_checks_through_host_chunks():
    """Host-buffer exec of a float64 two-pass plan runs in chunks of about
    128 MiB (here 8 transforms of 16 MiB, two chunks): every chunk starts its whole-
    transform sums from zero, and a fault in a later chunk is corrected once,
    on its global transform index."""
    n, batch = 1 << 20, 11
    x = ss.uniform_complex(14, batch, n, np.float64)
    ref = oracle.fft(x)
    tol = oracle.tolerance(np.float64, n)
    plan = tfl.Plan(n, batch, "complex128", "forward", "correct")
    xh = torch.from_numpy(x).pin_memory()
    for _ in range(2):
        y = plan.exec_host(xh)
        rep = plan.report()
        assert rep["detected"] == 0 and rep["groups_checked"] == batch, rep
        assert float(np.max(oracle.rel_l2(y.numpy(), ref))) <= tol
    plan.inject(9, 1, 2, 12345, 0, 62)
    y = plan.exec_host(xh)
    rep = plan.report()
    assert rep["detected"] == 1 and rep["corrected"] == 1 and rep["first_transform"] == 9, rep
    assert float(np.max(oracle.rel_l2(y.numpy(), ref))) <= tol
    plan.close()


@pytest.mark.parametrize("direction", ["inverse", "inverse_unscaled", "forward_scaled"])
def test_float64_whole_transform_checks_other_directions(direction):
    """The whole-transform checks hold in the conjugated (inverse) domain and
    before the output scaling: clean runs raise no alarm, a fault in either
    pass is corrected."""
    n, batch = 1 << 14, 6
    x = ss.uniform_complex(15, batch, n, np.float64)
    if direction == "forward_scaled":
        ref = oracle.fft(x) / n
    else:
        ref = oracle.fft(x, inverse=True, scaled=direction == "inverse")
    tol = oracle.tolerance(np.float64, n)
    plan = tfl.Plan(n, batch, "complex128", direction, "correct")
    assert plan.info()["transform_checks"] == 1
    xd = torch.from_numpy(x).cuda()
    y = plan.exec(xd).cpu().numpy()
    rep = plan.report()
    assert rep["detected"] == 0 and 0 < rep["max_clean_ratio"] < 0.8
    assert float(np.max(oracle.rel_l2(y, ref))) <= tol
    for p, st in ((0, 1), (1, 2)):
        plan.inject(4, p, st, 999, 1, 45)
        y = plan.exec(xd).cpu().numpy()
        rep = plan.report()
        assert rep["uncorrectable"] == 0
        if rep["detected"]:
            assert rep["corrected"] == 1 and rep["first_transform"] == 4
        assert float(np.max(oracle.rel_l2(y, ref))) <= tol
    plan.close()


@pytest.mark.parametrize("n,batch", [(1024, 40), (1 << 16, 3)])
@pytest.mark.parametrize("scale_log2", [70, 110])
def test_float64_checks_beyond_the_float32_range(n, batch, scale_log2):
    """float64 data far beyond the float32 range (|x| ~ 2^70 and 2^110, so
    that the threshold's energy sum overflows float32): no false alarm, and
    an exponent flip is detected and corrected (single pass: block-level
    checks; 2^16: whole-transform checks)."""
    x = ss.uniform_complex(31, batch, n, np.float64) * 2.0 ** scale_log2
    xd = torch.from_numpy(x).cuda()
    ref = oracle.fft(x)
    tol = oracle.tolerance(np.float64, n)
    p = tfl.Plan(n, batch, "complex128", "forward", "correct")
    y = p.exec(xd).cpu().numpy()
    rep = p.report()
    assert rep["detected"] == 0 and rep["status"] == tfl.SUCCESS, rep
    assert float(np.max(oracle.rel_l2(y, ref))) <= tol
    p.inject(batch // 2, 0, 1, 77, 0, 61)
    y = p.exec(xd).cpu().numpy()
    rep = p.report()
    assert rep["detected"] >= 1 and rep["corrected"] >= 1 and rep["status"] == tfl.SUCCESS, rep
    assert rep["first_transform"] == batch // 2, rep
    assert float(np.max(oracle.rel_l2(y, ref))) <= tol
    p.close()
