"""Threshold (ROC) and group-size studies of the ABFT on the GPU, at small
scale: the properties the full studies rest on."""
import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402
from paper_2412_05824_gb300 import abft_study  # noqa: E402


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
def test_roc_small(dtype):
    r = abft_study.roc(n=256, batch=300, dtype=dtype, faults=120, scales=(0.25, 1.0, 4.0, 64.0), seed=3)
    rows = r["rows"]
    # no false alarm at the default threshold or above
    assert rows[1]["false_alarm_rate"] == 0 and rows[2]["false_alarm_rate"] == 0
    # a lower threshold flags at least as much, a higher one at most as much
    det = [row["detection_rate"] for row in rows]
    assert det[0] >= det[1] >= det[2] >= det[3]
    # at the default threshold every fault that breaks the bar is caught
    assert r["breaking_faults"] > 10
    assert rows[1]["missed_breaking"] == 0, rows[1]


@pytest.mark.parametrize("dtype,n", [("complex64", 512), ("complex64", 1 << 15), ("complex128", 1024)])
@pytest.mark.parametrize("t", [1, 2, 8, 16])
def test_group_size_detects_and_corrects(dtype, n, t):
    batch = 37
    rdt = np.float32 if dtype == "complex64" else np.float64
    x = ss.uniform_complex(61, batch, n, rdt)
    ref = oracle.fft(x)
    tol = oracle.tolerance(rdt, n)
    p = tfl.Plan(n, batch, dtype, "forward", "correct")
    p.set_group_transactions(t)
    xd = torch.from_numpy(x).cuda()
    y = p.exec(xd).cpu().numpy()
    rep = p.report()
    assert rep["detected"] == 0 and float(np.max(oracle.rel_l2(y, ref))) <= tol
    bit = 30 if dtype == "complex64" else 62
    for tr in (0, batch // 2, batch - 1):
        p.inject(tr, 0, 1, n // 3, 1, bit)
        y = p.exec(xd).cpu().numpy()
        rep = p.report()
        assert rep["detected"] >= 1 and rep["corrected"] >= 1 and rep["first_transform"] == tr, rep
        assert float(np.max(oracle.rel_l2(y, ref))) <= tol
    p.close()


def test_group_size_rejects():
    p = tfl.Plan(64, 4, "complex64", "forward", "correct")
    for bad in (0, 17, -1):
        with pytest.raises(tfl.TurboFFTError):
            p.set_group_transactions(bad)
    p.close()


def test_ablation_runs():
    r = abft_study.ablation(1024, "complex64", elements=1 << 22, groups=(1, 4), reps=3)
    assert r["plain_ms"] > 0 and len(r["rows"]) == 2
    assert all(row["detected"] == 0 for row in r["rows"])


@pytest.mark.parametrize("dtype,n", [("complex64", 256), ("complex64", 1 << 15), ("complex128", 1024)])
def test_campaign_small(dtype, n):
    """The Sec. 5.3 campaign at small scale: 1 in 10 launches faulty; no false
    alarm on the clean launches, every detected fault corrected back within
    the bar, no fault that breaks the bar left undetected."""
    r = abft_study.campaign(n, dtype, elements=1 << 18, launches=120, every=10, timing_launches=20)
    assert r["clean_launches"] == 108 and r["faults"] == 12
    assert r["false_alarm_launches"] == 0 and r["max_clean_ratio"] < 1.0
    assert r["uncorrectable"] == 0
    assert r["corrected"] == r["detected"]
    assert r["located_right"] == r["detected"]
    assert r["escapes"] == [], r["escapes"]
    assert r["all_within_bar_after"]
    assert r["ms_plain"] > 0 and r["ms_ft_clean"] > 0 and r["ms_ft_injected"] > 0
