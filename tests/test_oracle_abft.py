"""Pins for the oracle's two-sided ABFT (CPU only, host-made faults).

Checks against what the paper and the mathematics fix:
  * Eq. 1-2: (e^T W) x = e^T (W x) for any x (left checksum identity);
  * the closed form of e^T W for Wang's encoding vector (Sec. 2.2.2);
  * Eq. 3-5: the right-side sums satisfy y_bar = W x_bar on clean data and
    y_bar - W x_bar equals the error of a single corrupted signal;
  * location encoding (Sec. 4.1 / 4.3): S2 / S1 = k + 1 for one error;
  * brute force over every (stage, element, component, bit) site of tiny
    transforms: a detected fault is always located on the faulted signal and
    corrected back to the accuracy bar; faults that escape detection stay
    within a narrow band above the bar; clean groups never trip the test.
"""
import math

import numpy as np
import pytest

import oracle
import synth_signals as ss
from oracle import abft


def test_wang_vector_closed_form():
    # e_j = w3^j  =>  (W e)_n = sum_j (w3 wN^n)^j = (1 - w3^N) / (1 - w3 wN^n)
    for n in [8, 64, 1024, 1 << 16]:
        e = abft.encoding_vector(n, "wang")
        v = abft.left_vector(e)
        w3 = np.exp(-2j * np.pi / 3)
        k = np.arange(n)
        wn = np.exp(-2j * np.pi * k / n)
        closed = (1 - w3 ** n) / (1 - w3 * wn)
        assert np.max(np.abs(v - closed)) <= 1e-12 * np.max(np.abs(closed)) * math.log2(n)


def test_phase_vector_unit_modulus_and_seeded():
    e1 = abft.encoding_vector(256, "phase", 1)
    e2 = abft.encoding_vector(256, "phase", 1)
    e3 = abft.encoding_vector(256, "phase", 2)
    np.testing.assert_array_equal(e1, e2)
    assert np.max(np.abs(np.abs(e1) - 1)) < 1e-15
    assert np.max(np.abs(e1 - e3)) > 0.1


@pytest.mark.parametrize("kind", ["phase", "wang", "ones"])
@pytest.mark.parametrize("inverse,scaled", [(False, True), (True, True), (True, False)])
def test_left_checksum_identity(kind, inverse, scaled):
    n = 128
    e = abft.encoding_vector(n, kind)
    v = abft.left_vector(e, inverse, scaled)
    x = ss.uniform_complex(3, 5, n, np.float64)
    y = oracle.dft_naive(x, inverse=inverse, scaled=scaled)  # the definition
    s_in, s_out = abft.checksums(x, y, e, v)
    assert np.max(np.abs(s_in - s_out)) <= 1e-12 * np.max(np.abs(s_out))


def test_checksum_orientation_is_unconjugated():
    # a transposed/conjugated operand breaks the identity
    n = 64
    e = abft.encoding_vector(n)
    v = abft.left_vector(e)
    x = ss.uniform_complex(4, 3, n, np.float64)
    y = oracle.fft(x)
    good = np.abs(x @ v - y @ e)
    bad = np.abs(x @ np.conj(v) - y @ e)
    assert good.max() < 1e-10 and bad.min() > 1e-3


def test_right_side_sums_and_delta():
    n, G, k = 64, 6, 4
    x = ss.uniform_complex(5, G, n, np.float64)
    y = oracle.fft(x)
    np.testing.assert_allclose(y.sum(0), oracle.fft(x.sum(0)), atol=1e-12)
    err = np.zeros(n, complex)
    err[7:19] = 0.01 * (1 + 2j)
    y[k] += err
    delta = y.sum(0) - oracle.fft(x.sum(0))
    np.testing.assert_allclose(delta, err, atol=1e-12)


def test_location_encoding_exact():
    n, G = 32, 8
    e = abft.encoding_vector(n)
    v = abft.left_vector(e)
    x = ss.uniform_complex(6, G, n, np.float64)
    for k in range(G):
        y = oracle.fft(x)
        y[k, 3] += 0.5 - 0.25j
        rep = abft.group_check(x, y, e, v, np.float64)
        assert rep["detected"] and rep["method"] == "encoding" and rep["location"] == k
        assert abs(rep["S2"] / rep["S1"] - (k + 1)) < 1e-9


@pytest.mark.parametrize("precision", [np.float32, np.float64])
@pytest.mark.parametrize("n", [16, 256, 2048])
def test_clean_groups_never_flagged(precision, n):
    e = abft.encoding_vector(n)
    v = abft.left_vector(e)
    groups = 60 if n <= 256 else 12
    worst = 0.0
    for g in range(groups):
        x = ss.uniform_complex(100 + g, 4, n, precision)
        y = np.array([abft.fft_radix2(r, precision) for r in x])
        rep = abft.group_check(x, y, e, v, precision)
        assert not rep["detected"]
        worst = max(worst, abs(rep["S1"]) / rep["tau"])
    assert worst < 0.6   # margin: the clean residual stays well below tau


def test_structured_inputs_never_flagged():
    for n in [64, 1024]:
        e = abft.encoding_vector(n)
        v = abft.left_vector(e)
        for kind in ["impulse", "constant", "tone"]:
            x = ss.structured(kind, 4, n, np.float32)
            y = np.array([abft.fft_radix2(r, np.float32) for r in x])
            assert not abft.group_check(x, y, e, v, np.float32)["detected"]


def _sweep(n, G, precision, bits, seed=1):
    e = abft.encoding_vector(n)
    v = abft.left_vector(e)
    x = ss.uniform_complex(seed, G, n, precision)
    y_clean = np.array([abft.fft_radix2(x[b], precision) for b in range(G)]).astype(complex)
    ref = oracle.fft(x)
    tol = oracle.tolerance(precision, n)
    k = G // 2
    out = dict(sites=0, breaking=0, detected=0, escaped=0, escaped_max_ratio=0.0)
    for s in range(int(math.log2(n)) + 1):
        for i in range(n):
            for c in (0, 1):
                for b in bits:
                    y = y_clean.copy()
                    y[k] = abft.fft_radix2(x[k], precision, dict(stage=s, element=i, component=c, bit=b))
                    with np.errstate(all="ignore"):
                        err = float(oracle.rel_l2(y[k], ref[k]))
                    breaking = not (err <= tol)
                    yc, rep = abft.correct_group(x, y, e, v, precision)
                    out["sites"] += 1
                    out["breaking"] += breaking
                    if rep["detected"]:
                        out["detected"] += 1
                        # never blames another signal
                        assert rep["location"] in (k, None)
                        # a detected fault is corrected back within the bar
                        assert rep["corrected"] and not rep["uncorrectable"], (s, i, c, b, rep)
                        assert np.max(oracle.rel_l2(yc, ref)) <= tol
                    elif breaking:
                        out["escaped"] += 1
                        out["escaped_max_ratio"] = max(out["escaped_max_ratio"], err / tol)
                    # other signals are never modified
                    mask = np.arange(G) != k
                    np.testing.assert_array_equal(yc[mask], y_clean[mask])
    return out


def test_bruteforce_fault_sweep_float32():
    res = _sweep(16, 4, np.float32, range(32))
    assert res["detected"] > 0.5 * res["sites"]
    # escapes only in a narrow band just above the bar (low checksum
    # sensitivity at that site), and rarely
    assert res["escaped"] <= 0.01 * res["breaking"], res
    assert res["escaped_max_ratio"] < 10.0, res


def test_bruteforce_fault_sweep_float64_high_bits():
    res = _sweep(16, 3, np.float64, list(range(40, 64)))
    assert res["escaped"] <= 0.01 * res["breaking"], res
    assert res["escaped_max_ratio"] < 10.0, res


def test_exponent_flips_always_detected_and_corrected():
    n, G = 64, 4
    e = abft.encoding_vector(n)
    v = abft.left_vector(e)
    x = ss.uniform_complex(9, G, n, np.float32)
    ref = oracle.fft(x)
    y_clean = np.array([abft.fft_radix2(r, np.float32) for r in x]).astype(complex)
    for s in range(7):
        for i in (0, 5, 33, 63):
            y = y_clean.copy()
            y[1] = abft.fft_radix2(x[1], np.float32, dict(stage=s, element=i, component=s % 2, bit=30))
            yc, rep = abft.correct_group(x, y, e, v, np.float32)
            assert rep["detected"] and rep["corrected"] and rep["location"] == 1
            assert np.max(oracle.rel_l2(yc, ref)) <= oracle.tolerance(np.float32, n)


def test_two_faults_in_one_group_not_silently_passed():
    n, G = 64, 6
    e = abft.encoding_vector(n)
    v = abft.left_vector(e)
    x = ss.uniform_complex(10, G, n, np.float64)
    ref = oracle.fft(x)
    y = ref.copy()
    y[1, 10] += 3.0
    y[4, 20] -= 2.0 + 1j
    yc, rep = abft.correct_group(x, y, e, v, np.float64)
    assert rep["detected"]
    assert rep["uncorrectable"] and not rep["corrected"]


def test_inverse_direction_correction():
    n, G = 128, 4
    e = abft.encoding_vector(n)
    for scaled in (True, False):
        v = abft.left_vector(e, inverse=True, scaled=scaled)
        x = ss.uniform_complex(12, G, n, np.float64)
        ref = oracle.fft(x, inverse=True, scaled=scaled)
        y = ref.copy()
        y[2, 5] += 1e-3 * np.max(np.abs(ref))
        yc, rep = abft.correct_group(x, y, e, v, np.float64, inverse=True, scaled=scaled)
        assert rep["detected"] and rep["location"] == 2 and rep["corrected"]
        assert np.max(oracle.rel_l2(yc, ref)) <= oracle.tolerance(np.float64, n)
