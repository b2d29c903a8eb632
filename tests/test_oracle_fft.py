"""Pins for the oracle FFT (CPU only).

Every check here ties the oracle to something other than itself: the
definition summed in long double, hand-worked small DFTs, closed forms
(impulse, shifted impulse, constant, tone), Parseval, linearity, the
round trip, and numpy's independent FFT.  A planted-mistake test confirms
that the pins reject plausible errors (sign, twiddle index, dropped scale,
transposed operands)."""
import math
import os

import numpy as np
import pytest

import oracle
import synth_signals as ss

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dft_definition_small.txt")


def _read_golden():
    cases = []
    cur = None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "case":
            cur = dict(name=parts[1], n=int(parts[2]), x=[], y=[])
            cases.append(cur)
        elif parts[0] in ("x", "y"):
            cur[parts[0]].append(float(parts[1]) + 1j * float(parts[2]))
    return cases


@pytest.mark.parametrize("case", _read_golden(), ids=lambda c: c["name"])
def test_golden_hand_worked(case):
    x = np.array(case["x"])
    y = np.array(case["y"])
    assert len(x) == case["n"]
    np.testing.assert_allclose(oracle.fft(x), y, rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.dft_naive(x), y, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# reusable pins: each returns the worst error observed
# ---------------------------------------------------------------------------
def pin_vs_naive(fft_fn, n, inverse=False, seed=11):
    x = ss.uniform_complex(seed, 3, n, np.float64)
    y = fft_fn(x, inverse=inverse)
    y_ref = oracle.dft_naive(x, inverse=inverse)
    return float(np.max(oracle.rel_l2(y, y_ref)))


def pin_impulse(fft_fn, n):
    worst = 0.0
    for n0 in sorted({0, min(1, n - 1), n // 2, n - 1}):
        x = np.zeros(n, complex)
        x[n0] = 1.0
        j = np.arange(n)
        q = (j * n0) % n
        expect = np.exp(-2j * np.pi * q / n)
        worst = max(worst, float(np.max(np.abs(fft_fn(x[None])[0] - expect))))
    return worst


def pin_constant(fft_fn, n, c=0.75 - 0.5j):
    x = np.full((1, n), c)
    expect = np.zeros(n, complex)
    expect[0] = n * c
    return float(np.max(np.abs(fft_fn(x)[0] - expect)) / (n * abs(c)))


def pin_tone(fft_fn, n):
    k = ss.tone_index(n)
    x = ss.tone(1, n, np.float64, k)
    expect = np.zeros(n, complex)
    expect[k % n] = n
    return float(np.max(np.abs(fft_fn(x)[0] - expect)) / n)


def pin_parseval(fft_fn, n, seed=5):
    x = ss.uniform_complex(seed, 4, n, np.float64)
    y = fft_fn(x)
    lhs = np.sum(np.abs(y) ** 2, axis=1)
    rhs = n * np.sum(np.abs(x) ** 2, axis=1)
    return float(np.max(np.abs(lhs - rhs) / rhs))


def pin_linearity(fft_fn, n, seed=6):
    a = ss.uniform_complex(seed, 1, n, np.float64)
    b = ss.uniform_complex(seed + 1, 1, n, np.float64)
    al, be = 0.3 - 1.1j, -0.7 + 0.2j
    lhs = fft_fn(al * a + be * b)
    rhs = al * fft_fn(a) + be * fft_fn(b)
    return float(np.max(oracle.rel_l2(lhs, rhs)))


def pin_roundtrip(fft_fn, n, seed=7):
    x = ss.uniform_complex(seed, 2, n, np.float64)
    back = fft_fn(fft_fn(x), inverse=True)
    return float(np.max(oracle.rel_l2(back, x)))


def pin_numpy(fft_fn, n, seed=8):
    x = ss.uniform_complex(seed, 2, n, np.float64)
    return max(float(np.max(oracle.rel_l2(fft_fn(x), np.fft.fft(x, axis=1)))),
               float(np.max(oracle.rel_l2(fft_fn(x, inverse=True), np.fft.ifft(x, axis=1)))))


ALL_PINS = dict(naive=pin_vs_naive, impulse=pin_impulse, constant=pin_constant, tone=pin_tone,
                parseval=pin_parseval, linearity=pin_linearity, roundtrip=pin_roundtrip,
                numpy=pin_numpy)


def pins_pass(fft_fn, n):
    l = max(1, int(math.log2(n)))
    bar = 1e-14 * l
    results = {}
    results["naive"] = pin_vs_naive(fft_fn, n) <= bar and pin_vs_naive(fft_fn, n, inverse=True) <= bar
    results["impulse"] = pin_impulse(fft_fn, n) <= bar
    results["constant"] = pin_constant(fft_fn, n) <= bar
    results["tone"] = pin_tone(fft_fn, n) <= bar
    results["parseval"] = pin_parseval(fft_fn, n) <= bar
    results["linearity"] = pin_linearity(fft_fn, n) <= bar
    results["roundtrip"] = pin_roundtrip(fft_fn, n) <= bar
    results["numpy"] = pin_numpy(fft_fn, n) <= bar
    return results


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024])
def test_oracle_pins_small(n):
    res = pins_pass(oracle.fft, n)
    assert all(res.values()), res


@pytest.mark.parametrize("n", [1 << 12, 1 << 16])
def test_oracle_pins_large(n):
    l = int(math.log2(n))
    bar = 1e-14 * l
    assert pin_impulse(oracle.fft, n) <= bar
    assert pin_constant(oracle.fft, n) <= bar
    assert pin_tone(oracle.fft, n) <= bar
    assert pin_parseval(oracle.fft, n) <= bar
    assert pin_linearity(oracle.fft, n) <= bar
    assert pin_roundtrip(oracle.fft, n) <= bar
    assert pin_numpy(oracle.fft, n) <= bar


def test_oracle_max_size_tone_and_numpy():
    n = 1 << 20
    assert pin_tone(oracle.fft, n) <= 1e-14 * 20
    assert pin_numpy(oracle.fft, n) <= 1e-14 * 20


def test_inverse_unscaled_is_adjoint():
    """<F x, y> = <x, F^H y>: the unscaled inverse is the adjoint of forward."""
    n = 256
    x = ss.uniform_complex(21, 1, n, np.float64)[0]
    y = ss.uniform_complex(22, 1, n, np.float64)[0]
    lhs = np.vdot(y, oracle.fft(x))
    rhs = np.vdot(oracle.fft(y, inverse=True, scaled=False), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_float32_inputs_widened_exactly():
    x32 = ss.uniform_complex(3, 2, 64, np.float32)
    np.testing.assert_array_equal(oracle.fft(x32), oracle.fft(x32.astype(np.complex128)))


def test_batch_independent_of_threads():
    x = ss.uniform_complex(9, 64, 512, np.float64)
    a = oracle.fft(x, threads=1)
    b = oracle.fft(x, threads=4)
    np.testing.assert_array_equal(a, b)


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.zeros((1, 12), complex))


# ---------------------------------------------------------------------------
# planted mistakes (made here, in CPU-only stand-ins, never in the GPU path):
# each one must be caught by at least one pin
# ---------------------------------------------------------------------------
def _mut_sign(x, inverse=False):
    return oracle.fft(x, inverse=not inverse, scaled=False) if not inverse else oracle.fft(x) / x.shape[-1]


def _mut_no_scale(x, inverse=False):
    return oracle.fft(x, inverse=inverse, scaled=False)


def _mut_conj_input(x, inverse=False):
    return oracle.fft(np.conj(x), inverse=inverse)


def _mut_reversed_output(x, inverse=False):
    y = oracle.fft(x, inverse=inverse)
    return np.roll(y[..., ::-1], 1, axis=-1) if y.shape[-1] > 2 else y * 1.0000001


def _mut_bad_twiddle(x, inverse=False):
    # twiddle index off by one in the last stage: emulate via naive DFT with
    # exponent (j*n + n) instead of j*n
    x = np.atleast_2d(x)
    n = x.shape[-1]
    j = np.arange(n)[:, None]
    k = np.arange(n)[None, :]
    s = 1 if inverse else -1
    W = np.exp(s * 2j * np.pi * ((j * k + k) % n) / n)
    y = x @ W.T
    return y / n if inverse else y


@pytest.mark.parametrize("mut", [_mut_sign, _mut_no_scale, _mut_conj_input,
                                 _mut_reversed_output, _mut_bad_twiddle])
def test_pins_catch_planted_mistakes(mut):
    res = pins_pass(mut, 16)
    assert not all(res.values()), "planted mistake passed every pin"
