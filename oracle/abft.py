"""Two-sided ABFT for a batch of DFTs, step by step, in float64 (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The method (TurboFFT):
  * Left-side checksum (Sec. 2.2.2, Eq. 1-2): for an encoding vector e the
    encoded DFT matrix has the extra row e^T W, so for every signal
    (e^T W) x_b = e^T (W x_b).  v := (e^T W)^T = W e because W is symmetric;
    v is the forward DFT of e.  Detection compares s_in,b = v . x_b with
    s_out,b = e . y_b.
  * Location encoding (Sec. 4.1 and Sec. 4.3): a second vector (1, 2, ...)
    weights the signals of a group, so with r_b = s_out,b - s_in,b,
        S1 = sum_b r_b,   S2 = sum_b (b + 1) r_b,
    and under the single-event-upset model (Sec. 2.2.4) one corrupted signal
    k gives S2 / S1 = k + 1.
  * Right-side checksum (Eq. 3-5): the group sums x_bar = X e, y_bar = Y e
    (e = ones over the batch).  By linearity y_bar = W x_bar for a clean
    group, so Delta = y_bar - W x_bar is the error of the corrupted signal and
    y_k <- y_k - Delta corrects it (Sec. 4.1.1; delayed, batched correction of
    Sec. 4.1.2: the group is checked once, after all its signals).

Readings where the paper is silent:
  * e: seeded unit-modulus random phases (default) or Wang's
    e_j = omega_3^j (Sec. 2.2.2) or all ones.
  * detection threshold: |S1| > tau with
        tau = gamma * u * sqrt(log2 N) * sqrt(sum_b ||y_b||^2),
    u the unit roundoff of the working precision, ||y_b||^2 from Parseval.
  * location accepted when q = S2/S1 is within 0.25 of an integer k+1 in
    [1, G]; otherwise every signal is rechecked on its own (rare path).
  * a non-finite checksum is located by the signal whose own residual is
    non-finite.
  * correction re-checks the corrected signal; if the paper's Delta
    correction does not pass (e.g. Delta is not finite), the signal is
    recomputed from its untouched input; if that fails too, the group is
    reported uncorrectable.  After a correction every other signal of the
    group is re-verified on its own checksum: more than one corrupted signal
    in a group violates the single-event model and is reported
    uncorrectable.
"""
from __future__ import annotations

import math

import numpy as np

from . import fft as _fft

UNIT_ROUNDOFF = {np.dtype(np.float32): 2.0**-24, np.dtype(np.float64): 2.0**-53}
# gamma per working precision (reading: chosen from clean-run residuals so
# that the largest clean |S1| stays several times below tau)
GAMMA = {np.dtype(np.float32): 8.0, np.dtype(np.float64): 16.0}
GAMMA_DEFAULT = None  # None -> GAMMA[precision]


# ---------------------------------------------------------------------------
# encoding vectors
# ---------------------------------------------------------------------------
_G64 = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _splitmix_mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * np.uint64(_M1)
        z = z ^ (z >> np.uint64(27))
        z = z * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def encoding_vector(n: int, kind: str = "phase", seed: int = 0x5EED) -> np.ndarray:
    """Left encoding vector e (complex128, length n).

    phase: e_j = exp(2 pi i theta_j), theta_j = word_j / 2^64 with word_j the
           j-th output of a SplitMix64 stream started at seed.
    wang:  e_j = omega_3^j = exp(-2 pi i j / 3)   (Sec. 2.2.2)
    ones:  e_j = 1."""
    if kind == "ones":
        return np.ones(n, dtype=np.complex128)
    if kind == "wang":
        j = np.arange(n) % 3
        ang = -2.0 * np.pi * j / 3.0
        return np.cos(ang) + 1j * np.sin(ang)
    if kind == "phase":
        with np.errstate(over="ignore"):
            st = np.uint64(seed) + np.arange(1, n + 1, dtype=np.uint64) * np.uint64(_G64)
        w = _splitmix_mix(st)
        theta = (w >> np.uint64(11)).astype(np.float64) * 2.0**-53
        return np.exp(2j * np.pi * theta)
    raise ValueError(kind)


def left_vector(e: np.ndarray, inverse: bool = False, scaled: bool = True) -> np.ndarray:
    """v = A^T e for the transform matrix A (A = W forward; A = conj(W)/N or
    conj(W) inverse).  Both matrices are symmetric, so v = A e: the transform
    of e itself (Eq. 1)."""
    return _fft(e, inverse=inverse, scaled=scaled)


# ---------------------------------------------------------------------------
# checksums and the group decision
# ---------------------------------------------------------------------------
def _mag(z) -> float:
    """|z| that returns inf instead of raising on overflow."""
    with np.errstate(all="ignore"):
        return float(np.abs(np.complex128(z)))


def checksums(x: np.ndarray, y: np.ndarray, e: np.ndarray, v: np.ndarray):
    """Per-signal left checksums s_in,b = v . x_b and s_out,b = e . y_b
    (unconjugated dot products, Eq. 1-2) in float64."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    with np.errstate(all="ignore"):
        # elementwise products, then numpy's pairwise summation along a row
        return np.sum(x * v, axis=-1), np.sum(y * e, axis=-1)


def threshold(x: np.ndarray, n: int, precision, gamma: float = GAMMA_DEFAULT,
              parseval: float | None = None) -> float:
    """tau = gamma * u * sqrt(log2 N) * sqrt(sum_b ||y_b||^2), where
    ||y_b||^2 = parseval * ||x_b||^2 (parseval = N for the forward transform)."""
    u = UNIT_ROUNDOFF[np.dtype(precision)]
    if gamma is None:
        gamma = GAMMA[np.dtype(precision)]
    if parseval is None:
        parseval = float(n)
    energy = float(np.sum(np.abs(np.asarray(x, dtype=np.complex128)) ** 2))
    return gamma * u * math.sqrt(max(1.0, math.log2(n))) * math.sqrt(parseval * energy)


def group_check(x, y, e, v, precision, gamma: float = GAMMA_DEFAULT,
                parseval: float | None = None) -> dict:
    """Detect and locate a corrupted signal in one group (rows of x / y).

    Returns a dict with S1, S2, tau, detected, location (signal index or
    None), method ('encoding' | 'nonfinite' | 'recheck') and bad (all signals
    the per-signal recheck flags, when it ran)."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    G, n = x.shape
    s_in, s_out = checksums(x, y, e, v)
    with np.errstate(all="ignore"):
        r = s_out - s_in
        w = np.arange(1, G + 1, dtype=np.float64)
        S1 = complex(np.sum(r))
        S2 = complex(np.sum(w * r))
    tau = threshold(x, n, precision, gamma, parseval)
    res = dict(S1=S1, S2=S2, tau=tau, detected=False, location=None, method=None, bad=[])
    finite = math.isfinite(S1.real) and math.isfinite(S1.imag)
    if finite and _mag(S1) <= tau:
        return res
    res["detected"] = True
    if not finite:
        bad = [b for b in range(G) if not (np.isfinite(r[b].real) and np.isfinite(r[b].imag))]
        res["method"] = "nonfinite"
        res["bad"] = bad
        res["location"] = bad[0] if len(bad) == 1 else None
        return res
    with np.errstate(all="ignore"):
        q = S2 / S1
    k = int(math.floor(q.real + 0.5)) - 1 if (math.isfinite(q.real) and math.isfinite(q.imag)) else -1
    if 0 <= k < G and _mag(q - (k + 1)) < 0.25:
        res["method"] = "encoding"
        res["location"] = k
        return res
    # ambiguous location: recheck every signal on its own threshold
    res["method"] = "recheck"
    bad = []
    for b in range(G):
        tb = threshold(x[b:b + 1], n, precision, gamma, parseval)
        if not (_mag(r[b]) <= tb):
            bad.append(b)
    res["bad"] = bad
    res["location"] = bad[0] if len(bad) == 1 else None
    return res


def correct_group(x, y, e, v, precision, gamma: float = GAMMA_DEFAULT,
                  inverse: bool = False, scaled: bool = True) -> tuple[np.ndarray, dict]:
    """Detect, locate and correct one group.  Returns (corrected y, report).

    report: detected, location, corrected (bool), uncorrectable (bool),
    how ('delta' | 'recompute' | None)."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.array(y, dtype=np.complex128, copy=True)
    G, n = x.shape
    parseval = (1.0 / n if scaled else float(n)) if inverse else float(n)
    rep = group_check(x, y, e, v, precision, gamma, parseval)
    rep.update(corrected=False, uncorrectable=False, how=None)
    if not rep["detected"]:
        return y, rep
    k = rep["location"]
    if k is None:
        rep["uncorrectable"] = True
        return y, rep

    def passes(row_y, row_x):
        s_in, s_out = checksums(row_x[None, :], row_y[None, :], e, v)
        rr = complex(s_out[0] - s_in[0])
        tb = threshold(row_x[None, :], n, precision, gamma, parseval)
        return math.isfinite(rr.real) and math.isfinite(rr.imag) and _mag(rr) <= tb

    def group_passes(yy):
        # after the fix every other signal of the group must pass its own
        # checksum test: a second corrupted signal (outside the single-event
        # model) would still show here
        return all(passes(yy[b], x[b]) for b in range(G) if b != k)

    # paper's correction: Delta = y_bar - W x_bar, y_k <- y_k - Delta
    with np.errstate(all="ignore"):
        x_bar = x.sum(axis=0)
        y_bar = y.sum(axis=0)
        delta = y_bar - _fft(x_bar, inverse=inverse, scaled=scaled)
        cand = y[k] - delta
    how = None
    if np.all(np.isfinite(cand)) and passes(cand, x[k]):
        how = "delta"
    else:
        # fallback: recompute the signal from its untouched input
        cand = _fft(x[k], inverse=inverse, scaled=scaled)
        if passes(cand, x[k]):
            how = "recompute"
    if how is not None:
        fixed = y.copy()
        fixed[k] = cand
        if group_passes(fixed):
            rep.update(corrected=True, how=how)
            return fixed, rep
    rep["uncorrectable"] = True
    return y, rep


# ---------------------------------------------------------------------------
# radix-2 FFT with a host-side bit flip (fault experiments, Sec. 5.3.1)
# ---------------------------------------------------------------------------
def flip_bit(value, bit: int, precision):
    """Flip one bit of the IEEE representation of a real scalar."""
    if np.dtype(precision) == np.float32:
        a = np.array([value], dtype=np.float32).view(np.uint32)
        a ^= np.uint32(1 << bit)
        return a.view(np.float32)[0]
    a = np.array([value], dtype=np.float64).view(np.uint64)
    a ^= np.uint64(1 << bit)
    return a.view(np.float64)[0]


def fft_radix2(x, precision=np.float64, fault: dict | None = None) -> np.ndarray:
    """Iterative radix-2 DIT FFT of one signal carried out in `precision`.

    fault = dict(stage=s, element=i, component=0|1, bit=b) flips bit b of the
    real (0) or imaginary (1) part of working-array element i as it enters
    butterfly stage s (s = 0 is the bit-reversed input, s = log2 N the final
    output).  Returns the result in the working precision's complex type."""
    ctype = np.complex64 if np.dtype(precision) == np.float32 else np.complex128
    x = np.asarray(x)
    n = x.shape[-1]
    logn = int(round(math.log2(n)))
    assert 1 << logn == n
    rev = np.array([int(format(i, "0%db" % logn)[::-1], 2) if logn else 0 for i in range(n)])
    a = np.asarray(x, dtype=ctype)[rev].copy()
    k = np.arange(max(1, n // 2))
    ang = -2.0 * np.pi * k.astype(np.longdouble) / np.longdouble(n)
    tw = (np.cos(ang).astype(np.float64) + 1j * np.sin(ang).astype(np.float64)).astype(ctype)

    def inject(stage):
        if fault is not None and fault["stage"] == stage:
            i, c, b = fault["element"], fault["component"], fault["bit"]
            if c == 0:
                a[i] = ctype(complex(flip_bit(a[i].real, b, precision), a[i].imag))
            else:
                a[i] = ctype(complex(a[i].real, flip_bit(a[i].imag, b, precision)))

    with np.errstate(all="ignore"):
        for s in range(logn):
            inject(s)
            m = 2 << s
            half = m >> 1
            a2 = a.reshape(n // m, m)
            w = tw[(np.arange(half) * (n // m))]
            t = a2[:, half:] * w
            u = a2[:, :half].copy()
            a2[:, :half] = u + t
            a2[:, half:] = u - t
        inject(logn)
    return a
