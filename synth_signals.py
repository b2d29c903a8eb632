"""Seeded synthetic input signals for batched complex FFT workloads.

This module holds only input generation: it contains none of the FFT or
checksum arithmetic.  Both the CPU oracle tests and the CUDA parity tests /
benchmark draw their inputs from here, so the two sides see bit-identical
data.

Random values come from a counter-based SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; the
finaliser constants are those of Vigna's public-domain splitmix64.c):

    key      = mix(seed + GAMMA)
    word(i)  = mix(key + (i + 1) * GAMMA)          (all mod 2^64)
    mix(z)   : z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
               z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31

Element i of a batch (i = b * n + k) takes its real part from word(2i) and its
imaginary part from word(2i + 1).  A uniform value in [-1, 1) is
(word >> 40) * 2^-23 - 1 for float32 data and (word >> 11) * 2^-52 - 1 for
float64 data; both are exactly representable in the target precision.

Structured inputs (impulse, constant, tone with k = round(N/3)) follow the
configurations of the size sweep.  The tone is evaluated with the phase
reduced exactly in integers and the trigonometric functions in numpy's
longdouble, then rounded to the target precision.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

__all__ = [
    "splitmix_words",
    "uniform_complex",
    "normal_complex",
    "impulse",
    "constant",
    "tone",
    "structured",
    "uniform_complex_torch",
    "ragged_sizes",
    "ragged_offsets",
]


def _mix_np(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(M1)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(M2)
    return z ^ (z >> np.uint64(31))


def _key(seed: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return _mix_np(np.array([(seed + GAMMA) & MASK64], dtype=np.uint64))[0]


def splitmix_words(seed: int, start: int, count: int) -> np.ndarray:
    """word(start), ..., word(start + count - 1) as uint64."""
    key = _key(seed)
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix_np(key + idx * np.uint64(GAMMA))


def _to_uniform(words: np.ndarray, dtype) -> np.ndarray:
    if np.dtype(dtype) == np.float32:
        return ((words >> np.uint64(40)).astype(np.float64) * 2.0**-23 - 1.0).astype(np.float32)
    return (words >> np.uint64(11)).astype(np.float64) * 2.0**-52 - 1.0


def uniform_complex(seed: int, batch: int, n: int, dtype=np.float32,
                    first_element: int = 0) -> np.ndarray:
    """[batch, n] complex array, real and imaginary parts i.i.d. uniform[-1,1).

    dtype is the real precision (float32 -> complex64, float64 -> complex128).
    first_element offsets the counter, so a slice of a large batch can be
    generated on its own and equals the same rows of the full batch."""
    count = batch * n
    out = np.empty(count, dtype=np.complex64 if np.dtype(dtype) == np.float32 else np.complex128)
    chunk = 1 << 22
    for s in range(0, count, chunk):
        m = min(chunk, count - s)
        w = splitmix_words(seed, 2 * (first_element + s), 2 * m)
        u = _to_uniform(w, dtype)
        out.real[s:s + m] = u[0::2]
        out.imag[s:s + m] = u[1::2]
    return out.reshape(batch, n)


def normal_complex(seed: int, batch: int, n: int, dtype=np.float32) -> np.ndarray:
    """[batch, n] complex array with standard-normal real and imaginary parts
    (Box-Muller on two uniform words per element)."""
    count = batch * n
    w = splitmix_words(seed, 0, 2 * count)
    u1 = ((w[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0**-53  # (0, 1]
    u2 = (w[1::2] >> np.uint64(11)).astype(np.float64) * 2.0**-53
    r = np.sqrt(-2.0 * np.log(u1))
    z = r * np.cos(2 * np.pi * u2) + 1j * r * np.sin(2 * np.pi * u2)
    ctype = np.complex64 if np.dtype(dtype) == np.float32 else np.complex128
    return z.astype(ctype).reshape(batch, n)


def _ctype(dtype):
    return np.complex64 if np.dtype(dtype) == np.float32 else np.complex128


def ragged_sizes(seed: int, count: int, lo_log: int = 6, hi_log: int = 16) -> np.ndarray:
    """Transform sizes 2^k with k drawn uniformly from [lo_log, hi_log]
    (log-uniform over the powers of two), as int64.  k = lo_log +
    floor(hi32(word(i)) * m / 2^32), m = hi_log - lo_log + 1."""
    m = np.uint64(hi_log - lo_log + 1)
    w = splitmix_words(seed, 0, count)
    k = ((w >> np.uint64(32)) * m) >> np.uint64(32)
    return (np.int64(1) << (k.astype(np.int64) + lo_log)).astype(np.int64)


def ragged_offsets(sizes, seed: int | None = None, max_gap: int = 0) -> tuple[np.ndarray, int]:
    """Element offsets of transforms packed in order; with a seed, an even gap
    in [0, max_gap) precedes each transform (gaps keep every start 16-byte
    aligned for complex64).  Returns (offsets int64, total span)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    gaps = np.zeros(len(sizes), dtype=np.int64)
    if seed is not None and max_gap > 1:
        w = splitmix_words(seed, 0, len(sizes))
        gaps = 2 * ((w >> np.uint64(33)) % np.uint64(max_gap // 2)).astype(np.int64)
    ends = np.cumsum(gaps + sizes)
    offsets = ends - sizes
    return offsets.astype(np.int64), int(ends[-1]) if len(sizes) else 0


def impulse(batch: int, n: int, dtype=np.float32, position: int = 0) -> np.ndarray:
    x = np.zeros((batch, n), dtype=_ctype(dtype))
    x[:, position] = 1.0
    return x


def constant(batch: int, n: int, dtype=np.float32, value: complex = 1.0 + 0.0j) -> np.ndarray:
    return np.full((batch, n), value, dtype=_ctype(dtype))


def tone_index(n: int) -> int:
    """k = round(N/3), the tone frequency of the size-sweep configuration."""
    return int(np.floor(n / 3.0 + 0.5))


def tone(batch: int, n: int, dtype=np.float32, k: int | None = None) -> np.ndarray:
    """x_m = exp(+2 pi i k m / N), phase reduced exactly, longdouble trig."""
    if k is None:
        k = tone_index(n)
    m = np.arange(n, dtype=np.int64)
    q = (m * (k % n)) % n
    ang = (2 * np.pi * np.longdouble(1)) * q.astype(np.longdouble) / np.longdouble(n)
    row = np.empty(n, dtype=_ctype(dtype))
    row.real = np.cos(ang).astype(np.float64)
    row.imag = np.sin(ang).astype(np.float64)
    return np.broadcast_to(row, (batch, n)).copy()


def structured(kind: str, batch: int, n: int, dtype=np.float32, seed: int = 2) -> np.ndarray:
    if kind == "uniform":
        return uniform_complex(seed, batch, n, dtype)
    if kind == "impulse":
        return impulse(batch, n, dtype)
    if kind == "constant":
        return constant(batch, n, dtype)
    if kind == "tone":
        return tone(batch, n, dtype)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# Device-side generation (torch int64 arithmetic wraps modulo 2^64, so the
# same words come out); used where a full-size batch would be slow to build
# on the host.  Bit-identical to uniform_complex.
# ---------------------------------------------------------------------------
def _s64(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _mix_torch(z):
    import torch  # noqa: F401
    z = z ^ ((z >> 30) & ((1 << 34) - 1))
    z = z * _s64(M1)
    z = z ^ ((z >> 27) & ((1 << 37) - 1))
    z = z * _s64(M2)
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def uniform_complex_torch(seed: int, batch: int, n: int, dtype: str = "float32",
                          device="cuda", out=None):
    """Same values as uniform_complex(seed, batch, n, dtype) built on device.

    Returns a torch complex tensor [batch, n] (complex64 or complex128)."""
    import torch
    key = int(_key(seed))
    count = batch * n
    cdt = torch.complex64 if dtype == "float32" else torch.complex128
    rdt = torch.float32 if dtype == "float32" else torch.float64
    if out is None:
        out = torch.empty((batch, n), dtype=cdt, device=device)
    flat = torch.view_as_real(out.view(-1))
    chunk = 1 << 24
    g = _s64(GAMMA)
    for s in range(0, count, chunk):
        m = min(chunk, count - s)
        idx = torch.arange(2 * s + 1, 2 * (s + m) + 1, dtype=torch.int64, device=device)
        z = idx * g + _s64(key)
        z = _mix_torch(z)
        if dtype == "float32":
            u = ((z >> 40) & ((1 << 24) - 1)).to(torch.float64) * 2.0**-23 - 1.0
        else:
            u = ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * 2.0**-52 - 1.0
        flat[s:s + m] = u.to(rdt).view(m, 2)
    return out
