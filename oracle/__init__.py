"""CPU oracle for the batched 1-D complex FFT with two-sided ABFT.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this package.  It shares no code with the
CUDA path (paper_2412_05824_gb300) and never imports it.

Contents
  fft(x, inverse, scaled)      batched radix-2 FFT in float64 (C, OpenMP)
                               -- TurboFFT Sec. 2.2.1, definition of the DFT
  dft_naive(x, inverse)        O(N^2) definition in long double (C)
                               -- TurboFFT Sec. 2.2.1
  oracle.abft                  two-sided checksum encode / detect / locate /
                               correct, and a radix-2 FFT with a host-side bit
                               flip for fault experiments
                               -- TurboFFT Sec. 2.2.2 Eq. 1-3, Sec. 4.1 Eq. 4-5,
                                  Sec. 4.3, Sec. 5.3.1
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def lib():
    """The compiled C part of the oracle (built on first use)."""
    global _lib
    if _lib is None:
        from . import build as _build
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_fft.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, dp, dp,
                                 ctypes.c_double, ctypes.c_int]
        L.oracle_fft.restype = ctypes.c_int
        L.oracle_dft_naive.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, ctypes.c_double]
        L.oracle_dft_naive.restype = None
        L.oracle_last_threads.restype = ctypes.c_int
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _as_c128(x) -> np.ndarray:
    x = np.asarray(x)
    if x.ndim == 1:
        x = x[None, :]
    return np.ascontiguousarray(x, dtype=np.complex128)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def fft(x, inverse: bool = False, scaled: bool = True, threads: int = 0) -> np.ndarray:
    """Batched transform of the rows of x ([batch, n] or [n]) in float64.

    forward:  y_j = sum_n x_n exp(-2 pi i j n / N)
    inverse:  x_j = (1/N) sum_n y_n exp(+2 pi i j n / N)   (scaled=True)
              or the same sum without 1/N                  (scaled=False)
    Input values are widened exactly to complex128; the result is complex128
    with the input's leading shape."""
    squeeze = np.asarray(x).ndim == 1
    a = _as_c128(x)
    batch, n = a.shape
    out = np.empty_like(a)
    sign = 1 if inverse else -1
    scale = (1.0 / n) if (inverse and scaled) else 1.0
    rc = lib().oracle_fft(n, batch, sign, _dptr(a), _dptr(out), scale, int(threads))
    if rc != 0:
        raise ValueError("oracle fft: n must be a power of two (got %d)" % n)
    return out[0] if squeeze else out


def last_threads() -> int:
    """OpenMP threads used by the most recent fft() call."""
    return int(lib().oracle_last_threads())


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def dft_naive(x, inverse: bool = False, scaled: bool = True) -> np.ndarray:
    """Definition of the DFT summed term by term in long double (small n)."""
    squeeze = np.asarray(x).ndim == 1
    a = _as_c128(x)
    batch, n = a.shape
    out = np.empty_like(a)
    sign = 1 if inverse else -1
    scale = (1.0 / n) if (inverse and scaled) else 1.0
    L = lib()
    for b in range(batch):
        row_in = np.ascontiguousarray(a[b])
        row_out = np.empty_like(row_in)
        L.oracle_dft_naive(n, sign, _dptr(row_in), _dptr(row_out), scale)
        out[b] = row_out
    return out[0] if squeeze else out


def rel_l2(y_hat, y_ref, axis=-1) -> np.ndarray:
    """Relative L2 error ||y_hat - y_ref|| / ||y_ref|| per transform (rows),
    the absolute error where ||y_ref|| = 0 (accuracy criterion of the size
    sweep; reading: the maximum over transforms is what must meet the bar)."""
    y_hat = np.asarray(y_hat, dtype=np.complex128)
    y_ref = np.asarray(y_ref, dtype=np.complex128)
    num = np.sqrt(np.sum(np.abs(y_hat - y_ref) ** 2, axis=axis))
    den = np.sqrt(np.sum(np.abs(y_ref) ** 2, axis=axis))
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def tolerance(dtype, n: int) -> float:
    """Accuracy bar: 2e-6*log2(N) for float32 data, 5e-15*log2(N) for float64."""
    l = max(1, int(np.log2(n)))
    return (2e-6 if np.dtype(dtype) in (np.float32, np.complex64) else 5e-15) * l
