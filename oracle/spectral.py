"""Oracle for the differentiable spectral filter (test infrastructure).

Model: y = IFFT(W * FFT(x)) over the last axis, W broadcast over the leading
(batch) axes, loss L = sum |y|^2, with FFT / IFFT the DFT and its 1/N
inverse (TurboFFT Sec. 2.2.1).

Closed forms (Parseval: L = (1/N) sum |W|^2 |FFT(x)|^2), in PyTorch's
convention grad = dL/dRe + i dL/dIm = 2 dL/d(conj z):
    grad_x = 2 IFFT(|W|^2 * FFT(x))
    grad_W = (2/N) W * sum_batch |FFT(x)|^2
All in float64 with the oracle FFT.
"""
from __future__ import annotations

import numpy as np

from . import fft as _fft


def loss(x, w) -> float:
    X = _fft(np.asarray(x, dtype=np.complex128).reshape(-1, x.shape[-1])).reshape(x.shape)
    y = _fft((X * w).reshape(-1, x.shape[-1]), inverse=True).reshape(x.shape)
    return float(np.sum(np.abs(y) ** 2))


def grads(x, w):
    """(grad_x, grad_W) by the closed forms."""
    n = x.shape[-1]
    x = np.asarray(x, dtype=np.complex128)
    w = np.asarray(w, dtype=np.complex128)
    X = _fft(x.reshape(-1, n)).reshape(x.shape)
    gx = 2.0 * _fft((np.abs(w) ** 2 * X).reshape(-1, n), inverse=True).reshape(x.shape)
    lead = tuple(range(x.ndim - w.ndim))
    gw = (2.0 / n) * w * np.sum(np.abs(X) ** 2, axis=lead)
    return gx, gw


def finite_difference(fn, z, h=1e-6):
    """Central differences of a real function of a complex array, in the
    convention grad = dL/dRe + i dL/dIm."""
    z = np.array(z, dtype=np.complex128, copy=True)
    g = np.zeros_like(z)
    flat = z.reshape(-1)
    gf = g.reshape(-1)
    for i in range(flat.size):
        v = flat[i]
        flat[i] = v + h
        lp = fn(z)
        flat[i] = v - h
        lm = fn(z)
        flat[i] = v + 1j * h
        ip = fn(z)
        flat[i] = v - 1j * h
        im = fn(z)
        flat[i] = v
        gf[i] = (lp - lm) / (2 * h) + 1j * (ip - im) / (2 * h)
    return g
