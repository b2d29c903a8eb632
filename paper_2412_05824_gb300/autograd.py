"""Differentiable FFTs on the library's kernels (argument marshalling only).

For a linear map y = A x, the backward pass of a real-valued loss is
grad_x = A^H grad_y (PyTorch's complex convention).  With W the DFT matrix
(forward transform, TurboFFT Sec. 2.2.1):

    y = W x            ->  grad_x = W^H grad_y        (unscaled inverse kernel)
    y = (1/N) W^H x    ->  grad_x = (1/N) W grad_y    (scaled forward kernel)

Both directions run in the same CUDA kernels, with the two-sided ABFT on when
requested, so the backward pass is fault tolerant too.
"""
from __future__ import annotations

import torch

from . import FORWARD, FORWARD_SCALED, INVERSE, INVERSE_UNSCALED, Plan

_plans: dict = {}


def _plan(n: int, batch: int, dtype, direction: int, ft: str, device) -> Plan:
    key = (n, batch, dtype, direction, ft, device.index)
    p = _plans.get(key)
    if p is None:
        p = _plans[key] = Plan(n, batch, dtype, direction, ft)
    return p


def _run(x: torch.Tensor, direction: int, ft: str) -> torch.Tensor:
    n = x.shape[-1]
    xc = x.contiguous()
    batch = xc.numel() // n
    return _plan(n, batch, xc.dtype, direction, ft, xc.device).exec(xc.view(batch, n)).view(x.shape)


class FFT(torch.autograd.Function):
    """y = FFT(x) over the last dimension (unscaled forward DFT)."""

    @staticmethod
    def forward(ctx, x, ft="correct"):
        ctx.ft = ft
        return _run(x, FORWARD, ft)

    @staticmethod
    def backward(ctx, gy):
        # adjoint of W: W^H = the unscaled inverse (conjugate-direction) transform
        return _run(gy, INVERSE_UNSCALED, ctx.ft), None


class IFFT(torch.autograd.Function):
    """y = IFFT(x) = (1/N) W^H x over the last dimension."""

    @staticmethod
    def forward(ctx, x, ft="correct"):
        ctx.ft = ft
        return _run(x, INVERSE, ft)

    @staticmethod
    def backward(ctx, gy):
        # adjoint of (1/N) W^H: (1/N) W, the scaled forward kernel
        return _run(gy, FORWARD_SCALED, ctx.ft), None


def fft(x: torch.Tensor, ft: str = "correct") -> torch.Tensor:
    return FFT.apply(x, ft)


def ifft(x: torch.Tensor, ft: str = "correct") -> torch.Tensor:
    return IFFT.apply(x, ft)


def spectral_filter(x: torch.Tensor, w: torch.Tensor, ft: str = "correct") -> torch.Tensor:
    """y = IFFT(W * FFT(x)) with W broadcast over the leading (batch) dims."""
    return ifft(fft(x, ft) * w, ft)
