"""Differentiable spectral filter y = IFFT(W * FFT(x)), loss = sum |y|^2,
with forward and backward through the library's kernels (backward = the
adjoint transforms), ABFT on: gradients against the oracle's closed forms
and against float64 central differences."""
import numpy as np
import pytest

import oracle
import synth_signals as ss
from oracle import spectral

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402
from paper_2412_05824_gb300 import autograd as tag  # noqa: E402


def _slice(dtype):
    x = ss.uniform_complex(31, 4, 64, np.float32 if dtype == torch.complex64 else np.float64).reshape(2, 2, 64)
    g = torch.Generator().manual_seed(5)
    rdt = torch.float32 if dtype == torch.complex64 else torch.float64
    w = torch.complex(torch.normal(0, 1 / 8, (2, 64), generator=g, dtype=rdt),
                      torch.normal(0, 1 / 8, (2, 64), generator=g, dtype=rdt))
    return x, w.numpy()


def _torch_grads(x, w, dtype, ft="correct"):
    xt = torch.tensor(x, dtype=dtype, device="cuda", requires_grad=True)
    wt = torch.tensor(w, dtype=dtype, device="cuda", requires_grad=True)
    y = tag.spectral_filter(xt, wt, ft)
    loss = (y.abs() ** 2).sum()
    loss.backward()
    return float(loss.detach()), xt.grad.cpu().numpy(), wt.grad.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_slice_matches_closed_form(dtype):
    x, w = _slice(dtype)
    L, gx, gw = _torch_grads(x, w, dtype)
    rgx, rgw = spectral.grads(x, w)
    prec = np.float32 if dtype == torch.complex64 else np.float64
    tol = 4 * oracle.tolerance(prec, 64)  # four transforms composed
    assert abs(L - spectral.loss(x, w)) <= tol * spectral.loss(x, w)
    assert _rel(gx, rgx) <= tol and _rel(gw, rgw) <= tol


def test_slice_matches_central_differences_float64():
    x, w = _slice(torch.complex128)

    def loss_x(z):
        with torch.no_grad():
            zt = torch.tensor(z, device="cuda")
            y = tag.spectral_filter(zt, torch.tensor(w, device="cuda"))
            return float((y.abs() ** 2).sum())

    def loss_w(z):
        with torch.no_grad():
            y = tag.spectral_filter(torch.tensor(x, device="cuda"), torch.tensor(z, device="cuda"))
            return float((y.abs() ** 2).sum())

    _, gx, gw = _torch_grads(x, w, torch.complex128)
    fdx = spectral.finite_difference(loss_x, x, 1e-6)
    fdw = spectral.finite_difference(loss_w, w, 1e-6)
    assert _rel(gx, fdx) <= 1e-6 and _rel(gw, fdw) <= 1e-6


def test_adjointness_of_the_kernels():
    """<F x, y> = <x, F^H y> for the forward / unscaled inverse kernels and
    <iF x, y> = <x, (1/N) F y> for the scaled pair."""
    n = 512
    x = torch.tensor(ss.uniform_complex(1, 8, n, np.float64), device="cuda")
    y = torch.tensor(ss.uniform_complex(2, 8, n, np.float64), device="cuda")
    f = tfl.Plan(n, 8, "complex128", "forward")
    fh = tfl.Plan(n, 8, "complex128", "inverse_unscaled")
    inv = tfl.Plan(n, 8, "complex128", "inverse")
    fs = tfl.Plan(n, 8, "complex128", "forward_scaled")
    a = torch.vdot(y.flatten(), f.exec(x).flatten())
    b = torch.vdot(fh.exec(y).flatten(), x.flatten())
    assert abs(complex(a - b)) <= 1e-12 * abs(complex(a))
    a = torch.vdot(y.flatten(), inv.exec(x).flatten())
    b = torch.vdot(fs.exec(y).flatten(), x.flatten())
    assert abs(complex(a - b)) <= 1e-12 * abs(complex(a))


def test_full_size_config():
    """x [64, 128, 4096] complex64 uniform[-1,1), W [128, 4096] with N(0, 1/64)
    real and imaginary parts; gradients against the closed forms."""
    b, ch, n = 64, 128, 4096
    x = ss.uniform_complex(6, b * ch, n, np.float32).reshape(b, ch, n)
    g = torch.Generator().manual_seed(6)
    w = torch.complex(torch.normal(0, 1 / 64, (ch, n), generator=g),
                      torch.normal(0, 1 / 64, (ch, n), generator=g)).numpy()
    L, gx, gw = _torch_grads(x, w, torch.complex64)
    rgx, rgw = spectral.grads(x, w)
    tol = 4 * oracle.tolerance(np.float32, n)
    assert _rel(gx, rgx) <= tol and _rel(gw, rgw) <= tol
    assert abs(L - spectral.loss(x, w)) <= tol * abs(L)
    # the ABFT of every transform of forward and backward stayed clean
    for p in tag._plans.values():
        rep = p.report()
        assert rep["detected"] == 0
