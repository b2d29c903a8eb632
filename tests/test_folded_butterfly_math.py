"""The float64 kernels' twiddled radix-8 (and radix-4, radix-2) passes run as
radix-2 layers with each twiddle folded into its butterfly,
a +- w b with w = c (1 + i t) (Linzer and Feig's factorisation for FMA
machines), using per-layer twiddles
    R = 8: omega^4, omega^2, W4 omega^2, omega, W4 omega, W8 omega, W8^3 omega
    R = 4: omega^2, omega, W4 omega
    R = 2: omega
for the pass twiddles w_{LR}^{k m} = omega^m.  These CPU checks restate that
network in numpy and compare it with the twiddled DFT it replaces (the
pass's definition: X_s = sum_m omega^m b_m W_R^{s m}), for every k of a few
(L, R), including the |Im w| > |Re w| form applied to i b."""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def root(n, q):
    return np.exp(-2j * np.pi * (q % n) / n)


def folded(w):
    """(c, t, rotated) with w = c (1 + i t), or w = c (1 + i t) i when rotated."""
    if abs(w.imag) > abs(w.real):
        return w.imag, -w.real / w.imag, True
    return w.real, w.imag / w.real, False


def bfly(a, b, w):
    c, t, rot = folded(w)
    p = 1j * b if rot else b
    u = p.real - t * p.imag
    v = p.imag + t * p.real
    return complex(a.real + c * u, a.imag + c * v), complex(a.real - c * u, a.imag - c * v)


def network(x, om, r):
    x = list(x)
    if r == 2:
        x[0], x[1] = bfly(x[0], x[1], om)
        return x
    w4, w8 = root(4, 1), root(8, 1)
    if r == 4:
        x[0], x[2] = bfly(x[0], x[2], om ** 2)
        x[1], x[3] = bfly(x[1], x[3], om ** 2)
        x[0], x[1] = bfly(x[0], x[1], om)
        x[2], x[3] = bfly(x[2], x[3], w4 * om)
        return [x[0], x[2], x[1], x[3]]
    for m in range(4):
        x[m], x[m + 4] = bfly(x[m], x[m + 4], om ** 4)
    x[0], x[2] = bfly(x[0], x[2], om ** 2)
    x[1], x[3] = bfly(x[1], x[3], om ** 2)
    x[4], x[6] = bfly(x[4], x[6], w4 * om ** 2)
    x[5], x[7] = bfly(x[5], x[7], w4 * om ** 2)
    x[0], x[1] = bfly(x[0], x[1], om)
    x[2], x[3] = bfly(x[2], x[3], w4 * om)
    x[4], x[5] = bfly(x[4], x[5], w8 * om)
    x[6], x[7] = bfly(x[6], x[7], w8 ** 3 * om)
    # the registers now hold X0, X4, X2, X6, X1, X5, X3, X7
    return [x[0], x[4], x[2], x[6], x[1], x[5], x[3], x[7]]


@pytest.mark.parametrize("r,l", [(8, 8), (8, 64), (4, 512), (2, 8), (4, 8), (8, 512)])
def test_folded_network_is_the_twiddled_dft(r, l):
    rng = np.random.default_rng(7)
    n = l * r
    for k in range(l):
        b = rng.standard_normal(r) + 1j * rng.standard_normal(r)
        om = root(n, k)
        want = [sum(om ** m * b[m] * root(r, s * m) for m in range(r)) for s in range(r)]
        got = network(b, om, r)
        assert np.allclose(got, want, rtol=0, atol=1e-13 * np.abs(b).sum()), (r, l, k)


def test_both_factorisations_cover_every_direction():
    # |t| <= 1 in either form, so the FMAs never scale a value up by more than 2
    for q in range(4096):
        c, t, rot = folded(root(4096, q))
        assert abs(t) <= 1 + 1e-15
        assert abs(c) >= np.sqrt(0.5) - 1e-15
