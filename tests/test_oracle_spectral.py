"""Pins for the oracle's spectral-filter gradients: the closed forms against
float64 central differences (h = 1e-6) on a [2, 2, 64] problem, and the loss
against Parseval computed without the inverse transform."""
import numpy as np

import oracle
import synth_signals as ss
from oracle import spectral


def _problem(seed=3):
    x = ss.uniform_complex(seed, 4, 64, np.float64).reshape(2, 2, 64)
    rng = np.random.default_rng(seed)
    w = (rng.normal(0, 1 / 8, (2, 64)) + 1j * rng.normal(0, 1 / 8, (2, 64)))
    return x, w


def test_loss_is_parseval():
    x, w = _problem()
    X = oracle.dft_naive(x.reshape(-1, 64)).reshape(x.shape)
    assert abs(spectral.loss(x, w) - np.sum(np.abs(w) ** 2 * np.abs(X) ** 2) / 64) <= 1e-12 * spectral.loss(x, w)


def test_grad_x_matches_central_differences():
    x, w = _problem()
    gx, _ = spectral.grads(x, w)
    fd = spectral.finite_difference(lambda z: spectral.loss(z, w), x)
    assert np.max(np.abs(gx - fd)) <= 1e-6 * np.max(np.abs(gx))


def test_grad_w_matches_central_differences():
    x, w = _problem(4)
    _, gw = spectral.grads(x, w)
    fd = spectral.finite_difference(lambda z: spectral.loss(x, z), w)
    assert np.max(np.abs(gw - fd)) <= 1e-6 * np.max(np.abs(gw))
