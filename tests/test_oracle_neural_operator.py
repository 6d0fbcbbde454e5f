"""Pins of the FP64 neural-operator reference: its backward pass against central
finite differences, the DFT pair against numpy's FFT, and GELU against its definition."""
import math

import numpy as np
import pytest

from oracle.neural_operator import NeuralOperator, dft_matrices, dgelu, gelu


def test_dft_pair_matches_numpy_fft():
    M, K = 16, 8
    D, Dinv = dft_matrices(M, K)
    x = np.random.default_rng(1).normal(size=M)
    X = np.fft.fft(x)
    np.testing.assert_allclose(D[0::2] @ x, X[:K].real, atol=1e-12)
    np.testing.assert_allclose(D[1::2] @ x, X[:K].imag, atol=1e-12)
    # a band-limited signal (modes < K) is reproduced by the truncated inverse
    m = np.arange(M)
    y = 0.3 + np.cos(2 * math.pi * 3 * m / M) - 0.5 * np.sin(2 * math.pi * 5 * m / M)
    np.testing.assert_allclose(Dinv @ (D @ y), y, atol=1e-12)


def test_gelu_and_derivative():
    x = np.linspace(-4, 4, 81)
    h = 1e-6
    np.testing.assert_allclose(dgelu(x), (gelu(x + h) - gelu(x - h)) / (2 * h), rtol=1e-7, atol=1e-9)
    assert gelu(0.0) == 0.0 and gelu(10.0) == pytest.approx(10.0)


def test_backward_matches_finite_differences():
    no = NeuralOperator(M=8, C=6, K=3, L=3, H=5)
    rng = np.random.default_rng(7)
    theta = no.init_params(3) * 0.7
    cond = np.array([[0.02, 0.1, 2.0], [3.0, 0.4, 1.7]])
    target = rng.normal(size=(2, 8, 4))
    loss, grad = no.loss_and_grad(theta, cond, target)
    idx = rng.choice(no.size, size=60, replace=False)
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (no.loss_and_grad(tp, cond, target)[0] - no.loss_and_grad(tm, cond, target)[0]) / (2 * eps)
        assert grad[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i
