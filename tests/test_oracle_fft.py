"""Pins of the oracle's own radix-2 FFT against brute-force DFTs and identities."""
import numpy as np
import pytest

import oracle



def dft_matrix(n, sign):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1_matches_bruteforce_dft(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = dft_matrix(n, sign) @ x
    np.testing.assert_allclose(oracle.fft1(x, sign), ref, atol=1e-12 * n, rtol=0)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_fft2_matches_bruteforce_dft(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    W = dft_matrix(n, -1)
    ref = W @ x @ W.T        # rows index y (slow), columns index x (fast)
    np.testing.assert_allclose(oracle.fft2(x, -1), ref, atol=1e-11 * n * n, rtol=0)


def test_fft2_roundtrip_and_parseval():
    n = 64
    rng = np.random.default_rng(7)
    x = rng.standard_normal((n, n))
    X = oracle.fft2(x, -1)
    np.testing.assert_allclose(oracle.fft2(X, +1).real / (n * n), x, atol=1e-13)
    assert abs(np.sum(np.abs(X) ** 2) / (n * n) - np.sum(x ** 2)) < 1e-9 * np.sum(x ** 2)


def test_fft2_of_cosine_is_two_spikes():
    n, mx, my = 32, 3, 5
    i = np.arange(n)
    X, Y = np.meshgrid(i, i, indexing="xy")
    f = np.cos(2 * np.pi * (mx * X + my * Y) / n)
    F = oracle.fft2(f.astype(complex), -1)
    ref = np.zeros((n, n), complex)
    ref[my, mx] = ref[(-my) % n, (-mx) % n] = n * n / 2
    np.testing.assert_allclose(F, ref, atol=1e-10)
