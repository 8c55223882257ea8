"""Pins of the oracle's F-step arithmetic against things other than itself.

The FFT convention (forward, e^{-2 pi i k n / N}, unnormalised) is the reading of
the paper's "FFT / cuFFT" (Sec. 2.5.1).  Checked against numpy.fft (a library
routine), closed forms of an impulse and of bin-centred tones, and the direct DFT.
"""
import numpy as np
import pytest

import oracle

POW2 = [1, 2, 4, 8, 16, 32, 64, 128, 256]
MIXED = [5, 10, 20, 40, 80, 160, 320, 640, 1280, 6400]


@pytest.mark.parametrize("n", POW2 + MIXED)
def test_fft_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    X = oracle.fft(x)
    ref = np.fft.fft(x)
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.sqrt(n) * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [1, 2, 3, 8, 10, 32, 40])
def test_dft_matches_numpy(n):
    rng = np.random.default_rng(100 + n)
    x = rng.integers(-128, 128, n) + 1j * rng.integers(-128, 128, n)
    assert np.allclose(oracle.dft(x), np.fft.fft(x), rtol=0, atol=1e-9)


@pytest.mark.parametrize("n", [8, 128, 1280])
def test_fft_impulse_closed_form(n):
    for n0 in (0, 1, n // 3, n - 1):
        x = np.zeros(n, complex)
        x[n0] = 1.0
        k = np.arange(n)
        expect = np.exp(-2j * np.pi * ((k * n0) % n) / n)
        assert np.max(np.abs(oracle.fft(x) - expect)) < 1e-11


@pytest.mark.parametrize("n", [16, 128, 640])
def test_fft_tone_lands_in_one_bin(n):
    # a e^{2 pi i u0 n / N} -> N a at bin u0 mod N, zero elsewhere (sign of the exponent)
    a = 3.0 - 2.0j
    for u0 in (1, 3, -2, n // 2 - 1):
        x = a * np.exp(2j * np.pi * u0 * np.arange(n) / n)
        X = oracle.fft(x)
        k0 = u0 % n
        assert abs(X[k0] - n * a) < 1e-9 * n
        X[k0] = 0
        assert np.max(np.abs(X)) < 1e-9 * n


@pytest.mark.parametrize("n", [32, 1280])
def test_fft_equals_direct_dft(n):
    rng = np.random.default_rng(7 * n)
    x = rng.integers(-127, 128, n) + 1j * rng.integers(-127, 128, n)
    X = oracle.fft(x)
    D = oracle.dft(x)
    assert np.max(np.abs(X - D)) <= 1e-10 * np.max(np.abs(D))
