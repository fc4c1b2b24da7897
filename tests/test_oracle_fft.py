"""Pins for the FFT oracle (Sec. 3.2.2 function block): closed forms,
Parseval, linearity, shift, round trip, DFT vs FFT and a library FFT."""
import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import synth


@pytest.mark.parametrize("fn", [oracle.dft, oracle.fft])
def test_delta_and_constant(fn):
    n = 64
    d = np.zeros(n, complex)
    d[0] = 1
    np.testing.assert_allclose(fn(d), np.ones(n), atol=1e-15)
    n0 = 5
    d = np.zeros(n, complex)
    d[n0] = 1
    k = np.arange(n)
    np.testing.assert_allclose(fn(d), np.exp(-2j * np.pi * k * n0 / n), atol=1e-14)
    np.testing.assert_allclose(fn(np.ones(n, complex)), n * (k == 0), atol=1e-12)


@pytest.mark.parametrize("fn", [oracle.dft, oracle.fft])
def test_single_tone(fn):
    n, m = 128, 17
    t = np.arange(n)
    X = fn(np.exp(2j * np.pi * m * t / n))
    expect = np.zeros(n, complex)
    expect[m] = n
    np.testing.assert_allclose(X, expect, atol=1e-11)


def test_parseval_linearity_shift_roundtrip():
    n = 1024
    x = synth.complex_normal(1, n)
    y = synth.complex_normal(2, n)
    X, Y = oracle.fft(x), oracle.fft(y)
    assert np.sum(abs(X) ** 2) == pytest.approx(n * np.sum(abs(x) ** 2), rel=1e-13)
    np.testing.assert_allclose(oracle.fft(2.5 * x - 1j * y), 2.5 * X - 1j * Y, atol=1e-11)
    s = 37
    k = np.arange(n)
    np.testing.assert_allclose(oracle.fft(np.roll(x, s)), X * np.exp(-2j * np.pi * k * s / n), atol=1e-11)
    back = oracle.fft(X, +1)
    assert np.linalg.norm(back - x) / np.linalg.norm(x) < 1e-15 * 20


@pytest.mark.parametrize("n", [2, 8, 256, 4096])
def test_fft_matches_dft(n):
    x = synth.complex_normal(n, n)
    a, b = oracle.fft(x), oracle.dft(x)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-14
    a, b = oracle.fft(x, +1), oracle.dft(x, +1)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-14


@pytest.mark.parametrize("logn", [10, 16, 20])
def test_fft_matches_library_fft(logn):
    n = 1 << logn
    x = synth.complex_normal(logn, n)
    a = oracle.fft(x)
    b = np.fft.fft(x)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-14


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12, complex))
