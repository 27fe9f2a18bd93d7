"""Pins of the oracle DFT against the definition, a library FFT and identities."""
import numpy as np
import pytest

from oracle import fft as offt


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 9, 12, 16, 18, 24, 27, 32, 48, 96])
def test_fast_matches_direct_1d(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    assert _rel(offt.fft(x), offt.dft_direct(x, -1)) < 1e-13
    assert _rel(offt.ifft(x), offt.dft_direct(x, +1) / n) < 1e-13


@pytest.mark.parametrize("n", [4, 6, 8, 12])
def test_rfft3_matches_direct_3d(n):
    rng = np.random.default_rng(100 + n)
    u = rng.standard_normal((n, n, n))
    ref = offt.dft_direct(offt.dft_direct(offt.dft_direct(u, -1, 0), -1, 1), -1, 2)
    assert _rel(offt.rfft3(u), ref[..., : n // 2 + 1]) < 1e-13


@pytest.mark.parametrize("n", [24, 32, 48])
def test_matches_library_fft(n):
    rng = np.random.default_rng(7 * n)
    u = rng.standard_normal((n, n, n))
    assert _rel(offt.rfft3(u), np.fft.rfftn(u)) < 1e-13
    U = np.fft.rfftn(u)
    assert _rel(offt.irfft3(U, n), u) < 1e-13


@pytest.mark.parametrize("n", [6, 16, 24])
def test_parseval_and_roundtrip(n):
    rng = np.random.default_rng(n + 3)
    u = rng.standard_normal((n, n, n))
    U = offt.fftn3(u)
    assert abs(np.sum(np.abs(U) ** 2) / n ** 3 - np.sum(u ** 2)) < 1e-11 * np.sum(u ** 2)
    assert _rel(offt.irfft3(offt.rfft3(u), n), u) < 1e-14


@pytest.mark.parametrize("n,m0", [(8, 3), (12, 5), (24, 7)])
def test_single_mode_is_delta(n, m0):
    j = np.arange(n)
    x = np.exp(2j * np.pi * m0 * j / n)
    X = offt.fft(x)
    ref = np.zeros(n, dtype=complex)
    ref[m0] = n
    assert np.max(np.abs(X - ref)) < 1e-12
