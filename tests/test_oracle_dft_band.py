"""Pins for the oracle's naive DFT and band mask (CPU only).

The DFT is checked against Parseval's theorem, inverse-after-forward identity, closed
forms for a cosine and a delta, and numpy's FFT; the band mask against the 30-80 MHz band
of the paper (Sec. 1) with the bin edges worked out by hand.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(__file__)


@pytest.mark.parametrize("n", [16, 64, 256])
def test_parseval(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = oracle.dft(x, -1)
    assert abs(np.sum(abs(x) ** 2) - np.sum(abs(X) ** 2) / n) <= 1e-12 * np.sum(abs(x) ** 2)


@pytest.mark.parametrize("n", [16, 100, 256])
def test_inverse_after_forward(n):
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = oracle.dft(oracle.dft(x, -1), +1) / n
    assert np.max(abs(y - x)) <= 1e-12 * np.max(abs(x))


def test_cosine_closed_form():
    n, k0 = 128, 19
    x = np.cos(2 * np.pi * k0 * np.arange(n) / n)
    X = oracle.dft(x, -1)
    ref = np.zeros(n, complex)
    ref[k0] = ref[n - k0] = n / 2
    assert np.max(abs(X - ref)) <= 1e-10


def test_delta_closed_form():
    n, n0 = 64, 11
    x = np.zeros(n)
    x[n0] = 1.0
    X = oracle.dft(x, -1)
    k = np.arange(n)
    ref = np.cos(2 * np.pi * k * n0 / n) - 1j * np.sin(2 * np.pi * k * n0 / n)
    assert np.max(abs(X - ref)) <= 1e-12


def test_matches_numpy_fft():
    n = 240
    rng = np.random.default_rng(7)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.max(abs(oracle.dft(x, -1) - np.fft.fft(x))) <= 1e-10 * np.max(abs(np.fft.fft(x)))
    assert np.max(abs(oracle.dft(x, +1) / n - np.fft.ifft(x))) <= 1e-12 * n


def test_station_spectrum_channels_separate():
    rng = np.random.default_rng(3)
    tr = rng.standard_normal((2, 128)).astype(np.float32)
    sp = oracle.station_spectrum(tr)
    for c in range(2):
        ref = np.fft.fft(tr[c].astype(np.float64))
        assert np.max(abs(sp[c] - ref)) <= 1e-11 * np.max(abs(ref))


def _band(n, fs=200e6):
    return [k for k in range(n) if oracle.in_band(n, fs, k)]


@pytest.mark.parametrize("n,lo,hi", [(1024, 154, 409), (2048, 308, 819), (4096, 615, 1638), (16, 3, 6), (64, 10, 25)])
def test_band_edges(n, lo, hi):
    # 30 MHz / (200 MHz / N) = 0.15 N and 80 MHz / (200 MHz / N) = 0.4 N: first bin is
    # ceil(0.15 N), last is floor(0.4 N); for these N that is exactly N/4 bins.
    b = _band(n)
    assert b[0] == lo and b[-1] == hi and len(b) == hi - lo + 1 == n // 4
    assert b == list(range(lo, hi + 1))


def test_band_edges_inclusive():
    # fs = 160 MHz, N = 16: bins are 10 MHz apart, so 30 and 80 MHz fall exactly on bins 3 and 8
    assert _band(16, 160e6) == [3, 4, 5, 6, 7, 8]


def test_band_is_the_papers():
    facts = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))
    lo, hi = facts["band_hz"]["value"]
    n, fs = 1000, 1000e6   # 1 MHz bins
    b = _band(n, fs)
    assert b[0] == int(lo / 1e6) and b[-1] == int(hi / 1e6)
