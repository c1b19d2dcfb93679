"""Pins for the oracle's full per-pair chain and the timing residual (CPU only).

- an in-band cosine through an identity antenna comes back unchanged with a constant
  envelope (Sec. 4's envelope of a pure tone is its amplitude);
- a band-limited random signal: envelope equals |scipy.signal.hilbert(x)|;
- a delta through a flat complex antenna: E-field and envelope equal the closed-form
  Dirichlet-kernel sums, and the envelope peaks at the delta;
- a band-limited field pushed through a real mixing matrix, and through a pattern linear
  in frequency, is recovered;
- small-N brute force with numpy's FFT and scipy's grid interpolator on the synthetic
  pattern;
- residuals: hand-computed plane-wave geometry gives zero; offsets give offset - mean.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth

FS = 200e6


def _band_bins(n, fs=FS):
    k = np.arange(n)
    f = k * fs / n
    return k[(f >= 30e6) & (f <= 80e6)]


def _flat(M):
    return synth.make_flat_pattern(np.asarray(M, complex))


def test_cosine_identity_antenna():
    n, k0, ph, A = 256, 80, 0.9, 3.0   # bin 80 of 256 at 200 MHz = 62.5 MHz, in band
    x = (A * np.cos(2 * np.pi * k0 * np.arange(n) / n + ph)).astype(np.float32)
    tr = np.stack([x, np.zeros(n, np.float32)])
    o = oracle.unfold_pair(_flat(np.eye(2)), tr, 0.3, 0.4, FS)
    assert np.max(abs(o["efield"][0] - x)) <= 1e-5 * A
    assert np.max(abs(o["efield"][1])) <= 1e-5 * A
    assert np.max(abs(o["env"] - A)) <= 1e-5 * A
    assert o["status"] == 0


def test_envelope_is_scipy_hilbert():
    from scipy.signal import hilbert
    n = 512
    rng = np.random.default_rng(11)
    kb = _band_bins(n)
    X = np.zeros(n // 2 + 1, complex)
    X[kb] = rng.standard_normal(kb.size) + 1j * rng.standard_normal(kb.size)
    x = np.fft.irfft(X, n)
    x32 = x.astype(np.float32)
    y = (0.5 * x + 0.25 * np.roll(x, 7)).astype(np.float32)
    tr = np.stack([x32, y])
    o = oracle.unfold_pair(_flat(np.eye(2)), tr, 0.2, 1.0, FS)
    env_ref = np.sqrt(abs(hilbert(x32.astype(np.float64))) ** 2 + abs(hilbert(y.astype(np.float64))) ** 2)
    assert np.max(abs(o["env"] - env_ref)) <= 1e-5 * np.max(env_ref)
    assert np.max(abs(o["efield"][0] - x32)) <= 1e-5 * np.max(abs(x32))


def _dirichlet(theta, a, b):
    """sum_{k=a}^{b} exp(i k theta) in closed form (theta not a multiple of 2 pi)."""
    m = b - a + 1
    out = np.empty(theta.shape, complex)
    small = np.isclose(np.sin(theta / 2), 0.0, atol=1e-15)
    th = theta[~small]
    out[~small] = np.exp(1j * th * (a + b) / 2) * np.sin(m * th / 2) / np.sin(th / 2)
    out[small] = m * np.exp(1j * theta[small] * (a + b) / 2)
    return out


@pytest.mark.parametrize("n,n0", [(256, 77), (1024, 500)])
def test_delta_flat_antenna_closed_form(n, n0):
    # the table stores complex64: take M at that precision so the closed form sees the same M
    M = np.array([[1.2 + 0.3j, -0.4 + 0.1j], [0.2 - 0.5j, 0.9 + 0.2j]]).astype(np.complex64).astype(complex)
    Minv = np.linalg.inv(M)
    tr = np.zeros((2, n), np.float32)
    tr[0, n0] = 1.0
    o = oracle.unfold_pair(_flat(M), tr, 0.5, 2.0, FS)
    kb = _band_bins(n)
    D = _dirichlet(2 * np.pi * (np.arange(n) - n0) / n, kb[0], kb[-1])   # sum over band of e^{2 pi i k (m - n0)/N}
    z = [(2.0 / n) * Minv[p, 0] * D for p in range(2)]
    for p in range(2):
        assert np.max(abs(o["efield"][p] - z[p].real)) <= 1e-12
    env = np.sqrt(abs(z[0]) ** 2 + abs(z[1]) ** 2)
    assert np.max(abs(o["env"] - env)) <= 1e-12
    assert o["peak_idx"] == n0
    assert abs(o["peak_amp"] - (2.0 / n) * kb.size * math.hypot(abs(Minv[0, 0]), abs(Minv[1, 0]))) <= 1e-12


def test_field_recovered_through_real_mixing():
    n = 512
    rng = np.random.default_rng(12)
    kb = _band_bins(n)
    e0 = []
    for p in range(2):
        X = np.zeros(n // 2 + 1, complex)
        X[kb] = rng.standard_normal(kb.size) + 1j * rng.standard_normal(kb.size)
        e0.append(np.fft.irfft(X, n))
    M = np.array([[0.8, -0.6], [0.3, 1.1]]).astype(np.float32).astype(np.float64)
    v = (M @ np.stack(e0)).astype(np.float32)
    o = oracle.unfold_pair(_flat(M), v, 0.4, 0.1, FS)
    for p in range(2):
        # v was rounded to float32: recovery is to float32 rounding, amplified by cond(M)
        assert np.max(abs(o["efield"][p] - e0[p])) <= 1e-5 * np.max(abs(e0[p]))


def test_pattern_linear_in_frequency_recovered():
    # H(f) = M0 + (f - 30 MHz)/1 MHz * M1 at every node: interpolation is exact, so a field
    # pushed through H bin by bin must come back out.
    n = 1024
    M0 = np.array([[1.0 + 0.2j, 0.3], [-0.2j, 0.9]])
    M1 = np.array([[0.01j, -0.005], [0.004, 0.008 - 0.003j]])
    g = synth.PATTERN_GRID
    fidx = np.arange(g["n_freq"])
    table = np.broadcast_to((M0[None] + fidx[:, None, None] * M1[None])[None, None],
                            (g["n_zen"], g["n_az"], g["n_freq"], 2, 2))
    pat = synth.make_flat_pattern(np.eye(2))
    pat.table = np.ascontiguousarray(table.astype(np.complex64))
    Ht = pat.table.astype(np.complex128)[0, 0]          # exact float32 node values
    rng = np.random.default_rng(13)
    kb = _band_bins(n)
    E = np.zeros((2, n // 2 + 1), complex)
    E[:, kb] = rng.standard_normal((2, kb.size)) + 1j * rng.standard_normal((2, kb.size))
    V = np.zeros_like(E)
    for k in kb:
        u = (k * FS / n - 30e6) / 1e6
        i = min(int(math.floor(u)), g["n_freq"] - 2)
        t = u - i
        H = (1 - t) * Ht[i] + t * Ht[i + 1]
        V[:, k] = H @ E[:, k]
    v = np.fft.irfft(V, n).astype(np.float32)
    e0 = np.fft.irfft(E, n)
    o = oracle.unfold_pair(pat, v, 0.1, 0.2, FS)
    for p in range(2):
        assert np.max(abs(o["efield"][p] - e0[p])) <= 2e-5 * np.max(abs(e0[p]))


@pytest.mark.parametrize("n", [16, 64, 128])
def test_brute_force_small_n_against_numpy_scipy(n):
    from scipy.interpolate import RegularGridInterpolator
    pat = synth.make_pattern(seed_key=6)
    rng = np.random.default_rng(n)
    tr = rng.standard_normal((2, n)).astype(np.float32)
    zen, az = math.radians(41.0), math.radians(212.0)
    o = oracle.unfold_pair(pat, tr, zen, az, FS)
    t = pat.table.astype(np.complex128)
    ext = np.concatenate([t, t[:, :1]], axis=1)
    grid = (pat.zen0_rad + pat.dzen_rad * np.arange(pat.n_zen),
            pat.az0_rad + pat.daz_rad * np.arange(pat.n_az + 1),
            pat.f0_hz + pat.df_hz * np.arange(pat.n_freq))
    rgi = RegularGridInterpolator(grid, ext.reshape(pat.n_zen, pat.n_az + 1, pat.n_freq, 4))
    V = np.fft.fft(tr.astype(np.float64), axis=1)
    Z = np.zeros((2, n), complex)
    for k in _band_bins(n):
        H = rgi([[zen, az, k * FS / n]])[0].reshape(2, 2)
        Z[:, k] = 2 * np.linalg.solve(H, V[:, k])
    z = np.fft.ifft(Z, axis=1)
    env = np.sqrt(np.sum(abs(z) ** 2, axis=0))
    assert np.max(abs(o["efield"] - z.real)) <= 1e-10 * np.max(abs(z.real))
    assert np.max(abs(o["env"] - env)) <= 1e-10 * np.max(env)
    assert o["peak_idx"] == int(np.argmax(env))


def test_peak_ties_lowest_index():
    # identical pulses at two positions -> identical envelope maxima; lowest index wins
    n = 64
    tr = np.zeros((2, n), np.float32)
    o0 = oracle.unfold_pair(_flat(np.eye(2)), tr, 0.1, 0.1, FS)
    assert o0["peak_idx"] == 0 and o0["peak_amp"] == 0.0       # all-zero envelope: index 0
    k0 = 20                                                  # 62.5 MHz at N = 64
    tr[0] = np.cos(2 * np.pi * k0 * np.arange(n) / n).astype(np.float32)
    o = oracle.unfold_pair(_flat(np.eye(2)), tr, 0.1, 0.1, FS)
    best = np.flatnonzero(o["env"] == o["env"].max())
    assert o["peak_idx"] == best[0]


def test_bad_direction():
    n = 64
    tr = np.ones((2, n), np.float32)
    o = oracle.unfold_pair(synth.make_pattern(), tr, float("nan"), 0.1, FS)
    assert o["status"] & oracle.ST_BAD_DIR and np.all(o["efield"] == 0) and o["peak_idx"] == 0


def test_unreducible_azimuth_is_a_bad_direction():
    """An azimuth 2^52 or more azimuth steps from az0 (one FP64 unit is then a whole step)
    has no cell: it is flagged like a non-finite one. 1000 turns plus 0.3 rad still reduce,
    to the direction at 0.3 rad (the azimuth axis is periodic)."""
    rng = np.random.default_rng(5)
    n = 256
    tr = rng.standard_normal((2, n)).astype(np.float32)
    pat = synth.make_pattern()
    daz = pat.daz_rad
    for az in (1e300, -1.7e308, 2.0 ** 54 * daz, -(2.0 ** 54) * daz):
        o = oracle.unfold_pair(pat, tr, 0.3, az, FS)
        assert o["status"] & oracle.ST_BAD_DIR and np.all(o["efield"] == 0) and np.all(o["env"] == 0)
    o = oracle.unfold_pair(pat, tr, 0.3, 2000 * math.pi + 0.3, FS)   # 72000 azimuth steps
    assert not o["status"] & oracle.ST_BAD_DIR
    ref = oracle.unfold_pair(pat, tr, 0.3, 0.3, FS)
    assert np.allclose(o["efield"], ref["efield"], rtol=1e-9, atol=1e-9 * np.abs(ref["efield"]).max())


# ---- residual ----------------------------------------------------------------------

C = 0.299792458  # m/ns


def test_residual_hand_geometry():
    pos = np.array([[0.0, 0.0, 0.0], [300.0, 0.0, 0.0], [0.0, 300.0, 0.0], [0.0, 0.0, 10.0]])
    # horizon source toward +x (zenith 90, azimuth 0): the +x station sees it 300 m / c earlier;
    # the others (on the y and z axes) at the same time as the origin
    t = np.array([5.0, 5.0 - 300.0 / C, 5.0, 5.0])
    r, t0, chi2 = oracle.residual(pos, t, math.pi / 2, 0.0)
    assert np.max(abs(r)) <= 1e-9 and chi2 <= 1e-18 and abs(t0 - 5.0) <= 1e-9
    # azimuth 90 deg is +y (counter-clockwise from east)
    t = np.array([5.0, 5.0, 5.0 - 300.0 / C, 5.0])
    r, _, _ = oracle.residual(pos, t, math.pi / 2, math.pi / 2)
    assert np.max(abs(r)) <= 1e-9
    # vertical source: the station 10 m up is hit 10 m / c earlier
    t = np.array([0.0, 0.0, 0.0, -10.0 / C])
    r, _, _ = oracle.residual(pos, t, 0.0, 1.234)
    assert np.max(abs(r)) <= 1e-9
    # refractive index n: delays scale by n
    t = np.array([0.0, -1.0003 * 300.0 / C, 0.0, 0.0])
    r, _, _ = oracle.residual(pos, t, math.pi / 2, 0.0, n_refr=1.0003)
    assert np.max(abs(r)) <= 1e-9


def test_residual_offsets():
    pos = synth.make_stations(40)
    zen, az = math.radians(33.0), math.radians(120.0)
    nvec = np.array([math.sin(zen) * math.cos(az), math.sin(zen) * math.sin(az), math.cos(zen)])
    base = -(pos @ nvec) / C + 1234.5
    delta = np.random.default_rng(1).normal(0, 7.0, 40)
    r, t0, chi2 = oracle.residual(pos, base + delta, zen, az)
    ref = delta - delta.mean()
    assert np.max(abs(r - ref)) <= 1e-9
    assert abs(chi2 - np.sum(ref ** 2)) <= 1e-9 * np.sum(ref ** 2)
    assert abs(t0 - (1234.5 + delta.mean())) <= 1e-9
