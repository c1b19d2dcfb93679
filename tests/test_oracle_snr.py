"""Oracle pins for the SNR variant (the paper defines no noise estimate and no timing weights;
the readings are: SNR = (env[k] / noise)^2 with noise^2 the mean of env^2 more than N/16
samples from the maximum k; the direction fit weights station s by w_s = SNR_s).

Each pin is a closed form worked out by hand, not the formula retyped.
"""
import numpy as np

import oracle


def test_flat_noise_and_a_peak():
    # noise level 2 everywhere outside the window, peak 14 at k: (14 / 2)^2 = 49
    e = np.full(256, 2.0)
    e[100] = 14.0
    assert oracle.snr(e, 100) == 49.0


def test_the_window_hides_the_pulse():
    # anything within 256/16 = 16 samples of the peak does not count as noise
    e = np.full(256, 2.0)
    e[84:117] = 9.0        # |n - 100| <= 16
    e[100] = 14.0
    assert oracle.snr(e, 100) == 49.0
    e[83] = 9.0            # 17 samples away: noise; mean of squares (222 * 4 + 81) / 223
    assert abs(oracle.snr(e, 100) - 196.0 / ((222 * 4 + 81) / 223)) <= 1e-12 * 49


def test_window_clipped_at_the_trace_ends():
    # N = 64, window 4: a peak at sample 0 leaves samples 5..63 (59 of them) as noise
    e = np.zeros(64)
    e[5:] = np.sqrt(3.0)   # env^2 = 3 there
    e[0] = 6.0
    assert abs(oracle.snr(e, 0) - 12.0) <= 1e-12
    f = e[::-1].copy()
    assert abs(oracle.snr(f, 63) - 12.0) <= 1e-12


def test_degenerate_cases():
    assert oracle.snr(np.zeros(128), 40) == 0.0          # no noise power
    assert oracle.snr(np.array([5.0]), 0) == 0.0         # no sample outside the window
    e = np.full(128, 0.5)
    e[64] = 4.0
    assert abs(oracle.snr(3.0 * e, 64) - oracle.snr(e, 64)) <= 1e-12 * 64   # scale free


def test_weighted_fit_by_hand():
    # zenith 0, stations at z = 0: tau = 0, so d = t. w = (1, 3), d = (0, 4):
    # t0 = 12 / 4 = 3, r = (-3, 1), chi2 = 1 * 9 + 3 * 1 = 12
    r, t0, chi2 = oracle.residual_weighted(np.zeros((2, 3)), np.array([0.0, 4.0]), np.array([1.0, 3.0]), 0.0, 0.0)
    assert t0 == 3.0 and chi2 == 12.0
    assert np.array_equal(r, [-3.0, 1.0])


def test_weighted_fit_special_cases():
    rng = np.random.default_rng(5)
    pos = rng.normal(0, 300, (9, 3))
    t = rng.normal(0, 50, 9)
    zen, az = 0.4, 1.1
    r0, t00, c0 = oracle.residual(pos, t, zen, az)
    # equal weights: the unweighted fit, chi2 scaled by the weight
    r, t0, c = oracle.residual_weighted(pos, t, np.full(9, 2.5), zen, az)
    assert np.allclose(r, r0, rtol=0, atol=1e-12) and abs(t0 - t00) <= 1e-12 and abs(c - 2.5 * c0) <= 1e-9 * c0
    # all weights zero: the unweighted fit exactly
    r, t0, c = oracle.residual_weighted(pos, t, np.zeros(9), zen, az)
    assert np.array_equal(r, r0) and t0 == t00 and c == c0
    # one station carries all the weight: it defines t0 and contributes nothing to chi2
    w = np.zeros(9)
    w[4] = 7.0
    r, t0, c = oracle.residual_weighted(pos, t, w, zen, az)
    assert abs(r[4]) <= 1e-12 and c <= 1e-20


def test_plane_wave_gives_zero_residual_for_any_weights():
    # arrival times of a plane wave from (zen, az): t_s = t0 - n.x_s / c with n toward the source
    rng = np.random.default_rng(6)
    pos = rng.normal(0, 500, (12, 3))
    zen, az, t0_true = 0.7, 2.3, 123.0
    n = np.array([np.sin(zen) * np.cos(az), np.sin(zen) * np.sin(az), np.cos(zen)])
    t = t0_true - pos @ n / 0.299792458
    r, t0, c = oracle.residual_weighted(pos, t, rng.uniform(0.1, 50, 12), zen, az)
    assert np.all(abs(r) <= 1e-9) and abs(t0 - t0_true) <= 1e-9 and c <= 1e-15
