"""Pins for the oracle's sub-sample peak (parabolic vertex through the envelope maximum and
its two neighbours; a variant, the paper times stations to the sample)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("x0", [10.0, 10.3, 9.6, 10.499, 9.5001])
def test_vertex_of_a_sampled_parabola(x0):
    x = np.arange(21, dtype=np.float64)
    env = 7.0 - 0.8 * (x - x0) ** 2
    k = int(np.argmax(env))
    assert abs(k + oracle.peak_offset(env, k) - x0) <= 1e-12


def test_symmetric_flat_and_edges():
    env = np.array([0.0, 1.0, 3.0, 1.0, 0.0])
    assert oracle.peak_offset(env, 2) == 0.0
    flat = np.array([1.0, 2.0, 2.0, 2.0, 1.0])
    assert oracle.peak_offset(flat, 2) == 0.0                    # no strict maximum
    ramp = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    assert oracle.peak_offset(ramp, 4) == 0.0 and oracle.peak_offset(ramp[::-1].copy(), 0) == 0.0
    assert oracle.peak_offset(ramp, 2) == 0.0                    # second difference zero


def test_direction_and_clamp():
    env = np.array([0.0, 2.0, 3.0, 2.9, 0.0])                    # right neighbour larger: vertex right of 2
    d = oracle.peak_offset(env, 2)
    assert 0.0 < d < 0.5
    assert abs(d - 0.5 * (2.0 - 2.9) / (2.0 - 6.0 + 2.9)) <= 1e-15
    skew = np.array([0.0, 0.0, 3.0, 3.0 - 1e-9, 0.0])           # near tie: vertex close to 2.5
    assert 0.49 < oracle.peak_offset(skew, 2) <= 0.5


def test_fine_times_of_an_event_layout():
    env = np.zeros((2, 3, 16))
    x = np.arange(16.0)
    for d in range(2):
        for s in range(3):
            env[d, s] = 5.0 - (x - (4.0 + 2 * s + 0.25 * d)) ** 2
    idx = env.argmax(axis=2)
    t = oracle.fine_peak_times(env, idx, np.array([100.0, 200.0, 300.0]), 200e6)
    want = np.array([[[100.0, 200.0, 300.0][s] + 5.0 * (4.0 + 2 * s + 0.25 * d) for s in range(3)] for d in range(2)])
    assert np.allclose(t, want, rtol=0, atol=1e-9)
