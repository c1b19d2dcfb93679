"""Pins for the oracle's iterative reconstruction (Sec. 2): voltage-maximum timing, the
least-squares plane-wave fit, and the loop."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth

C = 0.299792458


def _times(pos, zen, az, t0, n_refr=1.0):
    n = np.array([math.sin(zen) * math.cos(az), math.sin(zen) * math.sin(az), math.cos(zen)])
    return t0 - (pos @ n) * n_refr / C


@pytest.mark.parametrize("zen,az", [(0.0, 0.0), (0.3, 1.0), (1.0, 4.0), (1.3, 6.2), (0.05, 3.14159)])
def test_fit_recovers_exact_plane_wave(zen, az):
    pos = synth.make_stations(60, seed_key=3)            # heights ~ N(0, 2 m)
    z, a, t0 = oracle.plane_fit(pos, _times(pos, zen, az, 321.0))
    d = math.acos(min(1.0, math.sin(z) * math.sin(zen) * math.cos(a - az) + math.cos(z) * math.cos(zen)))
    assert d <= 1e-9 and abs(t0 - 321.0) <= 1e-6


def test_fit_equals_lstsq_for_a_flat_array():
    rng = np.random.default_rng(4)
    pos = synth.make_stations(40, seed_key=4)
    pos[:, 2] = 0.0
    t = _times(pos, 0.6, 2.0, 10.0) + rng.normal(0, 3.0, 40)
    z, a, t0 = oracle.plane_fit(pos, t)
    A = np.stack([np.ones(40), -pos[:, 0] / C, -pos[:, 1] / C], axis=1)
    sol = np.linalg.lstsq(A, t, rcond=None)[0]
    nx, ny = sol[1], sol[2]
    assert abs(t0 - sol[0]) <= 1e-6
    assert abs(math.sin(z) * math.cos(a) - nx) <= 1e-9 and abs(math.sin(z) * math.sin(a) - ny) <= 1e-9


def test_fit_refuses_degenerate_geometry():
    pos = np.array([[0.0, 0, 0], [100.0, 0, 0], [200.0, 0, 0], [300.0, 0, 0]])   # collinear
    assert oracle.plane_fit(pos, np.zeros(4)) is None
    assert oracle.plane_fit(pos[:2], np.zeros(2)) is None


def test_voltage_peaks_brute_force():
    ev = synth.make_event(7, 1024, synth.scan_directions(1, 1), seed_key=60)
    idx, t = oracle.voltage_peaks(ev)
    p = ev.traces[:, 0].astype(np.float64) ** 2 + ev.traces[:, 1].astype(np.float64) ** 2
    assert np.array_equal(idx, np.argmax(p, axis=1))
    assert np.allclose(t, ev.t_start_ns + idx * 5.0, rtol=0, atol=1e-9)


def test_loop_converges_near_the_true_direction():
    pat = synth.make_pattern()
    ev = synth.make_event(40, 2048, synth.scan_directions(1, 1), seed_key=61)
    r = oracle.reconstruct(pat, ev, max_iter=8)
    assert 1 <= r["iterations"] <= 8
    zt, at = ev.true_dir
    d = math.acos(min(1.0, math.sin(r["zenith"]) * math.sin(zt) * math.cos(r["azimuth"] - at) +
                      math.cos(r["zenith"]) * math.cos(zt)))
    assert d < math.radians(2.0), math.degrees(d)
    # the last fit is a fixed point: its station times reproduce the same direction
    z2, a2, _ = oracle.plane_fit(ev.pos_m, r["peak_time_ns"])
    assert abs(z2 - r["zenith"]) <= 1e-12 or r["iterations"] == 8
