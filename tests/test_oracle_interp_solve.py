"""Pins for the oracle's VEL interpolation (Sec. 3) and 2x2 solve (CPU only).

Interpolation: exact at grid nodes, exact for multilinear fields inside a cell, equal to
scipy's RegularGridInterpolator (linear) on a periodically extended table, continuous
across the azimuth wrap, clamped at the zenith and frequency edges.
Solve: identity, diagonal and rotation systems in closed form, H E = V on random
non-symmetric systems, numpy.linalg.solve, and the near-singular rule.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth


def _pattern_from(table):
    g = synth.PATTERN_GRID
    return synth.Pattern(table.shape[0], math.radians(g["zen0_deg"]), math.radians(g["dzen_deg"]),
                         table.shape[1], math.radians(g["az0_deg"]), math.radians(g["daz_deg"]),
                         table.shape[2], g["f0_hz"], g["df_hz"], table.astype(np.complex64))


def _coords(pat, iz, ia, ifr):
    return (pat.zen0_rad + iz * pat.dzen_rad, pat.az0_rad + ia * pat.daz_rad, pat.f0_hz + ifr * pat.df_hz)


def test_exact_at_nodes():
    pat = synth.make_pattern()
    rng = np.random.default_rng(0)
    nodes = [(0, 0, 0), (18, 71, 50), (18, 0, 0), (0, 71, 50)] + [
        tuple(int(v) for v in (rng.integers(19), rng.integers(72), rng.integers(51))) for _ in range(30)]
    for iz, ia, ifr in nodes:
        z, a, f = _coords(pat, iz, ia, ifr)
        H, st = oracle.vel(pat, z, a, f)
        ref = pat.table[iz, ia, ifr].astype(np.complex128)
        assert np.max(abs(H - ref)) <= 1e-6 * np.max(abs(ref)), (iz, ia, ifr)
        assert st == 0


def test_multilinear_field_exact():
    # table[c][p] = a + b*iz + c*ia + d*if + e*iz*ia*if: trilinear interpolation reproduces it
    nz, na, nf = 19, 72, 51
    IZ, IA, IF = np.meshgrid(np.arange(nz), np.arange(na), np.arange(nf), indexing="ij")
    coef = np.array([[(1, 2, -1, 3, 0.25), (2, -1, 1, 1, -0.5)], [(-3, 1, 2, -2, 0.125), (5, 0, -1, 1, 1)]])
    t = np.zeros((nz, na, nf, 2, 2), complex)
    for c in range(2):
        for p in range(2):
            a, b, cc, d, e = coef[c, p]
            t[..., c, p] = (a + b * IZ + cc * IA + d * IF + e * IZ * IA * IF) * (1 + 0.5j)
    pat = _pattern_from(t)
    rng = np.random.default_rng(1)
    for _ in range(50):
        uz, ua, uf = rng.uniform(0, 17.999), rng.uniform(0, 70.999), rng.uniform(0, 49.999)
        z, a, f = (pat.zen0_rad + uz * pat.dzen_rad, pat.az0_rad + ua * pat.daz_rad, pat.f0_hz + uf * pat.df_hz)
        H, _ = oracle.vel(pat, z, a, f)
        for c in range(2):
            for p in range(2):
                a0, b, cc, d, e = coef[c, p]
                ref = (a0 + b * uz + cc * ua + d * uf + e * uz * ua * uf) * (1 + 0.5j)
                assert abs(H[c, p] - ref) <= 1e-9 * max(1.0, abs(ref))


def test_matches_scipy_regular_grid():
    from scipy.interpolate import RegularGridInterpolator
    pat = synth.make_pattern(seed_key=3)
    t = pat.table.astype(np.complex128)
    ext = np.concatenate([t, t[:, :1]], axis=1)          # azimuth node 72 == node 0
    zen = pat.zen0_rad + pat.dzen_rad * np.arange(pat.n_zen)
    az = pat.az0_rad + pat.daz_rad * np.arange(pat.n_az + 1)
    f = pat.f0_hz + pat.df_hz * np.arange(pat.n_freq)
    rgi = RegularGridInterpolator((zen, az, f), ext.reshape(pat.n_zen, pat.n_az + 1, pat.n_freq, 4))
    rng = np.random.default_rng(2)
    pts = np.stack([rng.uniform(0, math.radians(90), 200), rng.uniform(0, 2 * math.pi * 0.9999, 200),
                    rng.uniform(30e6, 80e6, 200)], axis=1)
    ref = rgi(pts)
    for q in range(200):
        H, _ = oracle.vel(pat, *pts[q])
        assert np.max(abs(H.reshape(4) - ref[q])) <= 1e-10 * np.max(abs(ref[q]))


def test_azimuth_periodic():
    pat = synth.make_pattern(seed_key=4)
    z, f = math.radians(37.3), 55.5e6
    for a in (0.0, 0.3, math.radians(357.5), math.radians(359.999)):
        H1, _ = oracle.vel(pat, z, a, f)
        H2, _ = oracle.vel(pat, z, a + 2 * math.pi, f)
        H3, _ = oracle.vel(pat, z, a - 4 * math.pi, f)
        assert np.max(abs(H1 - H2)) <= 1e-12 and np.max(abs(H1 - H3)) <= 1e-12
    # continuity across 360 deg -> 0 deg
    Ha, _ = oracle.vel(pat, z, 2 * math.pi - 1e-9, f)
    Hb, _ = oracle.vel(pat, z, 1e-9, f)
    H0, _ = oracle.vel(pat, z, 0.0, f)
    assert np.max(abs(Ha - H0)) <= 1e-6 and np.max(abs(Hb - H0)) <= 1e-6
    # halfway between node 71 (355 deg) and node 0 (360 deg) is their mean
    Hm, _ = oracle.vel(pat, z, math.radians(357.5), 30e6)
    iz = int(37.3 // 5)
    tz = (37.3 - 5 * iz) / 5
    ref = 0.5 * ((1 - tz) * pat.table[iz, 71, 0] + tz * pat.table[iz + 1, 71, 0]) + \
        0.5 * ((1 - tz) * pat.table[iz, 0, 0] + tz * pat.table[iz + 1, 0, 0])
    assert np.max(abs(Hm - ref)) <= 1e-6


def test_clamping():
    pat = synth.make_pattern(seed_key=5)
    H90, st90 = oracle.vel(pat, math.radians(90), 1.0, 40e6)
    Hbig, stbig = oracle.vel(pat, math.radians(97), 1.0, 40e6)
    assert np.max(abs(H90 - Hbig)) == 0 and st90 == 0 and stbig == oracle.ST_ZEN_CLAMP
    Hlo, _ = oracle.vel(pat, 0.5, 1.0, 30e6)
    Hlo2, _ = oracle.vel(pat, 0.5, 1.0, 20e6)
    Hhi, _ = oracle.vel(pat, 0.5, 1.0, 80e6)
    Hhi2, _ = oracle.vel(pat, 0.5, 1.0, 95e6)
    assert np.max(abs(Hlo - Hlo2)) == 0 and np.max(abs(Hhi - Hhi2)) == 0
    _, stneg = oracle.vel(pat, -0.1, 1.0, 40e6)
    assert stneg == oracle.ST_ZEN_CLAMP


# ---- solve --------------------------------------------------------------------------

def test_solve_identity_and_diagonal():
    V = np.array([1.5 - 2j, -0.25 + 3j])
    E, s, _ = oracle.solve(np.eye(2), V)
    assert s == 0 and np.max(abs(E - V)) <= 1e-15
    D = np.diag([2 + 1j, -0.5j])
    E, s, _ = oracle.solve(D, V)
    assert np.max(abs(E - V / np.diag(D))) <= 1e-15


def test_solve_rotation():
    a = 0.7
    R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    V = np.array([0.3 + 1j, 2 - 0.5j])
    E, s, _ = oracle.solve(R, V)
    assert np.max(abs(E - R.T @ V)) <= 1e-15


def test_solve_reproduces_V_and_numpy():
    rng = np.random.default_rng(9)
    for _ in range(200):
        H = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        V = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        E, s, _ = oracle.solve(H, V)
        assert s == 0
        assert np.max(abs(H @ E - V)) <= 1e-12 * np.max(abs(V)) * np.linalg.cond(H)
        assert np.max(abs(E - np.linalg.solve(H, V))) <= 1e-12 * np.linalg.cond(H) * np.max(abs(E))


def test_solve_singular_rule():
    V = np.array([1.0 + 0j, 2.0 + 0j])
    E, s, m = oracle.solve(np.array([[1, 2], [2, 4]], complex), V)  # rank one
    assert s == 1 and np.all(E == 0) and m == 0
    # det = eps; scale = |H0t||H1p| + |H0p||H1t| = 1 + 1 = 2 (up to eps)
    for eps, expect in ((1e-7, 1), (1.9e-6, 1), (2.1e-6, 0), (1e-3, 0)):
        H = np.array([[1.0, 1.0], [1.0, 1.0 + eps]], complex)
        E, s, m = oracle.solve(H, V)
        assert s == expect, eps
        if not s:
            assert np.max(abs(H @ E - V)) <= 1e-6


@pytest.mark.parametrize("scale", [1e-12, 1e12])
def test_solve_and_singular_rule_are_scale_invariant(scale):
    """H scaled by s gives E / s and the same singular decisions: the rule compares |det| with
    a product of two magnitudes, both quadratic in s. Powers of ten are not exact in binary,
    so E is compared to FP64 rounding."""
    rng = np.random.default_rng(12)
    V = rng.standard_normal(2) + 1j * rng.standard_normal(2)
    for _ in range(100):
        H = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        E, s, m = oracle.solve(H, V)
        Es, ss, ms = oracle.solve(H * scale, V)
        assert ss == s and abs(ms - m) <= 1e-12 * max(m, 1e-300)
        assert np.max(abs(Es * scale - E)) <= 1e-12 * np.linalg.cond(H) * np.max(abs(E))
    for eps, expect in ((1e-7, 1), (1.9e-6, 1), (2.1e-6, 0)):
        H = np.array([[1.0, 1.0], [1.0, 1.0 + eps]], complex) * scale
        assert oracle.solve(H, V)[1] == expect, (scale, eps)
