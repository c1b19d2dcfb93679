"""Shared comparison rules for GPU-vs-oracle parity tests.

Tolerances (stated once, used everywhere):
- E-field and envelope: relative L2 error per (station, direction) pair <= 1e-5;
- peak index: equal, or a neighbour of the oracle's index (|diff| == 1) whose oracle
  envelope lies within 1e-6 relative of the oracle's maximum (two samples that tie at FP32
  resolution);
- peak amplitude: relative error <= 1e-5;
- peak time, residual, t0: |diff| <= 1e-9 * max(|oracle|, 1 ns); chi2: relative 1e-9 with
  a 1 ns^2 floor. Where a peak index legitimately differs, the residual of that direction
  is compared with the oracle's residual recomputed from the GPU's peak times.
- status bits: equal, except pairs whose smallest |det|/scale lies within 10x of the
  near-singular threshold (1e-6).
"""
import numpy as np

import oracle

REL_L2 = 1e-5
TIE = 1e-6
TIME_REL = 1e-9


def rel_l2(a, b, axis_len):
    a = np.asarray(a, np.float64).reshape(-1, axis_len)
    b = np.asarray(b, np.float64).reshape(-1, axis_len)
    nb = np.linalg.norm(b, axis=1)
    return np.linalg.norm(a - b, axis=1) / np.where(nb > 0, nb, 1.0)


def is_tie(env, gi, oi):
    """A peak index other than the oracle's is accepted only as its neighbour, with the oracle's
    envelope at the two samples equal within TIE relative to the maximum."""
    env = np.asarray(env, np.float64)
    top = env[oi]
    return abs(int(gi) - int(oi)) == 1 and abs(env[gi] - top) <= TIE * top


def near_threshold(ref):
    return np.asarray(ref["min_margin"]) <= 1e-5


def check_pairs(gpu, ref, n_samples, efield=True):
    """Compare per-pair outputs (arrays shaped [..pairs..] / [..pairs.., N])."""
    skip = near_threshold(ref).reshape(-1)
    if efield:
        e = rel_l2(gpu["efield"], ref["efield"], 2 * n_samples)[~skip]
        v = rel_l2(gpu["envelope"], ref["envelope"], n_samples)[~skip]
        assert e.size == 0 or e.max() <= REL_L2, f"E-field rel L2 max {e.max():.3g} median {np.median(e):.3g}"
        assert v.size == 0 or v.max() <= REL_L2, f"envelope rel L2 max {v.max():.3g}"
    gi = np.asarray(gpu["peak_idx"]).reshape(-1)
    oi = np.asarray(ref["peak_idx"]).reshape(-1)
    env = np.asarray(ref["envelope"]).reshape(gi.size, n_samples) if ref.get("envelope") is not None else None
    diff = np.flatnonzero(gi != oi)
    for q in diff:
        assert env is not None, f"peak index differs at pair {q} and no envelope to judge a tie"
        assert is_tie(env[q], gi[q], oi[q]), f"pair {q}: gpu idx {gi[q]} vs oracle {oi[q]} is not an adjacent tie"
    pa = np.asarray(gpu["peak_amp"], np.float64).reshape(-1)
    ra = np.asarray(ref["peak_amp"]).reshape(-1)
    assert np.all(abs(pa - ra) <= REL_L2 * np.maximum(ra, 1e-30) + 1e-30), "peak amplitude"
    gs = np.asarray(gpu["status"]).reshape(-1).astype(np.uint32)
    rs = np.asarray(ref["status"]).reshape(-1).astype(np.uint32)
    assert np.array_equal(gs[~skip], rs[~skip]), "status bits"
    return diff


def check_times(gpu_t, ref_t, what):
    g = np.asarray(gpu_t, np.float64)
    r = np.asarray(ref_t, np.float64)
    both_nan = np.isnan(g) & np.isnan(r)
    tol = TIME_REL * np.maximum(abs(np.nan_to_num(r)), 1.0)
    bad = ~both_nan & ~(abs(g - r) <= tol)
    assert not bad.any(), f"{what}: max |diff| {np.nanmax(abs(g - r)):.3g}"


def check_event(gpu, ref, ev, efield=True):
    """Full-event comparison: per-pair outputs, peak times, residuals, t0, chi2."""
    D, S = ev.n_dirs, ev.n_stations
    diff = check_pairs(gpu, ref, ev.n_samples, efield)
    gi = np.asarray(gpu["peak_idx"]).reshape(D, S)
    dt = 1e9 / ev.fs_hz
    # peak time follows from the index the GPU chose
    check_times(gpu["peak_time_ns"], ev.t_start_ns[None, :] + gi * dt, "peak time")
    if diff.size == 0:
        check_times(gpu["residual_ns"], ref["residual_ns"], "residual")
        check_times(gpu["t0_ns"], ref["t0_ns"], "t0")
        chi_ref = ref["chi2"]
    else:
        res = np.empty((D, S))
        t0 = np.empty(D)
        chi_ref = np.empty(D)
        for d in range(D):
            res[d], t0[d], chi_ref[d] = oracle.residual(ev.pos_m, np.asarray(gpu["peak_time_ns"])[d],
                                                        *ev.dirs_rad[d])
        check_times(gpu["residual_ns"], res, "residual (recomputed at GPU peaks)")
        check_times(gpu["t0_ns"], t0, "t0 (recomputed)")
    g = np.asarray(gpu["chi2"], np.float64)
    ok = (np.isnan(g) & np.isnan(chi_ref)) | (abs(g - chi_ref) <= TIME_REL * np.maximum(abs(np.nan_to_num(chi_ref)), 1.0))
    assert np.all(ok), "chi2"
