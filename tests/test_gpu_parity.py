"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Cases: every supported trace length with ragged station/direction counts, the plain
single event (10 stations x 2048 samples, 1 direction), the same at 4096 samples, and
the 124-station x 64-direction scan at full size in the launch configuration the
benchmark times (every pair against the oracle, plus properties checked for all pairs). Edge cases: one pair, non-finite and out-of-table directions, a singular antenna,
peaks-only mode, host-buffer entry point, determinism, argument validation.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_event, check_pairs, check_times, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1507_07733_gb300 import binding
    c = binding.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pat():
    return synth.make_pattern()


@pytest.fixture(scope="module")
def pid(ctx, pat):
    return ctx.load_pattern(pat)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_gpu(ctx, pid, ev, traces_out=True, n_refr=1.0):
    out = ctx.unfold(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad),
                     fs_hz=ev.fs_hz, refractive_index=n_refr, traces_out=traces_out, sync=True)
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


@pytest.mark.parametrize("n,s,d", [(1024, 5, 3), (2048, 7, 5), (4096, 3, 2), (2048, 1, 1), (1024, 13, 9)])
def test_parity_full_event(ctx, pat, pid, n, s, d):
    rng = np.random.default_rng(n + 10 * s + d)
    ev = synth.make_event(s, n, synth.random_directions(d, rng), seed_key=n + s)
    gpu = run_gpu(ctx, pid, ev)
    ref = oracle.unfold_event(pat, ev)
    check_event(gpu, ref, ev)


def test_parity_plain_single_event(ctx, pat, pid):
    ev = synth.single_event(2048)
    gpu = run_gpu(ctx, pid, ev)
    ref = oracle.unfold_event(pat, ev)
    check_event(gpu, ref, ev)


def test_parity_single_event_4096(ctx, pat, pid):
    ev = synth.single_event(4096)
    gpu = run_gpu(ctx, pid, ev)
    ref = oracle.unfold_event(pat, ev)
    check_event(gpu, ref, ev)


def test_parity_direction_scan_full_size(ctx, pat, pid):
    """Every one of the scan's 7,936 pairs against the oracle (about 16 s of oracle time on 16
    host cores), in the launch configuration the benchmark times."""
    ev = synth.direction_scan()
    gpu = run_gpu(ctx, pid, ev)
    D = ev.n_dirs
    ref = oracle.unfold_event(pat, ev)
    check_event(gpu, ref, ev)
    # properties that hold for every pair
    env = gpu["envelope"]
    amp = gpu["peak_amp"]
    idx = gpu["peak_idx"]
    assert np.all(np.take_along_axis(env, idx[..., None].astype(np.int64), axis=2)[..., 0] == amp)
    assert np.all(env.max(axis=2) == amp)
    first = np.argmax(env == amp[..., None], axis=2)
    assert np.array_equal(first, idx)
    assert np.all(gpu["status"] == 0)
    # residuals, t0 and chi2 of every direction from the GPU's own peak times
    for d in range(D):
        r, t0, chi2 = oracle.residual(ev.pos_m, gpu["peak_time_ns"][d], *ev.dirs_rad[d])
        check_times(gpu["residual_ns"][d], r, "residual")
        check_times(gpu["t0_ns"][d], t0, "t0")
        assert abs(gpu["chi2"][d] - chi2) <= 1e-9 * max(chi2, 1.0)


# Sampling rates whose band window starts at every kind of k_lo modulo the pass-2 size P (16
# at 1024 and 2048 samples, 32 at 4096): the band rows past k_lo mod P are the ones the
# inverse transform treats separately (at 2048 samples a one-slot input shift in pass 1).
# k_lo mod P: 2048 -> 240 MHz 0, 213 MHz 1, 204.8 MHz 12, 227 MHz 15; 1024 -> 240 MHz 0,
# 213 MHz 1, 227 MHz 8; 4096 -> 240 MHz 0, 233 MHz 16, 227 MHz 30.
@pytest.mark.parametrize("n,fs_mhz", [(2048, 240.0), (2048, 213.0), (2048, 204.8), (2048, 227.0),
                                      (1024, 240.0), (1024, 213.0), (1024, 227.0),
                                      (4096, 240.0), (4096, 233.0), (4096, 227.0)])
def test_parity_band_offsets(ctx, pat, pid, n, fs_mhz):
    rng = np.random.default_rng(int(fs_mhz * 10) + n)
    ev = synth.make_event(6, n, synth.random_directions(4, rng), seed_key=40 + n // 1024, fs_hz=fs_mhz * 1e6)
    gpu = run_gpu(ctx, pid, ev)
    ref = oracle.unfold_event(pat, ev)
    check_event(gpu, ref, ev)


def test_edge_directions(ctx, pat, pid):
    dirs = np.array([[math.radians(30), math.radians(45)], [float("nan"), 0.1], [0.2, float("inf")],
                     [math.radians(97.0), 1.0], [-0.05, 2.0], [math.radians(20), -7.5],
                     [math.radians(59.9), 4 * math.pi + 0.3], [math.radians(90), math.radians(355)],
                     [0.3, 1e300], [0.4, -1.7e308]])   # azimuths too large to reduce: no cell
    ev = synth.make_event(4, 2048, dirs, seed_key=21)
    gpu = run_gpu(ctx, pid, ev)
    ref = oracle.unfold_event(pat, ev)
    check_event(gpu, ref, ev)
    assert np.all(gpu["status"][1:3] == oracle.ST_BAD_DIR) and np.all(gpu["status"][8:10] == oracle.ST_BAD_DIR)
    assert np.all(gpu["efield"][1:3] == 0) and np.all(gpu["peak_idx"][1:3] == 0)
    assert np.all(gpu["efield"][8:10] == 0) and np.all(gpu["envelope"][8:10] == 0)
    assert np.all(gpu["status"][3:5] & oracle.ST_ZEN_CLAMP)


def test_singular_antenna(ctx):
    pat = synth.make_flat_pattern(np.array([[1.0, 2.0], [0.5, 1.0]]))   # rank one everywhere
    pid = ctx.load_pattern(pat)
    ev = synth.make_event(3, 1024, synth.scan_directions(2, 2), seed_key=22)
    gpu = run_gpu(ctx, pid, ev)
    assert np.all(gpu["status"] == oracle.ST_SINGULAR)
    assert np.all(gpu["efield"] == 0) and np.all(gpu["envelope"] == 0)
    ref = oracle.unfold_event(pat, ev)
    assert np.array_equal(ref["status"], gpu["status"].astype(np.uint32))


@pytest.mark.parametrize("scale", [1e-12, 1e12])
def test_parity_with_the_table_scaled(ctx, pat, scale):
    """The same antenna in other units: the VEL table times 1e-12 or 1e12. The near-singular
    test and the per-bin inverse work on H normalised by a power of two, so no bin is flagged
    or lost to FP32 underflow or overflow; the FP64 oracle is exact at both scales. Also on the
    tensor-core variant, which shares the per-bin inverse."""
    import dataclasses
    sp = dataclasses.replace(pat, table=(pat.table.astype(np.complex128) * scale).astype(np.complex64))
    pid_s = ctx.load_pattern(sp)
    rng = np.random.default_rng(31)
    ev = synth.make_event(6, 2048, synth.random_directions(4, rng), seed_key=32)
    gpu = run_gpu(ctx, pid_s, ev)
    ref = oracle.unfold_event(sp, ev)
    assert np.all(ref["status"] == 0) and np.all(gpu["status"] == 0)
    check_event(gpu, ref, ev)
    tc = ctx.unfold_tc(pid_s, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad),
                       split_terms=6, sync=True)
    tc = {k: (v.cpu().numpy() if v is not None else None) for k, v in tc.items()}
    check_event(tc, ref, ev)


def test_peaks_only_matches_full(ctx, pid):
    ev = synth.make_event(9, 2048, synth.scan_directions(3, 3), seed_key=23)
    full = run_gpu(ctx, pid, ev)
    peaks = run_gpu(ctx, pid, ev, traces_out=False)
    for k in ("peak_idx", "peak_amp", "peak_time_ns", "residual_ns", "t0_ns", "chi2", "status"):
        assert np.array_equal(full[k], peaks[k]), k


def test_host_entry_point_matches_device(ctx, pid):
    ev = synth.make_event(6, 4096, synth.scan_directions(2, 3), seed_key=24)
    dev = run_gpu(ctx, pid, ev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    host = ctx.unfold_host(pid, t(ev.traces), t(ev.pos_m), t(ev.t_start_ns), t(ev.dirs_rad))
    for k, v in dev.items():
        assert np.array_equal(v, host[k].numpy()), k


def test_deterministic(ctx, pid):
    ev = synth.make_event(17, 1024, synth.scan_directions(4, 5), seed_key=25)
    a = run_gpu(ctx, pid, ev)
    b = run_gpu(ctx, pid, ev)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_refractive_index(ctx, pat, pid):
    ev = synth.make_event(8, 1024, synth.scan_directions(2, 2), seed_key=26)
    gpu = run_gpu(ctx, pid, ev, n_refr=1.000292)
    for d in range(ev.n_dirs):
        r, t0, chi2 = oracle.residual(ev.pos_m, gpu["peak_time_ns"][d], *ev.dirs_rad[d], n_refr=1.000292)
        check_times(gpu["residual_ns"][d], r, "residual with n")


def test_argument_validation(ctx, pid):
    from paper_1507_07733_gb300 import binding
    ev = synth.make_event(2, 1024, synth.scan_directions(1, 2), seed_key=27)
    tr, pos, ts, dirs = _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad)
    with pytest.raises(binding.ArError) as e:
        ctx.unfold(pid, _dev(np.zeros((2, 2, 512), np.float32)), pos, ts, dirs)
    assert e.value.status == 2
    with pytest.raises(binding.ArError) as e:
        ctx.unfold(pid + 100, tr, pos, ts, dirs)
    assert e.value.status == 3
    with pytest.raises(binding.ArError) as e:
        ctx.unfold(pid, tr, pos, ts, dirs, fs_hz=100e6)   # 80 MHz above Nyquist
    assert e.value.status == 1
    out, st = binding.alloc_outputs(2, 2, 1024)
    st.peak_idx = None
    with pytest.raises(binding.ArError) as e:
        binding.ar_unfold(ctx.h, binding.make_event(pid, tr, pos, ts, dirs), st)
    assert e.value.status == 1


@pytest.mark.parametrize("n,s,d", [(1024, 124, 16), (4096, 40, 16), (2048, 124, 12)])
def test_parity_many_pairs_per_cta(ctx, pat, pid, n, s, d):
    """More pairs than resident CTAs, so every CTA walks several pairs (and directions):
    sampled pairs against the oracle, every direction's residual from the GPU's peaks."""
    rng = np.random.default_rng(n + s + d)
    ev = synth.make_event(s, n, synth.random_directions(d, rng), seed_key=30 + n)
    gpu = run_gpu(ctx, pid, ev)
    q = np.concatenate([[0, s * d - 1], rng.choice(s * d, 30, replace=False)])
    di, si = q // s, q % s
    ref = oracle.unfold_sample(pat, ev, si, di)
    sub = {k: gpu[k][di, si] for k in ("efield", "envelope", "peak_idx", "peak_amp", "status")}
    check_pairs(sub, ref, n)
    check_times(gpu["peak_time_ns"][di, si], ref["peak_time_ns"], "peak time")
    env, amp, idx = gpu["envelope"], gpu["peak_amp"], gpu["peak_idx"]
    assert np.all(env.max(axis=2) == amp)
    assert np.array_equal(np.argmax(env == amp[..., None], axis=2), idx)
    for dd in range(d):
        r, t0, chi2 = oracle.residual(ev.pos_m, gpu["peak_time_ns"][dd], *ev.dirs_rad[dd])
        check_times(gpu["residual_ns"][dd], r, "residual")
        assert abs(gpu["chi2"][dd] - chi2) <= 1e-9 * max(chi2, 1.0)
