"""GPU: the tensor-core DFT variant (ar_unfold_tc) against the FP64 oracle.

The three-way split with six products (x6) carries FP32-level precision and must meet the
path's bar (E-field and envelope rel L2 <= 1e-5 per pair, peaks, timing). The two-way split
with three products (x3) keeps about 16 significant bits per product: its bar is derived from
that, rel L2 <= 1e-4 per pair, peak ties judged at 1e-4, and it is reported beside the FP32
path's error on the single event at 4096 samples (10 stations, zenith 30 deg, azimuth 45 deg).
"""
import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_event, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

X3_REL_L2 = 1e-4


@pytest.fixture(scope="module")
def env():
    from paper_1507_07733_gb300 import binding
    ctx = binding.Context(0)
    pat = synth.make_pattern()
    pid = ctx.load_pattern(pat)
    yield binding, ctx, pat, pid
    ctx.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(ctx, pid, ev, terms, traces_out=True):
    out = ctx.unfold_tc(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad),
                        split_terms=terms, fs_hz=ev.fs_hz, traces_out=traces_out, sync=True)
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


@pytest.mark.parametrize("n,s,d", [(4096, 10, 1), (2048, 7, 5), (1024, 13, 9), (4096, 3, 2), (2048, 1, 1)])
def test_x6_meets_the_parity_bar(env, n, s, d):
    binding, ctx, pat, pid = env
    if (n, s, d) == (4096, 10, 1):
        ev = synth.single_event(n_samples=4096)
    else:
        rng = np.random.default_rng(3 * n + s + d)
        ev = synth.make_event(s, n, synth.random_directions(d, rng), seed_key=900 + n + s)
    gpu = _run(ctx, pid, ev, 6)
    ref = oracle.unfold_event(pat, ev)
    check_event(gpu, ref, ev)


@pytest.mark.parametrize("n,fs_mhz", [(2048, 227.0), (1024, 240.0), (4096, 233.0)])
def test_x6_parity_off_the_default_band_offset(env, n, fs_mhz):
    """Sampling rates whose band starts at k_lo = 271 (2048), 128 (1024) and 528 (4096)
    instead of the 200 MHz windows: the transform tables follow k_lo."""
    binding, ctx, pat, pid = env
    rng = np.random.default_rng(n + int(fs_mhz))
    ev = synth.make_event(5, n, synth.random_directions(3, rng), seed_key=960 + n // 1024, fs_hz=fs_mhz * 1e6)
    check_event(_run(ctx, pid, ev, 6), oracle.unfold_event(pat, ev), ev)


def test_x3_error_on_the_single_event(env):
    binding, ctx, pat, pid = env
    ev = synth.single_event(n_samples=4096)
    ref = oracle.unfold_event(pat, ev)
    gpu = _run(ctx, pid, ev, 3)
    N = ev.n_samples
    e = rel_l2(gpu["efield"], ref["efield"], 2 * N)
    v = rel_l2(gpu["envelope"], ref["envelope"], N)
    print(f"x3: E-field rel L2 max {e.max():.3g} median {np.median(e):.3g}; envelope max {v.max():.3g}")
    assert e.max() <= X3_REL_L2 and v.max() <= X3_REL_L2
    gi, oi = gpu["peak_idx"].reshape(-1), ref["peak_idx"].reshape(-1)
    envr = ref["envelope"].reshape(gi.size, N)
    for q in np.flatnonzero(gi != oi):
        assert abs(envr[q, gi[q]] - envr[q, oi[q]]) <= X3_REL_L2 * envr[q, oi[q]]
    assert np.array_equal(gpu["status"], ref["status"])
    # the timing follows the peaks
    assert np.allclose(gpu["peak_time_ns"], ev.t_start_ns[None, :] + gpu["peak_idx"] * 5.0, rtol=0, atol=1e-9)


def test_x6_agrees_with_the_fp32_path_over_chunks(env):
    """Enough pairs for two inverse chunks (2^25 / N pairs each): every pair against the FP32
    FFT path, a sample against the oracle."""
    binding, ctx, pat, pid = env
    rng = np.random.default_rng(77)
    ev = synth.make_event(124, 1024, synth.random_directions(300, rng), seed_key=977)
    gpu = _run(ctx, pid, ev, 6)
    fp32 = ctx.unfold(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad), sync=True)
    fp32 = {k: v.cpu().numpy() for k, v in fp32.items()}
    e = rel_l2(gpu["efield"], fp32["efield"], 2 * 1024)
    assert e.max() <= 1e-5, e.max()
    assert np.array_equal(gpu["status"], fp32["status"])
    same = gpu["peak_idx"] == fp32["peak_idx"]
    assert same.mean() > 0.999
    q = rng.choice(ev.n_stations * ev.n_dirs, 6, replace=False)
    di, si = q // ev.n_stations, q % ev.n_stations
    ref = oracle.unfold_sample(pat, ev, si, di)
    for k in ("efield", "envelope"):
        n = 2 * 1024 if k == "efield" else 1024
        assert rel_l2(gpu[k][di, si], ref[k], n).max() <= 1e-5


def test_peaks_only_and_argument_checks(env):
    binding, ctx, pat, pid = env
    ev = synth.make_event(5, 2048, synth.scan_directions(2, 2), seed_key=978)
    full = _run(ctx, pid, ev, 6)
    peaks = _run(ctx, pid, ev, 6, traces_out=False)
    for k in ("peak_idx", "peak_amp", "peak_time_ns", "residual_ns", "t0_ns", "chi2", "status"):
        assert np.array_equal(full[k], peaks[k]), k
    with pytest.raises(binding.ArError) as e:
        ctx.unfold_tc(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad), split_terms=4)
    assert e.value.status == 1
    # S * N above 2^24 is refused before any work (buffers of the full size are given)
    big_s = (1 << 14) + 1
    tr = torch.zeros((big_s, 2, 1024), dtype=torch.float32, device="cuda")
    pos = torch.zeros((big_s, 3), dtype=torch.float64, device="cuda")
    ts = torch.zeros(big_s, dtype=torch.float64, device="cuda")
    dirs = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.ArError) as e:
        ctx.unfold_tc(pid, tr, pos, ts, dirs, split_terms=3)
    assert e.value.status == 1


def test_x3_and_x6_on_the_scan_in_the_benchmark_configuration(env):
    """The direction scan (124 stations x 64 directions x 2048 samples) as the benchmark runs
    it: x6 at the full bar and x3 at its bar on sampled pairs; every pair's peak time follows
    its index; residuals against the oracle's residuals at the GPU's peak times."""
    binding, ctx, pat, pid = env
    ev = synth.direction_scan()
    rng = np.random.default_rng(2048)
    q = rng.choice(ev.n_stations * ev.n_dirs, 24, replace=False)
    di, si = q // ev.n_stations, q % ev.n_stations
    ref = oracle.unfold_sample(pat, ev, si, di)
    for terms, bar in ((6, 1e-5), (3, X3_REL_L2)):
        gpu = _run(ctx, pid, ev, terms)
        e = rel_l2(gpu["efield"][di, si], ref["efield"], 2 * ev.n_samples)
        v = rel_l2(gpu["envelope"][di, si], ref["envelope"], ev.n_samples)
        assert e.max() <= bar and v.max() <= bar, (terms, e.max(), v.max())
        assert np.array_equal(gpu["status"][di, si], ref["status"])
        assert np.allclose(gpu["peak_time_ns"], ev.t_start_ns[None, :] + gpu["peak_idx"] * 5.0, rtol=0, atol=1e-9)
        for d in range(0, ev.n_dirs, 9):
            r, t0, chi2 = oracle.residual(ev.pos_m, gpu["peak_time_ns"][d], *ev.dirs_rad[d])
            assert np.allclose(gpu["residual_ns"][d], r, rtol=0, atol=1e-9 * max(1.0, np.abs(r).max()))


def test_fine_times_and_snr_on_the_scan(env):
    """The scan through the tensor-core path with sub-sample times and SNRs: peaks only equals
    full outputs bit for bit, and the times and SNRs agree with the FP32 path to the x6
    precision."""
    binding, ctx, pat, pid = env
    ev = synth.direction_scan()
    args = (pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad))
    res = {}
    for traces in (True, False):
        out, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cuda", traces=traces,
                                       fine=True, snr=True)
        ctx.unfold_tc(*args, split_terms=6, fs_hz=ev.fs_hz, out=out, sync=True)
        res[traces] = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    for k in ("peak_idx", "peak_amp", "peak_time_ns", "peak_time_fine_ns", "snr", "residual_ns", "t0_ns", "chi2",
              "status"):
        assert np.array_equal(res[True][k], res[False][k]), k
    fp, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cuda", fine=True, snr=True)
    ctx.unfold(*args, ev.fs_hz, out=fp, sync=True)
    fp = {k: v.cpu().numpy() for k, v in fp.items()}
    tc = res[True]
    same = tc["peak_idx"] == fp["peak_idx"]
    assert same.mean() > 0.999
    assert np.all(abs(tc["peak_time_fine_ns"][same] - fp["peak_time_fine_ns"][same]) <= 0.01 * 5.0)
    assert np.all(abs(tc["snr"][same] - fp["snr"][same]) <= 1e-4 * fp["snr"][same])
    e = rel_l2(tc["envelope"], fp["envelope"], ev.n_samples)
    assert e.max() <= 1e-5, e.max()
