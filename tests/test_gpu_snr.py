"""GPU: the pulse SNR and the SNR-weighted direction fit (a variant) against the oracle.

SNR bound, derived from the path's envelope bar: if the envelope e carries an error d with
||d||_2 <= eta ||e||_2 (eta = 1e-5), then e_k^2 moves by at most 2 e_k eta ||e||_2 and the
noise sum of squares by at most 2 ||e_noise||_2 eta ||e||_2, so the SNR's relative error is
at most 2 eta ||e||_2 (1 / e_k + 1 / ||e_noise||_2) to first order, plus 1e-5 for the FP32
sums. Pairs whose peak index is a tie or whose solve is near the singular threshold are
skipped, as in the main parity tests. The weighted residual, t0 and chi2 are compared
(1e-9 relative) with the oracle's weighted fit at the GPU's own peak times and SNRs.
"""
import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_pairs, check_times

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ETA = 1e-5


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


def _run(binding, ctx, pid, ev, traces=True, tc_terms=0, station_pattern=None):
    out, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cuda", traces=traces, snr=True)
    args = (pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad))
    sp = _dev(np.asarray(station_pattern, np.int32)) if station_pattern is not None else None
    if tc_terms:
        ctx.unfold_tc(*args, split_terms=tc_terms, fs_hz=ev.fs_hz, out=out, sync=True, station_pattern=sp)
    else:
        ctx.unfold(*args, ev.fs_hz, out=out, sync=True, station_pattern=sp)
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def check_weighted_fit(gpu, ev):
    for d in range(ev.n_dirs):
        w = gpu["snr"][d].astype(np.float64)
        r, t0, chi2 = oracle.residual_weighted(ev.pos_m, gpu["peak_time_ns"][d], w, *ev.dirs_rad[d])
        check_times(gpu["residual_ns"][d], r, "weighted residual")
        check_times(gpu["t0_ns"][d], t0, "weighted t0")
        assert abs(gpu["chi2"][d] - chi2) <= 1e-9 * max(abs(chi2), 1.0), (d, gpu["chi2"][d], chi2)


def check_snr(gpu, ref, ev):
    N = ev.n_samples
    want = oracle.event_snr(ref["envelope"], ref["peak_idx"])
    checked = 0
    for d in range(ev.n_dirs):
        for s in range(ev.n_stations):
            k = int(ref["peak_idx"][d, s])
            if gpu["peak_idx"][d, s] != k or ref["min_margin"][d, s] <= 1e-5:
                continue
            e = ref["envelope"][d, s]
            far = np.abs(np.arange(N) - k) > N // 16
            bound = 2 * ETA * np.linalg.norm(e) * (1 / e[k] + 1 / np.linalg.norm(e[far])) + 1e-5
            assert abs(gpu["snr"][d, s] - want[d, s]) <= bound * want[d, s], (d, s, gpu["snr"][d, s], want[d, s])
            checked += 1
    assert checked >= ev.n_dirs * ev.n_stations // 2
    check_weighted_fit(gpu, ev)


@pytest.mark.parametrize("n,s,d", [(1024, 13, 5), (2048, 9, 4), (4096, 6, 3)])
def test_snr_and_weighted_fit(env, n, s, d):
    binding, ctx, pat, pid = env
    rng = np.random.default_rng(11 * n + s)
    ev = synth.make_event(s, n, synth.random_directions(d, rng), seed_key=1400 + s)
    gpu = _run(binding, ctx, pid, ev)
    ref = oracle.unfold_event(pat, ev)
    check_pairs(gpu, ref, n)
    check_snr(gpu, ref, ev)
    assert np.all(gpu["snr"] > 0.0)
    # the weights change the fit: t0 differs from the unweighted one
    r, t0, _ = oracle.residual(ev.pos_m, gpu["peak_time_ns"][0], *ev.dirs_rad[0])
    assert gpu["t0_ns"][0] != t0
    # peaks only: the same SNRs and fit
    po = _run(binding, ctx, pid, ev, traces=False)
    for k in ("peak_idx", "peak_time_ns", "snr", "residual_ns", "t0_ns", "chi2"):
        assert np.array_equal(po[k], gpu[k]), k


def test_zero_weights_fall_back_to_the_unweighted_fit(env):
    """Stations with an unknown pattern id have a zero envelope, SNR 0 and no weight; a
    direction whose stations all have weight 0 gets the unweighted fit."""
    binding, ctx, pat, pid = env
    ev = synth.make_event(10, 2048, synth.scan_directions(2, 1), seed_key=1410)
    ids = np.full(10, pid, np.int32)
    ids[[2, 7]] = 99
    gpu = _run(binding, ctx, pid, ev, station_pattern=ids)
    assert np.all(gpu["snr"][:, [2, 7]] == 0) and np.all(gpu["snr"][:, ids == pid] > 0)
    check_weighted_fit(gpu, ev)
    allbad = _run(binding, ctx, pid, ev, station_pattern=np.full(10, 99, np.int32))
    assert np.all(allbad["snr"] == 0)
    for d in range(ev.n_dirs):
        r, t0, chi2 = oracle.residual(ev.pos_m, allbad["peak_time_ns"][d], *ev.dirs_rad[d])
        check_times(allbad["residual_ns"][d], r, "unweighted residual")
        check_times(allbad["t0_ns"][d], t0, "unweighted t0")


def test_snr_on_the_tensor_core_host_batch_and_server_paths(env):
    binding, ctx, pat, pid = env
    ev = synth.single_event(4096)
    ref = oracle.unfold_event(pat, ev)
    tc = _run(binding, ctx, pid, ev, tc_terms=6)
    check_pairs(tc, ref, 4096)
    check_snr(tc, ref, ev)
    dev = _run(binding, ctx, pid, ev)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hin = (pin(ev.traces), pin(ev.pos_m), pin(ev.t_start_ns), pin(ev.dirs_rad))
    hout, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cpu", pin_memory=True, snr=True)
    ctx.unfold_host(pid, *hin, ev.fs_hz, out=hout)
    for k, v in hout.items():
        assert np.array_equal(v.numpy(), dev[k]), k
    # batch (device buffers) and server (host buffers)
    keep = (_dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad))
    bout, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cuda", snr=True)
    b = ctx.batch(2, 16, 4, max_n_freq=64)
    b.run([binding.make_event(pid, *keep, ev.fs_hz)], [bout])
    torch.cuda.synchronize()
    for k, v in bout.items():
        assert np.array_equal(v.cpu().numpy(), dev[k]), k
    b.close()
    srv = binding.Server(ctx, max_batch_events=2, max_inflight=2, max_n_freq=64)
    sout, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cpu", pin_memory=True, snr=True)
    assert srv.wait(srv.submit(binding.make_event(pid, *hin, ev.fs_hz), sout)) == 0
    for k, v in sout.items():
        assert np.array_equal(v.numpy(), dev[k]), k
    srv.close()


def test_batch_switches_between_the_two_instantiations(env):
    """A batch plan run without SNRs, with them, and without again (one captured graph per
    instantiation): every run equals the plain calls bit for bit."""
    binding, ctx, pat, pid = env
    evs = [synth.make_event(20, 2048, synth.scan_directions(2, 2), seed_key=1420),
           synth.make_event(9, 1024, synth.scan_directions(3, 1), seed_key=1421)]
    keep = [(_dev(e.traces), _dev(e.pos_m), _dev(e.t_start_ns), _dev(e.dirs_rad)) for e in evs]
    structs = [binding.make_event(pid, *k, e.fs_hz) for k, e in zip(keep, evs)]
    b = ctx.batch(2, 40, 8, max_n_freq=64)
    for snr in (False, True, False):
        outs = [binding.alloc_outputs(e.n_dirs, e.n_stations, e.n_samples, device="cuda", snr=snr)[0] for e in evs]
        b.run(structs, outs)
        torch.cuda.synchronize()
        for e, k, o in zip(evs, keep, outs):
            ref, _ = binding.alloc_outputs(e.n_dirs, e.n_stations, e.n_samples, device="cuda", snr=snr)
            ctx.unfold(pid, *k, e.fs_hz, out=ref, sync=True)
            for k, v in o.items():
                assert np.array_equal(v.cpu().numpy(), ref[k].cpu().numpy()), (snr, k)
    b.close()
