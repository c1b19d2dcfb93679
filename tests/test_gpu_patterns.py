"""GPU: several antenna patterns per event (per-station pattern ids, Sec. 3: the patterns of
every antenna type are resident on the device together).

Three patterns: two on the standard 19 x 72 x 51 grid and one on the paper's largest grid
(31 zenith x 48 periodic azimuth x 98 frequency nodes). The oracle runs each station with its
own pattern; the residuals follow from the oracle's peak times. Stations grouped by pattern
and mixed give the same per-pair results as one-pattern runs (bit for bit); an id that was
never loaded zeroes that station's pairs and sets AR_STATUS_BAD_PATTERN; the batch, server,
host-buffer and tensor-core paths take the ids too.
"""
import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_event, check_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BAD_PATTERN = 8


@pytest.fixture(scope="module")
def env():
    from paper_1507_07733_gb300 import binding
    ctx = binding.Context(0)
    pats = synth.mixed_antenna_patterns()
    ids = [ctx.load_pattern(p) for p in pats]
    yield binding, ctx, pats, ids
    ctx.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(out):
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def _run(ctx, pid, ev, station_pattern=None, tc_terms=0, traces_out=True):
    args = (pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad))
    sp = _dev(np.asarray(station_pattern, np.int32)) if station_pattern is not None else None
    if tc_terms:
        out = ctx.unfold_tc(*args, split_terms=tc_terms, fs_hz=ev.fs_hz, traces_out=traces_out, sync=True,
                            station_pattern=sp)
    else:
        out = ctx.unfold(*args, ev.fs_hz, traces_out=traces_out, sync=True, station_pattern=sp)
    return _np(out)


def _oracle(pats, ev, types):
    """Each station through the oracle with its own pattern; residuals from those peak times."""
    D, S, N = ev.n_dirs, ev.n_stations, ev.n_samples
    ref = dict(efield=np.zeros((D, S, 2, N)), envelope=np.zeros((D, S, N)), peak_idx=np.zeros((D, S), np.int32),
               peak_amp=np.zeros((D, S)), peak_time_ns=np.zeros((D, S)), status=np.zeros((D, S), np.uint32),
               min_margin=np.ones((D, S)))
    for t, pat in enumerate(pats):
        st = np.flatnonzero(types == t)
        if st.size == 0:
            continue
        si = np.tile(st, D)
        di = np.repeat(np.arange(D), st.size)
        r = oracle.unfold_sample(pat, ev, si, di)
        for k in ("efield", "envelope", "peak_idx", "peak_amp", "peak_time_ns", "status", "min_margin"):
            ref[k][di, si] = r[k]
    ref["residual_ns"] = np.empty((D, S))
    ref["t0_ns"] = np.empty(D)
    ref["chi2"] = np.empty(D)
    for d in range(D):
        ref["residual_ns"][d], ref["t0_ns"][d], ref["chi2"][d] = oracle.residual(ev.pos_m, ref["peak_time_ns"][d],
                                                                                 *ev.dirs_rad[d])
    return ref


@pytest.mark.parametrize("n,s,d,grouped", [(2048, 24, 5, True), (1024, 31, 4, False), (4096, 9, 3, False)])
def test_mixed_patterns_match_the_oracle(env, n, s, d, grouped):
    binding, ctx, pats, ids = env
    rng = np.random.default_rng(n + s)
    ev = synth.make_event(s, n, synth.random_directions(d, rng), seed_key=1200 + s)
    types = synth.station_antenna_types(s, sort=grouped, seed_key=s)
    gpu = _run(ctx, ids[0], ev, np.asarray(ids, np.int32)[types])
    check_event(gpu, _oracle(pats, ev, types), ev)


def test_each_station_equals_its_one_pattern_run(env):
    """Per-pair results do not depend on the other stations' patterns or on the walk order."""
    binding, ctx, pats, ids = env
    ev = synth.make_event(40, 2048, synth.scan_directions(3, 2), seed_key=1210)
    types = synth.station_antenna_types(40, sort=False, seed_key=5)
    mixed = _run(ctx, ids[0], ev, np.asarray(ids, np.int32)[types])
    for t, pid in enumerate(ids):
        one = _run(ctx, pid, ev)
        st = types == t
        for k in ("efield", "envelope", "peak_idx", "peak_amp", "peak_time_ns", "status"):
            assert np.array_equal(mixed[k][:, st], one[k][:, st]), (t, k)
    # every station on one pattern through the ids equals the plain call
    same = _run(ctx, ids[1], ev, np.full(40, ids[1], np.int32))
    plain = _run(ctx, ids[1], ev)
    for k in plain:
        assert np.array_equal(same[k], plain[k]), k


def test_unknown_pattern_id(env):
    binding, ctx, pats, ids = env
    ev = synth.make_event(12, 1024, synth.scan_directions(2, 2), seed_key=1220)
    sp = np.full(12, ids[0], np.int32)
    sp[3], sp[7] = 99, -1
    gpu = _run(ctx, ids[0], ev, sp)
    good = _run(ctx, ids[0], ev)
    bad = np.zeros(12, bool)
    bad[[3, 7]] = True
    assert np.all(gpu["status"][:, bad] == BAD_PATTERN)
    assert not np.any(gpu["efield"][:, bad]) and not np.any(gpu["envelope"][:, bad])
    assert np.all(gpu["peak_idx"][:, bad] == 0) and np.all(gpu["peak_amp"][:, bad] == 0)
    for k in ("efield", "envelope", "peak_idx", "peak_amp", "status"):
        assert np.array_equal(gpu[k][:, ~bad], good[k][:, ~bad]), k


def test_tensor_core_and_host_paths_take_the_ids(env):
    binding, ctx, pats, ids = env
    ev = synth.make_event(14, 4096, synth.scan_directions(2, 1), seed_key=1230)
    types = synth.station_antenna_types(14, sort=False, seed_key=6)
    sp = np.asarray(ids, np.int32)[types]
    ref = _oracle(pats, ev, types)
    check_event(_run(ctx, ids[0], ev, sp, tc_terms=6), ref, ev)
    dev = _run(ctx, ids[0], ev, sp)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    host = ctx.unfold_host(ids[0], pin(ev.traces), pin(ev.pos_m), pin(ev.t_start_ns), pin(ev.dirs_rad), ev.fs_hz,
                           station_pattern=pin(sp))
    for k, v in host.items():
        assert np.array_equal(v.numpy(), dev[k]), k


def test_batch_and_server_take_the_ids(env):
    binding, ctx, pats, ids = env
    evs, sps = [], []
    for i, (s, n, d) in enumerate([(10, 2048, 6), (25, 1024, 3), (7, 4096, 5)]):
        rng = np.random.default_rng(40 + i)
        evs.append(synth.make_event(s, n, synth.random_directions(d, rng), seed_key=1240 + i))
        sps.append(np.asarray(ids, np.int32)[synth.station_antenna_types(s, sort=i != 1, seed_key=20 + i)])
    plain = [_run(ctx, ids[0], e, sp) for e, sp in zip(evs, sps)]
    # batch: one graph launch over the three events
    keep, structs, outs = [], [], []
    for e, sp in zip(evs, sps):
        k = (_dev(e.traces), _dev(e.pos_m), _dev(e.t_start_ns), _dev(e.dirs_rad), _dev(sp))
        keep.append(k)
        structs.append(binding.make_event(ids[0], *k[:4], e.fs_hz, 1.0, k[4]))
        outs.append(binding.alloc_outputs(e.n_dirs, e.n_stations, e.n_samples, device="cuda")[0])
    b = ctx.batch(4, 64, 64, max_n_freq=128)
    b.run(structs, outs)
    torch.cuda.synchronize()
    for o, p in zip(outs, plain):
        for k, v in o.items():
            assert np.array_equal(v.cpu().numpy(), p[k]), k
    b.close()
    # server: host buffers
    srv = binding.Server(ctx, max_batch_events=4, max_inflight=2, max_n_freq=128)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    tickets, houts, hkeep = [], [], []
    for e, sp in zip(evs, sps):
        k = (pin(e.traces), pin(e.pos_m), pin(e.t_start_ns), pin(e.dirs_rad), pin(sp))
        hkeep.append(k)
        o, _ = binding.alloc_outputs(e.n_dirs, e.n_stations, e.n_samples, device="cpu", pin_memory=True)
        houts.append(o)
        tickets.append(srv.submit(binding.make_event(ids[0], *k[:4], e.fs_hz, 1.0, k[4]), o))
    for t in tickets:
        assert srv.wait(t) == 0
    for o, p in zip(houts, plain):
        for k, v in o.items():
            assert np.array_equal(v.numpy(), p[k]), k
    srv.close()


def test_reconstruction_takes_the_ids(env):
    """The iterative loop with every station's id set to one pattern equals the loop on that
    pattern (same directions, iterations and last unfold, bit for bit)."""
    binding, ctx, pats, ids = env
    ev = synth.make_event(40, 2048, synth.scan_directions(1, 1), seed_key=1250)
    args = (_dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns))
    plain = ctx.reconstruct(ids[1], *args, ev.fs_hz, max_iter=6)
    sp = _dev(np.full(40, ids[1], np.int32))
    unused_dirs = torch.zeros((1, 2), dtype=torch.float64, device="cuda")   # the event holds raw pointers
    e = binding.make_event(ids[0], *args, unused_dirs, ev.fs_hz, 1.0, sp)
    # the binding's reconstruct builds its own event; run the ABI call directly with the ids
    last, _ = binding.alloc_outputs(1, 40, 2048, device="cuda")
    res = dict(direction=torch.empty(2, dtype=torch.float64, device="cuda"),
               t0_ns=torch.empty(1, dtype=torch.float64, device="cuda"),
               chi2=torch.empty(1, dtype=torch.float64, device="cuda"),
               iterations=torch.empty(1, dtype=torch.int32, device="cuda"),
               history=torch.empty((7, 2), dtype=torch.float64, device="cuda"))
    out = binding.ar_recon_out(binding._ptr(res["direction"]), binding._ptr(res["t0_ns"]), binding._ptr(res["chi2"]),
                               binding._ptr(res["iterations"]), binding._ptr(res["history"]),
                               binding.outputs_struct(last))
    st = torch.cuda.current_stream()
    binding.ar_reconstruct(ctx.h, e, 6, 1e-6, out, st.cuda_stream)
    binding.ar_sync(ctx.h, st.cuda_stream)
    for k in ("direction", "t0_ns", "chi2", "iterations", "history"):
        assert np.array_equal(np.nan_to_num(res[k].cpu().numpy()), np.nan_to_num(plain[k].cpu().numpy())), k
    for k, v in last.items():
        assert np.array_equal(v.cpu().numpy(), plain["last"][k].cpu().numpy()), k


def test_batch_mixes_events_with_and_without_ids(env):
    """A batch whose CTAs walk from an event without ids (its first key is built before the
    wait for the station kernel) into one with ids (stations walked grouped by pattern, in an
    order the station kernel writes): bit for bit the plain calls of each event."""
    binding, ctx, pats, ids = env
    evs = [synth.make_event(124, 1024, synth.scan_directions(4, 4), seed_key=1260),
           synth.make_event(100, 1024, synth.scan_directions(5, 2), seed_key=1261)]
    sps = [None, np.asarray(ids, np.int32)[synth.station_antenna_types(100, sort=False, seed_key=31)]]
    plain = [_run(ctx, ids[0], e, sp) for e, sp in zip(evs, sps)]
    keep, structs, outs = [], [], []
    for e, sp in zip(evs, sps):
        k = (_dev(e.traces), _dev(e.pos_m), _dev(e.t_start_ns), _dev(e.dirs_rad),
             _dev(sp) if sp is not None else None)
        keep.append(k)
        structs.append(binding.make_event(ids[0], *k[:4], e.fs_hz, 1.0, k[4]))
        outs.append(binding.alloc_outputs(e.n_dirs, e.n_stations, e.n_samples, device="cuda")[0])
    b = ctx.batch(2, 224, 32, max_n_freq=128)
    for _ in range(2):   # a replay reuses the walk workspace
        b.run(structs, outs)
        torch.cuda.synchronize()
        for o, p in zip(outs, plain):
            for k, v in o.items():
                assert np.array_equal(v.cpu().numpy(), p[k]), k
    b.close()
