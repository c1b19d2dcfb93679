"""GPU: the continuous-batching server.

Every request's result must be the same alone and in the mix (bit for bit: the per-pair
arithmetic and the residual's summation order do not depend on the batch), equal to the
plain ar_unfold result, and within the oracle's tolerance on sampled pairs. Admission under
a state budget that fits one event at a time still completes every request; events that can
never fit are refused at submission.
"""
import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _host_event(binding, pid, ev):
    arrays = tuple(_pinned(a) for a in (ev.traces, ev.pos_m, ev.t_start_ns, ev.dirs_rad))
    return binding.make_event(pid, *arrays, ev.fs_hz), arrays


def _host_out(binding, ev, traces=True):
    o, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cpu", traces=traces,
                                 pin_memory=True)
    return o


def _np(o):
    return {k: v.numpy().copy() for k, v in o.items() if v is not None}


@pytest.fixture(scope="module")
def env():
    from paper_1507_07733_gb300 import binding
    ctx = binding.Context(0)
    pat = synth.make_pattern()
    pid = ctx.load_pattern(pat)
    rng = np.random.default_rng(808)
    evs = [synth.make_event(S, N, synth.random_directions(D, rng), seed_key=800 + i)
           for i, (S, N, D) in enumerate([(12, 2048, 20), (40, 1024, 33), (7, 4096, 16), (124, 2048, 17),
                                          (3, 1024, 64), (60, 4096, 5), (25, 2048, 40), (90, 1024, 8)])]
    yield binding, ctx, pat, pid, evs
    ctx.close()


def test_alone_equals_in_the_mix(env):
    binding, ctx, pat, pid, evs = env
    srv = binding.Server(ctx, max_batch_events=8, max_inflight=2)
    target = 2
    # alone: the server is idle when the event arrives
    ev_t, keep_t = _host_event(binding, pid, evs[target])
    out_alone = _host_out(binding, evs[target])
    tk = srv.submit(ev_t, out_alone)
    assert srv.wait(tk) == 0
    alone = _np(out_alone)
    # in the mix: every event submitted back to back, three rounds, the target among them
    keeps, tickets, outs = [], [], []
    for rnd in range(3):
        for i, e in enumerate(evs):
            ev_s, keep = _host_event(binding, pid, e)
            o = _host_out(binding, e)
            keeps.append(keep)
            outs.append((i, o))
            tickets.append(srv.submit(ev_s, o))
    for t in tickets:
        assert srv.wait(t) == 0
    for i, o in outs:
        if i == target:
            mixed = _np(o)
            for k in alone:
                assert np.array_equal(alone[k], mixed[k]), k
    # equal to the plain path, and to the oracle on sampled pairs
    e = evs[target]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    plain = ctx.unfold(pid, dev(e.traces), dev(e.pos_m), dev(e.t_start_ns), dev(e.dirs_rad), sync=True)
    for k, v in plain.items():
        assert np.array_equal(v.cpu().numpy(), alone[k]), k
    rng = np.random.default_rng(1)
    q = rng.choice(e.n_stations * e.n_dirs, 4, replace=False)
    di, si = q // e.n_stations, q % e.n_stations
    ref = oracle.unfold_sample(pat, e, si, di)
    check_pairs({k: alone[k][di, si] for k in ("efield", "envelope", "peak_idx", "peak_amp", "status")}, ref,
                e.n_samples)
    for t in tickets + [tk]:
        st, t_sub, t_done = srv.times(t)
        assert st == 0 and t_done >= t_sub > 0
        assert srv.release(t) == 0
    srv.close()


def test_admission_under_a_small_budget(env):
    binding, ctx, pat, pid, evs = env
    sizes = []
    for e in evs[:4]:
        S, D, N = e.n_stations, e.n_dirs, e.n_samples
        sizes.append(S * 2 * N * 4 + D * S * 12 * N + D * S * 40 + 64 * 1024)
    srv = binding.Server(ctx, state_budget_bytes=int(max(sizes) * 1.05), max_batch_events=4, max_inflight=2)
    keeps, tickets, outs = [], [], []
    for e in evs[:4]:
        ev_s, keep = _host_event(binding, pid, e)
        o = _host_out(binding, e)
        keeps.append(keep)
        outs.append(o)
        tickets.append(srv.submit(ev_s, o))
    for t in tickets:
        assert srv.wait(t) == 0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for e, o in zip(evs[:4], outs):
        plain = ctx.unfold(pid, dev(e.traces), dev(e.pos_m), dev(e.t_start_ns), dev(e.dirs_rad), sync=True)
        for k, v in plain.items():
            assert np.array_equal(v.cpu().numpy(), o[k].numpy()), k
    srv.close()


def test_refusals(env):
    binding, ctx, pat, pid, evs = env
    srv = binding.Server(ctx, state_budget_bytes=1 << 20, max_batch_events=2, max_inflight=1)
    ev_s, keep = _host_event(binding, pid, evs[3])            # 124 x 17 x 2048 x 12 B >> 1 MiB
    o = _host_out(binding, evs[3])
    with pytest.raises(binding.ArError) as e:
        srv.submit(ev_s, o)
    assert e.value.status == 5
    assert srv.poll(123456) == 1                                # unknown ticket
    # peaks only: small enough for the budget
    small = synth.make_event(3, 1024, synth.scan_directions(2, 2), seed_key=850)
    ev2, keep2 = _host_event(binding, pid, small)
    o2 = _host_out(binding, small, traces=False)
    tk = srv.submit(ev2, o2)
    assert srv.wait(tk, 0) in (0, 7)                            # done already, or timed out at once
    assert srv.wait(tk) == 0
    srv.close()
