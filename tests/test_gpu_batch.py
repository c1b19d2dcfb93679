"""GPU: the batched path (one graph launch over uneven events) against the plain path and
the FP64 oracle.

The batch runs the same per-pair arithmetic as ar_unfold, so its outputs must equal the
plain per-event outputs bit for bit; sampled pairs are also checked against the oracle,
including the full 256-event uneven workload in the launch configuration the benchmark
times (autotuned plan).
"""
import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_pairs, check_times

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _upload(ev):
    return tuple(_dev(a) for a in (ev.traces, ev.pos_m, ev.t_start_ns, ev.dirs_rad))


@pytest.fixture(scope="module")
def setup():
    from paper_1507_07733_gb300 import binding
    ctx = binding.Context(0)
    pat = synth.make_pattern()
    pid = ctx.load_pattern(pat)
    yield binding, ctx, pat, pid
    ctx.close()


def _plain(binding, ctx, pid, ev, inputs):
    return {k: v.cpu().numpy() if v is not None else None
            for k, v in ctx.unfold(pid, *inputs, fs_hz=ev.fs_hz, sync=True).items()}


def test_batch_equals_plain_bit_for_bit(setup):
    binding, ctx, pat, pid = setup
    rng = np.random.default_rng(5)
    # (stations, samples, directions, seed, sampling rate in MHz): three events off the 200 MHz
    # band window, so that one launch walks events with different k_lo and twiddle tables
    descs = [(3, 1024, 16, 701, 200.0), (17, 4096, 5, 702, 200.0), (124, 2048, 3, 703, 227.0),
             (9, 1024, 40, 704, 200.0), (1, 2048, 1, 705, 200.0), (33, 4096, 2, 706, 233.0),
             (64, 2048, 11, 707, 240.0), (5, 1024, 1, 708, 200.0)]
    evs = [synth.make_event(S, N, synth.random_directions(D, rng), seed_key=k, fs_hz=f * 1e6)
           for S, N, D, k, f in descs]
    inputs = [_upload(e) for e in evs]
    plan = ctx.batch(16, 400, 200, 51)
    outs = [binding.alloc_outputs(e.n_dirs, e.n_stations, e.n_samples)[0] for e in evs]
    structs = [binding.make_event(pid, *inp, e.fs_hz) for e, inp in zip(evs, inputs)]
    plan.run(structs, outs)
    torch.cuda.synchronize()
    binding.ar_sync(ctx.h)
    for e, inp, o in zip(evs, inputs, outs):
        ref = _plain(binding, ctx, pid, e, inp)
        for k, v in o.items():
            assert np.array_equal(v.cpu().numpy(), ref[k]), k
    # a second run on the other staging set with a different event order gives the same
    order = list(reversed(range(len(evs))))
    outs2 = [binding.alloc_outputs(evs[i].n_dirs, evs[i].n_stations, evs[i].n_samples)[0] for i in order]
    plan.run([structs[i] for i in order], outs2)
    torch.cuda.synchronize()
    for i, o in zip(order, outs2):
        for k, v in o.items():
            assert np.array_equal(v.cpu().numpy(), outs[i][k].cpu().numpy()), k
    plan.close()


def test_batch_limits_refused(setup):
    binding, ctx, pat, pid = setup
    ev = synth.make_event(10, 1024, synth.scan_directions(2, 2), seed_key=710)
    inp = _upload(ev)
    plan = ctx.batch(2, 15, 100, 51)
    out, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples)
    with pytest.raises(binding.ArError) as e:
        plan.run([binding.make_event(pid, *inp)] * 2, [out, out])     # 20 stations > 15
    assert e.value.status == 5
    with pytest.raises(binding.ArError) as e:
        plan.run([binding.make_event(pid, *inp)] * 3, [out] * 3)      # 3 events > 2
    assert e.value.status == 5
    plan.close()


def test_uneven_stream_full_size_sampled_against_oracle():
    """The 256-event uneven workload (S 3-124, N 1024/2048/4096, D 16-256), autotuned plan;
    about 2,000 of its 2.2 M pairs against the oracle, spread over the three lengths."""
    from paper_1507_07733_gb300 import binding
    ctx = binding.Context(0, autotune=True)
    pat = synth.make_pattern()
    pid = ctx.load_pattern(pat)
    stream = synth.uneven_stream(256)
    evs = [synth.materialise(d) for d in stream]
    inputs = [_upload(e) for e in evs]
    outs = [binding.alloc_outputs(e.n_dirs, e.n_stations, e.n_samples)[0] for e in evs]
    plan = ctx.batch(256, sum(e.n_stations for e in evs), sum(e.n_dirs for e in evs), 51)
    plan.run([binding.make_event(pid, *inp, e.fs_hz) for e, inp in zip(evs, inputs)], outs)
    torch.cuda.synchronize()
    binding.ar_sync(ctx.h)
    ctas, ms = plan.tuning()
    assert all(c >= 1 for c in ctas) and min(m for m in ms if m > 0) > 0
    info = plan.tuning_info()   # the per-class plan: within each class's limits, no slower than the default
    assert info["tuned"] and info["candidates"] >= 6 and info["ctas_per_sm"] == list(ctas)
    assert all(1 <= c <= m for c, m in zip(info["ctas_per_sm"], info["max_ctas_per_sm"]))
    assert 0 < info["tuned_ms"] <= info["default_ms"]
    # about 2,000 pairs against the oracle, a third per trace length, over 16 events per length
    rng = np.random.default_rng(256)
    checked = 0
    for n in (1024, 2048, 4096):
        cls = [i for i, e in enumerate(evs) if e.n_samples == n]
        pick = rng.choice(cls, min(16, len(cls)), replace=False)
        for ei in pick:
            e, o = evs[ei], outs[ei]
            k = min(e.n_stations * e.n_dirs, -(-667 // len(pick)))
            q = rng.choice(e.n_stations * e.n_dirs, k, replace=False)
            di, si = q // e.n_stations, q % e.n_stations
            ref = oracle.unfold_sample(pat, e, si, di)
            sub = {kk: o[kk].cpu().numpy()[di, si] for kk in ("efield", "envelope", "peak_idx", "peak_amp", "status")}
            check_pairs(sub, ref, e.n_samples)
            check_times(o["peak_time_ns"].cpu().numpy()[di, si], ref["peak_time_ns"], "peak time")
            checked += k
            # two directions' residuals from the batch's own peak times
            pt = o["peak_time_ns"].cpu().numpy()
            res = o["residual_ns"].cpu().numpy()
            for d in rng.choice(e.n_dirs, 2, replace=False):
                r, t0, chi2 = oracle.residual(e.pos_m, pt[d], *e.dirs_rad[d])
                check_times(res[d], r, "residual")
    assert checked >= 1900
    plan.close()
    del outs, inputs
    torch.cuda.empty_cache()
    ctx.close()
