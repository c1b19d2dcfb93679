"""ar_unfold_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a real-time acquisition loop whose device memory map is fixed after start-up,
a plug-in inside another program's CUDA context) get the same unfolding from a fixed scratch
array inside the library. The tests call it through the C ABI:
- three calls in a row on the shared scratch array, events of different shapes and sampling
  rates, each result compared with ar_unfold's on the same inputs and with the FP64 oracle,
  within the tolerances of the parity tests (tests/parity_util.py);
- the scratch array's limits: 240 stations x 4096 samples (the most station-samples) and
  4096 directions, compared with ar_unfold;
- refusals: an event beyond the scratch, and the descriptor and event checks that ar_unfold
  makes (a non-finite azimuth origin, a negative refractive index), each with a message.
Collected last (file name) so that a failure here stops a -x run only after every other test
has run; it needs nothing from the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_event

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL_L2 = 1e-5
TIE = 1e-6


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel_l2(a, b, n):
    a = a.astype(np.float64).reshape(-1, n)
    b = b.astype(np.float64).reshape(-1, n)
    nb = np.linalg.norm(b, axis=1)
    return np.linalg.norm(a - b, axis=1) / np.where(nb > 0, nb, 1.0)


def _compare(got, ref, n):
    """The allocation-free result against ar_unfold's, at the parity tolerances."""
    assert _rel_l2(got["efield"], ref["efield"], 2 * n).max() <= REL_L2
    assert _rel_l2(got["envelope"], ref["envelope"], n).max() <= REL_L2
    gi, ri = got["peak_idx"].reshape(-1), ref["peak_idx"].reshape(-1)
    env = ref["envelope"].reshape(gi.size, n).astype(np.float64)
    for q in np.flatnonzero(gi != ri):   # only neighbours that tie at FP32 resolution may differ
        assert abs(int(gi[q]) - int(ri[q])) == 1
        assert abs(env[q, gi[q]] - env[q, ri[q]]) <= TIE * env[q, ri[q]]
    assert np.allclose(got["peak_amp"], ref["peak_amp"], rtol=REL_L2, atol=0)
    assert np.array_equal(got["status"], ref["status"])
    if np.array_equal(gi, ri):
        for k in ("peak_time_ns", "residual_ns", "t0_ns"):
            assert np.all(abs(got[k] - ref[k]) <= 1e-9 * np.maximum(abs(ref[k]), 1.0)), k
        assert np.all(abs(got["chi2"] - ref["chi2"]) <= 1e-9 * np.maximum(ref["chi2"], 1.0))


def _noalloc(binding, pat, table, ev, stream):
    tr, pos, ts, dirs = _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad)
    out, st = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples)
    keep = (tr, pos, ts, dirs)   # the inputs stay alive until the call has run
    binding.ar_unfold_noalloc(pat.desc(), table.data_ptr(), binding.make_event(-1, tr, pos, ts, dirs, ev.fs_hz),
                              st, stream.cuda_stream)
    return out, keep


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


def test_noalloc_matches_ar_unfold_and_the_oracle_on_three_calls_in_a_row():
    from paper_1507_07733_gb300 import binding
    pat = synth.make_pattern()
    ctx = binding.Context(0)
    pid = ctx.load_pattern(pat)
    table = _dev(pat.table)            # the caller's own device copy of the VEL table
    rng = np.random.default_rng(99)
    events = [synth.make_event(9, 2048, synth.random_directions(5, rng), seed_key=91),
              synth.make_event(4, 1024, synth.random_directions(3, rng), seed_key=92),
              # 227 MHz: the band starts at k_lo = 271, 15 mod 16 (the device-built twiddles)
              synth.make_event(5, 2048, synth.random_directions(3, rng), seed_key=93, fs_hz=227e6)]
    stream = torch.cuda.current_stream()
    runs = [_noalloc(binding, pat, table, ev, stream) for ev in events]   # back to back, one scratch
    torch.cuda.synchronize()
    for ev, (out, _) in zip(events, runs):
        got = _host(out)
        ref = _host(ctx.unfold(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad),
                               fs_hz=ev.fs_hz, sync=True))
        _compare(got, ref, ev.n_samples)
        # and directly against the oracle: the tables this entry point builds on the device
        # (twiddles, frequency cells) are checked by their results, not by ar_unfold's
        check_event(got, oracle.unfold_event(pat, ev), ev)
    ctx.close()


@pytest.mark.parametrize("s,n,d", [(240, 4096, 1), (3, 1024, 4096)])
def test_noalloc_at_its_limits(s, n, d):
    """The most station-samples (240 x 4096 = 983,040) and the most directions (4096)."""
    from paper_1507_07733_gb300 import binding
    pat = synth.make_pattern()
    ctx = binding.Context(0)
    pid = ctx.load_pattern(pat)
    table = _dev(pat.table)
    rng = np.random.default_rng(s + d)
    dirs = synth.random_directions(d, rng)
    if s <= 124:
        ev = synth.make_event(s, n, dirs, seed_key=s + n)
    else:   # more stations than the synthetic array: two halves side by side, the second 3 km east
        a = synth.make_event(s // 2, n, dirs, seed_key=s + n)
        b = synth.make_event(s - s // 2, n, dirs, seed_key=s + n + 1)
        ev = synth.Event(np.concatenate([a.traces, b.traces]), np.concatenate([a.pos_m, b.pos_m + [3000.0, 0.0, 0.0]]),
                         np.concatenate([a.t_start_ns, b.t_start_ns]), dirs, a.fs_hz)
    out, keep = _noalloc(binding, pat, table, ev, torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = _host(out)
    ref = _host(ctx.unfold(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad),
                           fs_hz=ev.fs_hz, sync=True))
    _compare(got, ref, n)
    ctx.close()


def test_noalloc_refuses_events_beyond_its_scratch_and_bad_arguments():
    from paper_1507_07733_gb300 import binding
    pat = synth.make_pattern()
    table = _dev(pat.table)
    S, N, D = 241, 4096, 1              # 241 x 4096 > 983,040 stations x samples
    tr = torch.zeros((S, 2, N), dtype=torch.float32, device="cuda")
    pos = torch.zeros((S, 3), dtype=torch.float64, device="cuda")
    ts = torch.zeros((S,), dtype=torch.float64, device="cuda")
    dirs = torch.zeros((D, 2), dtype=torch.float64, device="cuda")
    out, st = binding.alloc_outputs(D, S, N)
    with pytest.raises(binding.ArError) as e:
        binding.ar_unfold_noalloc(pat.desc(), table.data_ptr(), binding.make_event(-1, tr, pos, ts, dirs), st)
    assert e.value.status == 1 and "983040" in str(e.value)
    # the checks ar_load_pattern and ar_unfold make hold here too
    ok = synth.make_event(3, 2048, synth.scan_directions(1, 1), seed_key=5)
    tr3, pos3, ts3, dirs3 = _dev(ok.traces), _dev(ok.pos_m), _dev(ok.t_start_ns), _dev(ok.dirs_rad)
    out3, st3 = binding.alloc_outputs(1, 3, 2048)
    bad = pat.desc()
    bad["az0_rad"] = float("nan")
    with pytest.raises(binding.ArError) as e:
        binding.ar_unfold_noalloc(bad, table.data_ptr(), binding.make_event(-1, tr3, pos3, ts3, dirs3), st3)
    assert e.value.status == 1 and "finite" in str(e.value)
    with pytest.raises(binding.ArError) as e:
        binding.ar_unfold_noalloc(pat.desc(), table.data_ptr(),
                                  binding.make_event(-1, tr3, pos3, ts3, dirs3, 200e6, -1.0), st3)
    assert e.value.status == 1 and "refractive_index" in str(e.value)
