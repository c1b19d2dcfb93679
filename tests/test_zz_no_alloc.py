"""ar_unfold_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a real-time acquisition loop whose device memory map is fixed after start-up,
a plug-in inside another program's CUDA context) get the same unfolding from a fixed scratch
array inside the library. This test calls it through the C ABI three times in a row, on
events of different shapes and sampling rates, and compares each result with ar_unfold's on the same inputs, within the
tolerances of the parity tests. It also checks that an event beyond the scratch limit is
refused with a message. Collected last (file name) so that a failure here stops a -x run only
after every other test has run; it needs nothing from the other tests.
"""
import numpy as np
import pytest

from paper_1507_07733_gb300 import synth

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
    assert _rel_l2(got["efield"], ref["efield"], 2 * n).max() <= REL_L2
    assert _rel_l2(got["envelope"], ref["envelope"], n).max() <= REL_L2
    gi, ri = got["peak_idx"].reshape(-1), ref["peak_idx"].reshape(-1)
    env = ref["envelope"].reshape(gi.size, n).astype(np.float64)
    for q in np.flatnonzero(gi != ri):   # only ties at FP32 resolution may differ
        assert abs(env[q, gi[q]] - env[q, ri[q]]) <= TIE * env[q, ri[q]]
    assert np.allclose(got["peak_amp"], ref["peak_amp"], rtol=REL_L2, atol=0)
    assert np.array_equal(got["status"], ref["status"])
    if np.array_equal(gi, ri):
        for k in ("peak_time_ns", "residual_ns", "t0_ns"):
            assert np.all(abs(got[k] - ref[k]) <= 1e-9 * np.maximum(abs(ref[k]), 1.0)), k
        assert np.all(abs(got["chi2"] - ref["chi2"]) <= 1e-9 * np.maximum(ref["chi2"], 1.0))


def test_noalloc_matches_ar_unfold_on_two_calls_in_a_row():
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
    got_all = []
    for ev in events:                  # two calls in a row on the shared scratch array
        tr, pos, ts, dirs = _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad)
        out, st = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples)
        binding.ar_unfold_noalloc(pat.desc(), table.data_ptr(), binding.make_event(-1, tr, pos, ts, dirs, ev.fs_hz),
                                  st, stream.cuda_stream)
        got_all.append(out)
    torch.cuda.synchronize()
    for ev, out in zip(events, got_all):
        got = {k: v.cpu().numpy() for k, v in out.items()}
        ref = {k: v.cpu().numpy() for k, v in ctx.unfold(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns),
                                                         _dev(ev.dirs_rad), fs_hz=ev.fs_hz, sync=True).items()}
        _compare(got, ref, ev.n_samples)
    ctx.close()


def test_noalloc_refuses_events_beyond_its_scratch():
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
