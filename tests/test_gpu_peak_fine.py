"""GPU: sub-sample peak times (a variant; parabolic vertex through the envelope maximum and its
two neighbours) against the oracle.

Bound, derived from the path's envelope bar: with envelope values a, b, c around the peak
known to eta = 1e-5 b each, the vertex offset delta = (a - c) / (2 (a - 2b + c)) moves by at
most 3 eta / |a - 2b + c| (|a - c| <= |a - 2b + c| for a maximum), so the refined times must
agree within that many samples (plus 1e-9 ns of FP64 rounding). Pairs whose peak index is a
tie or whose solve is near the singular threshold are skipped, as in the main parity tests.
With refined times the residual, t0 and chi2 follow them (1e-9 relative, recomputed by the
oracle from the GPU's refined times).
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


def _run(binding, ctx, pid, ev, traces=True, tc_terms=0):
    out, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cuda", traces=traces, fine=True)
    args = (pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad))
    if tc_terms:
        ctx.unfold_tc(*args, split_terms=tc_terms, fs_hz=ev.fs_hz, out=out, sync=True)
    else:
        ctx.unfold(*args, ev.fs_hz, out=out, sync=True)
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def check_fine(gpu, ref, ev):
    D, S, N = ev.n_dirs, ev.n_stations, ev.n_samples
    dt = 1e9 / ev.fs_hz
    want = oracle.fine_peak_times(ref["envelope"], ref["peak_idx"], ev.t_start_ns, ev.fs_hz)
    envr = ref["envelope"]
    checked = 0
    for d in range(D):
        for s in range(S):
            k = int(ref["peak_idx"][d, s])
            if gpu["peak_idx"][d, s] != k or ref["min_margin"][d, s] <= 1e-5:
                continue
            if 0 < k < N - 1:
                second = envr[d, s, k - 1] - 2 * envr[d, s, k] + envr[d, s, k + 1]
                bound = 3 * ETA * envr[d, s, k] / abs(second) if second < 0 else 0.5
            else:
                bound = 0.0
            assert abs(gpu["peak_time_fine_ns"][d, s] - want[d, s]) <= min(bound, 0.5) * dt + 1e-9, (d, s)
            checked += 1
    assert checked >= D * S // 2
    # the residual follows the refined times
    for d in range(D):
        r, t0, chi2 = oracle.residual(ev.pos_m, gpu["peak_time_fine_ns"][d], *ev.dirs_rad[d])
        check_times(gpu["residual_ns"][d], r, "residual at refined times")
        check_times(gpu["t0_ns"][d], t0, "t0 at refined times")
        assert abs(gpu["chi2"][d] - chi2) <= 1e-9 * max(abs(chi2), 1.0)


@pytest.mark.parametrize("n,s,d", [(1024, 13, 5), (2048, 9, 4), (4096, 6, 3)])
def test_refined_peak_times(env, n, s, d):
    binding, ctx, pat, pid = env
    rng = np.random.default_rng(7 * n + s)
    ev = synth.make_event(s, n, synth.random_directions(d, rng), seed_key=1300 + s)
    gpu = _run(binding, ctx, pid, ev)
    ref = oracle.unfold_event(pat, ev)
    check_pairs(gpu, ref, n)
    check_fine(gpu, ref, ev)
    # the refined time lies within half a sample of the sample peak
    dt = 1e9 / ev.fs_hz
    assert np.all(abs(gpu["peak_time_fine_ns"] - gpu["peak_time_ns"]) <= 0.5 * dt + 1e-9)
    # peaks only: the same refined times and timing
    po = _run(binding, ctx, pid, ev, traces=False)
    for k in ("peak_idx", "peak_time_ns", "peak_time_fine_ns", "residual_ns", "t0_ns", "chi2"):
        assert np.array_equal(po[k], gpu[k]), k


def test_refined_times_on_the_tensor_core_and_host_paths(env):
    binding, ctx, pat, pid = env
    ev = synth.single_event(4096)
    ref = oracle.unfold_event(pat, ev)
    tc = _run(binding, ctx, pid, ev, tc_terms=6)
    check_pairs(tc, ref, 4096)
    check_fine(tc, ref, ev)
    dev = _run(binding, ctx, pid, ev)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hout, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cpu", pin_memory=True, fine=True)
    ctx.unfold_host(pid, pin(ev.traces), pin(ev.pos_m), pin(ev.t_start_ns), pin(ev.dirs_rad), ev.fs_hz, out=hout)
    for k, v in hout.items():
        assert np.array_equal(v.numpy(), dev[k]), k
