"""The error path of the unfold kernel's bounded waits, made to run on a GPU without a fault.

ar_set_test_fault(ctx, 1) makes every corner-slab mbarrier of ar_unfold expect 16 bytes more
than its four bulk copies deliver, and shortens the wait limit to 1 ms; the copies are
unchanged and in bounds. Each wait then runs out: the kernel sets bit 0 of the error word,
waits once more (bounded), and its CTAs return; ar_sync reports AR_ERR_DEVICE. The pattern is
small (11 frequency nodes), so the kernel stages its corner slabs in shared memory and does
wait on them. Afterwards the same context unfolds normally and matches the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_event

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL_GRID = dict(synth.PATTERN_GRID, n_freq=11, df_hz=5e6)   # 30-80 MHz in 5 MHz steps


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_a_wait_that_runs_out_is_reported_and_the_context_recovers():
    from paper_1507_07733_gb300 import binding
    pat = synth.make_pattern(grid=SMALL_GRID)
    ctx = binding.Context(0)
    pid = ctx.load_pattern(pat)
    ev = synth.make_event(7, 2048, synth.scan_directions(2, 2), seed_key=41)
    args = (_dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), _dev(ev.dirs_rad))
    binding.ar_set_test_fault(ctx.h, 1)
    with pytest.raises(binding.ArError) as e:
        ctx.unfold(pid, *args, sync=True)
    assert e.value.status == binding.STATUS_NAMES.index("AR_ERR_DEVICE")
    assert "bounded wait" in str(e.value)
    binding.ar_set_test_fault(ctx.h, 0)
    out = ctx.unfold(pid, *args, sync=True)
    gpu = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    check_event(gpu, oracle.unfold_event(pat, ev), ev)
    with pytest.raises(binding.ArError):
        binding.ar_set_test_fault(ctx.h, 2)
    ctx.close()
