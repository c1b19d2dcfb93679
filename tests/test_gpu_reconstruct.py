"""GPU: the iterative reconstruction (Sec. 2) against the oracle's loop.

Same number of iterations, the same direction after every fit (1e-9 rad: both sides fit in
FP64 from the same integer peak indices), the same final t0 and chi2, and the last unfold's
outputs within the parity bar. A degenerate geometry gives no direction on both sides."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_07733_gb300 import synth
from parity_util import check_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def env():
    from paper_1507_07733_gb300 import binding
    ctx = binding.Context(0)
    pat = synth.make_pattern()
    pid = ctx.load_pattern(pat)
    yield ctx, pat, pid
    ctx.close()


@pytest.mark.parametrize("s,n,key", [(40, 2048, 71), (20, 1024, 72), (60, 4096, 73), (124, 2048, 74)])
def test_reconstruct_matches_oracle(env, s, n, key):
    ctx, pat, pid = env
    ev = synth.make_event(s, n, synth.scan_directions(1, 1), seed_key=key)
    g = ctx.reconstruct(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), max_iter=8, tol_rad=1e-6)
    r = oracle.reconstruct(pat, ev, max_iter=8, tol_rad=1e-6)
    it = int(g["iterations"].item())
    assert it == r["iterations"]
    hist = g["history"].cpu().numpy()
    ok = ~np.isnan(r["history"][:, 0])
    assert np.array_equal(~np.isnan(hist[:, 0]), ok)
    assert np.max(np.abs(hist[ok] - r["history"][ok])) <= 1e-9
    d = g["direction"].cpu().numpy()
    assert abs(d[0] - r["zenith"]) <= 1e-9 and abs(d[1] - r["azimuth"]) <= 1e-9
    assert abs(g["t0_ns"].item() - r["t0_ns"]) <= 1e-9 * max(1.0, abs(r["t0_ns"]))
    assert abs(g["chi2"].item() - r["chi2"]) <= 1e-9 * max(1.0, r["chi2"])
    last = {k: v.cpu().numpy()[0] for k, v in g["last"].items() if v is not None and v.dim() > 1}
    ref = dict(efield=r["efield"], envelope=r["envelope"], peak_idx=r["peak_idx"], peak_amp=r["peak_amp"],
               status=r["status"], min_margin=np.ones(s))
    check_pairs({k: last[k] for k in ("efield", "envelope", "peak_idx", "peak_amp", "status")}, ref, n)
    zt, at = ev.true_dir
    ang = math.acos(min(1.0, math.sin(d[0]) * math.sin(zt) * math.cos(d[1] - at) + math.cos(d[0]) * math.cos(zt)))
    assert ang < math.radians(2.0)


def test_reconstruct_degenerate_geometry(env):
    ctx, pat, pid = env
    ev = synth.make_event(5, 1024, synth.scan_directions(1, 1), seed_key=75)
    ev.pos_m[:, 1] = 0.0
    ev.pos_m[:, 2] = 0.0
    ev.pos_m[:, 0] = np.arange(5) * 100.0                 # collinear stations
    g = ctx.reconstruct(pid, _dev(ev.traces), _dev(ev.pos_m), _dev(ev.t_start_ns), max_iter=4)
    r = oracle.reconstruct(pat, ev, max_iter=4)
    assert int(g["iterations"].item()) == -1 == r["iterations"]
    assert np.all(np.isnan(g["direction"].cpu().numpy()))
