#!/usr/bin/env python3
"""Benchmark of the unfolding path: station.direction unfolds per second.

Workload (one step): the 124-station direction scan -- 124 stations x 2 channels x 2048
float32 samples at 200 MHz, 64 candidate directions (zenith 0-60 deg x 8, azimuth 0-315 deg
x 8), the 19 x 72 x 51 synthetic VEL table -- unfolded pair by pair through the C ABI
(ar_unfold: station transform, then the fused unfold with the per-direction residual).
7936 pairs per step.

  value        pairs / s over the K timed steps (device time, CUDA events per step on the
               launching stream, L2 flushed by a 256 MiB write between steps, outside the
               step's events), summed over ranks; max over ranks of the time
  e2e          the same metric through the serving API (ar_submit / ar_wait) with pinned host
               buffers: the inputs' host->device copy, the kernels, and the device->host copy
               of every output inside the timed region (host wall clock; one event's copies
               overlap the next one's kernels); e2e_synchronous through ar_unfold_host
  roofline     the fused unfold kernel: algorithmic bytes per launch / its mean duration
               (CUDA events recorded by the library around it, same stream) vs measured HBM;
               roofline_alu the same duration against the FP32 issue peak
  cpu_baseline the FP64 oracle on a bounded sample of the same workload on the host cores

--impl reference times the oracle alone (each step: one station x 16 directions of the
same workload) and prints the same JSON line with "impl": "reference".

Multi-GPU (torchrun): every rank runs its own replica of the workload ("replicas only":
the pairs are independent and need no exchange); value is all ranks' pairs over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "station-direction unfolds/s (124 st x 2048 samples x 64 dirs, FP32, <=1e-5 rel err)"
UNIT = "unfolds/s"
WORKLOAD = "direction scan: 124 stations x 2 ch x 2048 float32 @ 200 MHz, 64 directions (8 zen 0-60 x 8 az 0-315), 19x72x51 VEL table"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "unfold_kernel_traffic.json")


def kernel_source_hash() -> str:
    """Hash of the unfold kernel's source with comments and blank lines removed, so that the
    recorded ncu traffic stays attached to the code it was measured on across comment edits."""
    h = hashlib.sha256()
    for f in ("kernels.cuh", "dft.cuh"):
        src = open(os.path.join(ROOT, "paper_1507_07733_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        lines = (re.sub(r"//.*", "", ln).rstrip() for ln in src.splitlines())
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


# ---- distributed plumbing ---------------------------------------------------------------

def dist_setup(want_cuda: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if want_cuda else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks -----------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampled every 20 ms in the background; samples keep their host timestamps."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)   # let the first samples arrive

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self, t0: float, t1: float) -> dict:
        rows = []
        for ts, line in self.samples:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((ts, float(p[1]), float(p[2]), p[4], p[5:9]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 <= r[0] <= t1]
        window = "timed region"
        if len(inside) < 3 and rows:   # a short timed region: take the samples nearest to it
            rows.sort(key=lambda r: 0 if t0 <= r[0] <= t1 else min(abs(r[0] - t0), abs(r[0] - t1)))
            inside = rows[:3]
            window = "timed region plus nearest samples"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in inside for n, v in zip(names, r[4]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside), "window": window}


# ---- algorithmic work -----------------------------------------------------------------

def unfold_bytes_per_launch(S: int, D: int, N: int, n_f: int) -> int:
    """Bytes the fused unfold kernel must move: per pair, writes of E-field (8N), envelope (4N),
    peak index/amplitude/time, status and residual (28 B); per station, reads of its band
    spectrum (N/4 bins x 16 B), position and window start (32 B); per direction, reads of its
    four corner slabs (4 x n_f x 32 B) and angles (16 B) and writes of t0 and chi2 (16 B)."""
    return S * D * (12 * N + 28) + S * ((N // 4) * 16 + 32) + D * (4 * n_f * 32 + 32)


def unfold_l2_bytes_per_launch(S: int, D: int, N: int, n_f: int) -> int:
    """Bytes the fused unfold kernel moves through L2: its DRAM bytes, plus the station
    spectrum (N/4 bins x 16 B) read again for every pair (it stays in L2 after the first)."""
    return unfold_bytes_per_launch(S, D, N, n_f) + S * (D - 1) * (N // 4) * 16


def unfold_flops_per_pair(N: int, D: int) -> float:
    """benchFFT convention: two complex N-point inverse transforms (5 N log2 N each), ~16 N for
    solve, envelope and peak, plus the station's forward transform amortised over D."""
    import math
    return 10 * N * math.log2(N) + 16 * N + 5 * N * math.log2(N) / D


# ---- CPU (oracle) sample -------------------------------------------------------------------

def oracle_sample(pat, ev, n_dirs: int = 16, station: int = 0):
    from paper_1507_07733_gb300 import synth
    return synth.Event(ev.traces[station:station + 1], ev.pos_m[station:station + 1],
                       ev.t_start_ns[station:station + 1], ev.dirs_rad[:n_dirs], ev.fs_hz)


def time_oracle(pat, ev, steps: int, warmup: int):
    import oracle
    threads = int(os.environ.get("OMP_NUM_THREADS", "0")) or os.cpu_count() or 1
    oracle.set_threads(threads)
    pairs = 0
    dt = 0.0
    for k in range(warmup + steps):
        sub = oracle_sample(pat, ev, 16, station=k % ev.n_stations)
        t = time.perf_counter()
        oracle.unfold_event(pat, sub)
        el = time.perf_counter() - t
        if k >= warmup:
            dt += el
            pairs += sub.n_stations * sub.n_dirs
    return pairs, dt, threads


def time_oracle_configs(pat):
    """The oracle over whole workloads: the single event (10 x 2048, 1 direction), the same at
    4096 samples, and the whole direction scan (124 x 2048 x 64 directions, 7,936 pairs), each
    once, on all host cores."""
    import oracle
    from paper_1507_07733_gb300 import synth
    threads = int(os.environ.get("OMP_NUM_THREADS", "0")) or os.cpu_count() or 1
    oracle.set_threads(threads)
    out = {}
    for name, ev in (("single_event_10x2048x1", synth.single_event(2048)),
                     ("single_event_10x4096x1", synth.single_event(4096)),
                     ("direction_scan_124x2048x64", synth.direction_scan())):
        t = time.perf_counter()
        oracle.unfold_event(pat, ev)
        el = time.perf_counter() - t
        pairs = ev.n_stations * ev.n_dirs
        out[name] = {"pairs": pairs, "seconds": round(el, 3), "unfolds_per_s": round(pairs / el, 2), "cores": threads}
    return out


# ---- the GPU arm -----------------------------------------------------------------------

def run_gpu(args):
    import torch
    world, rank, local = dist_setup(True)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1507_07733_gb300 import binding, synth

    pat = synth.make_pattern()
    ev = synth.direction_scan()
    S, N, D = ev.n_stations, ev.n_samples, ev.n_dirs
    ctx = binding.Context(local)
    pid = ctx.load_pattern(pat)
    ctx.prepare(N, ev.fs_hz, pid, S)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    tr, pos, ts, dirs = t(ev.traces), t(ev.pos_m), t(ev.t_start_ns), t(ev.dirs_rad)
    out, ost = binding.alloc_outputs(D, S, N, device=dev)
    evs = binding.make_event(pid, tr, pos, ts, dirs, ev.fs_hz, 1.0)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        binding.ar_unfold(ctx.h, evs, ost, sp)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    binding.ar_sync(ctx.h, sp)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    h0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    h1 = time.perf_counter()
    clocks.stop()
    binding.ar_sync(ctx.h, sp)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = allmax(world, sum(step_ms), dev)
    pairs = S * D
    value = pairs * world * args.steps / (total_ms / 1e3)

    # the fused kernel's own duration, from events the library records around it
    binding.ar_set_profiling(ctx.h, True)
    k_ms = []
    for _ in range(min(args.steps, 200)):
        flush.zero_()
        step()
        k_ms.append(binding.ar_kernel_times(ctx.h))
    binding.ar_set_profiling(ctx.h, False)
    binding.ar_sync(ctx.h, sp)
    k3 = statistics.mean(m[1] for m in k_ms)
    k1 = statistics.mean(m[0] for m in k_ms)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    nbytes = unfold_bytes_per_launch(S, D, N, pat.n_freq)
    l2_bytes = unfold_l2_bytes_per_launch(S, D, N, pat.n_freq)
    achieved = nbytes / (k3 / 1e3) / 1e9
    traffic = None
    if os.path.exists(PROFILE_TRAFFIC):
        pt = json.load(open(PROFILE_TRAFFIC))
        if pt.get("kernel_hash") == kernel_source_hash():
            traffic = pt.get("dram_bytes_per_launch")
    sm_clock = 2070e6
    fp32_peak = 152 * 128 * 2 * sm_clock / 1e12   # TFLOP/s, FFMA on every FP32 lane at max clock
    flops = unfold_flops_per_pair(N, D) * pairs
    alu = {"bound": "alu", "achieved": round(flops / (k3 / 1e3) / 1e12, 2), "peak": round(fp32_peak, 1),
           "unit": "TFLOP/s", "frac": round(flops / (k3 / 1e3) / 1e12 / fp32_peak, 3),
           "flops_per_launch": flops, "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}

    # end to end through the host-buffer entry point (pinned host memory both ways)
    e2e = None
    e2e_sync = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        htr, hpos, hts, hdirs = pin(ev.traces), pin(ev.pos_m), pin(ev.t_start_ns), pin(ev.dirs_rad)
        hout, host = binding.alloc_outputs(D, S, N, device="cpu", pin_memory=True)
        hev = binding.make_event(pid, htr, hpos, hts, hdirs, ev.fs_hz, 1.0)
        n_e2e = max(3, min(args.steps, 50))
        for _ in range(2):
            binding.ar_unfold_host(ctx.h, hev, host, sp)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            binding.ar_unfold_host(ctx.h, hev, host, sp)
        el = allmax(world, time.perf_counter() - t0, dev)
        h2d = sum(x.numel() * x.element_size() for x in (htr, hpos, hts, hdirs))
        d2h = sum(v.numel() * v.element_size() for v in hout.values() if v is not None)
        e2e_sync = {"value": round(pairs * world * n_e2e / el, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": n_e2e, "ms_per_step": round(el / n_e2e * 1e3, 4),
                    "api": "ar_unfold_host (synchronous: copies in, unfold, copies out)"}
        # the headline end-to-end figure: a stream of events through the server, each event's
        # inputs copied in from pinned host memory and all its outputs copied back
        e2e = run_e2e_pipelined(binding, ctx, pid, (htr, hpos, hts, hdirs), ev.fs_hz, D, S, N, pairs, n_e2e,
                                world, dev)
        e2e.update({"h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h})

    back_to_back = run_back_to_back(binding, ctx, evs, ost, pairs, stream)
    l2_gbs = measure_l2_gbs(dev)
    peaks_only = run_peaks_only(binding, ctx, pid, (tr, pos, ts, dirs), ev.fs_hz, D, S, N, pairs, flops, fp32_peak,
                                l2_gbs, dev, stream)
    single = run_single_event(binding, synth, ctx, pid, dev, stream)
    recon = run_reconstruction(binding, synth, ctx, pid, dev, stream)
    precision = None
    if rank == 0 and not args.no_cpu_baseline:
        precision = run_precision(binding, synth, ctx, pid, dev, stream)
    tensor_core = run_tensor_core(binding, synth, ctx, pid, dev, stream, peaks)
    mixed = run_mixed_antennas(binding, synth, ctx, dev, stream, peaks.get("hbm_gbs"))
    refine = run_output_variant(binding, synth, ctx, pid, dev, stream, peaks.get("hbm_gbs"), "fine")
    weighted = run_output_variant(binding, synth, ctx, pid, dev, stream, peaks.get("hbm_gbs"), "snr")
    lengths = run_trace_lengths(binding, synth, ctx, pid, dev, stream, peaks.get("hbm_gbs"))

    batched = None
    if not args.no_batch:
        batched = run_batched(args, binding, synth, ctx, pid, dev, stream)

    serving = None
    if not args.no_serve:
        serving = run_serving(args, binding, synth, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle over whole workloads; the whole scan (about 16 s of CPU work on 16 cores)
        # is the baseline
        oc = time_oracle_configs(pat)
        scan = oc["direction_scan_124x2048x64"]
        cpu = {"value": scan["unfolds_per_s"], "unit": UNIT, "cores": scan["cores"], "kind": "oracle",
               "sample": f"the whole workload once: {scan['pairs']} pairs in {scan['seconds']} s, FP64 oracle "
                         f"(naive DFTs), OpenMP over pairs",
               "configs": oc}

    ctx.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "stations": S, "samples": N, "directions": D,
                       "pairs_per_step": pairs, "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (256 MiB write, outside the step events)"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 3), "traffic": traffic, "peak_source": peak_src,
                         "kernel": "unfold_kernel<2048>", "kernel_ms": round(k3, 5),
                         "algorithmic_bytes_per_launch": nbytes,
                         "note": "about 63 MB of each launch's 196.7 MB of outputs are still dirty in L2 when "
                                 "the kernel ends (ncu: 134 MB written to DRAM inside the launch) and are "
                                 "written back during the untimed L2 flush between steps; back-to-back calls "
                                 "without the flush are in back_to_back"},
            "roofline_l2": {"bound": "l2", "achieved": round(l2_bytes / (k3 / 1e3) / 1e9, 1), "peak": l2_gbs,
                            "unit": "GB/s", "frac": round(l2_bytes / (k3 / 1e3) / 1e9 / l2_gbs, 3) if l2_gbs else None,
                            "algorithmic_bytes_per_launch": l2_bytes,
                            "peak_source": "bench's own L2-resident copy rate (a lower bound on L2 bandwidth)"},
            "roofline_alu": alu,
            "kernel_ms": {"station_spectrum": round(k1, 5), "unfold_with_residual": round(k3, 5)},
            "gpu_launches": 2 * args.steps,
            "e2e": e2e,
            "e2e_synchronous": e2e_sync,
            "back_to_back": back_to_back,
            "peaks_only": peaks_only,
            "l2_gbs_measured": l2_gbs,
            "single_event": single,
            "reconstruction": recon,
            "precision": precision,
            "tensor_core_variant": tensor_core,
            "mixed_antennas": mixed,
            "peak_refinement": refine,
            "snr_weighting": weighted,
            "trace_lengths": lengths,
            "batched_uneven": batched,
            "serving": serving,
            "cpu_baseline": cpu,
            "clocks": clocks.summary(h0, h1),
        }
        print(json.dumps(line), flush=True)


def run_single_event(binding, synth, ctx, pid, dev, stream, reps=200):
    """The plain single event (10 stations x 2048 samples, one direction): latency-bound.
    Device time per call (CUDA events around each call), host latency of a synchronous call
    on device buffers, and of ar_unfold_host (copies both ways)."""
    import torch
    ev = synth.single_event(2048)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    keep = (t(ev.traces), t(ev.pos_m), t(ev.t_start_ns), t(ev.dirs_rad))   # the event holds raw pointers
    e = binding.make_event(pid, *keep, ev.fs_hz)
    o, ost = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device=dev)
    sp = stream.cuda_stream
    for _ in range(20):
        binding.ar_unfold(ctx.h, e, ost, sp)
    torch.cuda.synchronize(dev)
    a = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    b = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    for i in range(reps):
        a[i].record(stream)
        binding.ar_unfold(ctx.h, e, ost, sp)
        b[i].record(stream)
    torch.cuda.synchronize(dev)
    dev_us = sorted(x.elapsed_time(y) * 1e3 for x, y in zip(a, b))
    host_us = []
    for _ in range(reps):
        t0 = time.perf_counter()
        binding.ar_unfold(ctx.h, e, ost, sp)
        binding.ar_sync(ctx.h, sp)
        host_us.append((time.perf_counter() - t0) * 1e6)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    hkeep = (pin(ev.traces), pin(ev.pos_m), pin(ev.t_start_ns), pin(ev.dirs_rad))
    he = binding.make_event(pid, *hkeep, ev.fs_hz)
    ho, host_o = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device="cpu", pin_memory=True)
    e2e_us = []
    for _ in range(reps):
        t0 = time.perf_counter()
        binding.ar_unfold_host(ctx.h, he, host_o, sp)
        e2e_us.append((time.perf_counter() - t0) * 1e6)
    host_us.sort()
    e2e_us.sort()
    med = lambda v: round(v[len(v) // 2], 2)
    return {"workload": "10 stations x 2 x 2048 samples, 1 direction (zenith 30, azimuth 45)",
            "device_us_p50": med(dev_us), "device_us_min": round(dev_us[0], 2),
            "host_sync_us_p50": med(host_us), "host_buffers_us_p50": med(e2e_us),
            "host_buffers_us_p99": round(e2e_us[int(0.99 * (len(e2e_us) - 1))], 2),
            "note": "two kernels per call; latency-bound (about 0.25 MB of traffic)"}


def run_reconstruction(binding, synth, ctx, pid, dev, stream, reps=20):
    """The iterative loop on the 124-station event of the scan workload: device time per
    reconstruction, iterations, and the angle between the result and the generator's true
    direction."""
    import math
    import torch
    ev = synth.direction_scan()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    tr, pos, ts = t(ev.traces), t(ev.pos_m), t(ev.t_start_ns)
    r = ctx.reconstruct(pid, tr, pos, ts, ev.fs_hz, max_iter=8, tol_rad=1e-6, stream=stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        r = ctx.reconstruct(pid, tr, pos, ts, ev.fs_hz, max_iter=8, tol_rad=1e-6, stream=stream, sync=False)
    b.record(stream)
    torch.cuda.synchronize(dev)
    d = r["direction"].cpu().numpy()
    zt, at = ev.true_dir
    ang = math.acos(min(1.0, math.sin(d[0]) * math.sin(zt) * math.cos(d[1] - at) + math.cos(d[0]) * math.cos(zt)))
    return {"workload": "124 stations x 2048 samples, max 8 iterations, tol 1e-6 rad",
            "device_ms_per_reconstruction": round(a.elapsed_time(b) / reps, 4),
            "iterations": int(r["iterations"].item()), "angle_to_true_direction_deg": round(math.degrees(ang), 4)}


def _pair_errors(g, ref, n):
    def rel(a, b, m):
        a = np.asarray(a, np.float64).reshape(-1, m)
        b = np.asarray(b, np.float64).reshape(-1, m)
        return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    ef = rel(g["efield"], ref["efield"], 2 * n)
    en = rel(g["envelope"], ref["envelope"], n)
    pa = np.abs(g["peak_amp"].astype(np.float64) - ref["peak_amp"]) / ref["peak_amp"]
    return {"efield_rel_l2_max": float(ef.max()), "efield_rel_l2_median": float(np.median(ef)),
            "envelope_rel_l2_max": float(en.max()), "peak_amp_rel_max": float(pa.max()),
            "peak_idx_equal": int((g["peak_idx"] == ref["peak_idx"]).sum()), "pairs": int(ef.size),
            "residual_abs_max_ns": float(np.abs(g["residual_ns"] - ref["residual_ns"]).max()),
            "chi2_rel": float(np.abs(g["chi2"] - ref["chi2"]).max() / max(float(np.abs(ref["chi2"]).max()), 1.0))}


def run_precision(binding, synth, ctx, pid, dev, stream, reps=50):
    """Precision workload: the single event (10 stations, 1 direction) at 4096 samples
    through the FP32 FFT path and the tensor-core split-BF16 DFT variant (x3, x6), each
    output's error against the FP64 oracle and the device time per call; the FP32 path at
    2048 samples as well."""
    import torch
    import oracle
    pat = synth.make_pattern()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    res = {"workload": "single event: 10 stations x 4096 samples, 1 direction (30, 45 deg)"}
    sp = stream.cuda_stream
    for n in (4096, 2048):
        ev = synth.single_event(n)
        keep = (t(ev.traces), t(ev.pos_m), t(ev.t_start_ns), t(ev.dirs_rad))
        es = binding.make_event(pid, *keep, ev.fs_hz)
        out, ost = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device=dev)
        ref = oracle.unfold_event(pat, ev)
        variants = [("fp32_fft", lambda: binding.ar_unfold(ctx.h, es, ost, sp))]
        if n == 4096:
            variants += [("tc_split_bf16_x3", lambda: binding.ar_unfold_tc(ctx.h, es, ost, 3, sp)),
                         ("tc_split_bf16_x6", lambda: binding.ar_unfold_tc(ctx.h, es, ost, 6, sp))]
        for name, fn in variants:
            fn()
            ctx.sync(stream)
            row = _pair_errors({k: v.cpu().numpy() for k, v in out.items()}, ref, n)
            if n == 4096:   # device time per call: CUDA events around each call, median
                for _ in range(10):
                    fn()
                a = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
                b = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
                for i in range(reps):
                    a[i].record(stream)
                    fn()
                    b[i].record(stream)
                ctx.sync(stream)
                ms = sorted(x.elapsed_time(y) for x, y in zip(a, b))
                row["device_ms_per_call"] = round(ms[len(ms) // 2], 4)
                res[name] = row
            else:
                res[name + "_2048"] = row
    return res


def run_e2e_pipelined(binding, ctx, pid, host_inputs, fs_hz, D, S, N, pairs, n, world, dev, depth=3):
    """End to end through the server API: the scan event submitted n times from pinned host
    buffers with full outputs returned to pinned host buffers (three output sets in rotation,
    at most `depth` requests in flight), so one event's copies overlap the next one's unfold."""
    srv = binding.Server(ctx, max_batch_events=1, max_inflight=2, max_stations_per_event=S)
    hev = binding.make_event(pid, *host_inputs, fs_hz, 1.0)
    outs = [binding.alloc_outputs(D, S, N, device="cpu", pin_memory=True)[0] for _ in range(depth)]
    for o in outs[:2]:   # warm-up
        assert srv.wait(srv.submit(hev, o)) == 0
    barrier(world)
    t0 = time.perf_counter()
    tickets = []
    for i in range(n):
        if i >= depth:
            assert srv.wait(tickets[i - depth]) == 0
        tickets.append(srv.submit(hev, outs[i % depth]))
    for tk in tickets[-depth:]:
        assert srv.wait(tk) == 0
    el = allmax(world, time.perf_counter() - t0, dev)
    for tk in tickets:
        srv.release(tk)
    srv.close()
    return {"value": round(pairs * world * n / el, 1), "unit": UNIT, "steps": n,
            "ms_per_step": round(el / n * 1e3, 4),
            "api": "ar_submit / ar_wait (server: copies of one event overlap the next one's unfold)"}


def measure_l2_gbs(dev, copies=200):
    """L2 bandwidth on this GPU: device copies whose source and destination stay resident in
    L2 (2 x 4, 8 and 16 MiB), replayed from a captured CUDA graph so that the copies run back
    to back; read + write bytes over CUDA-event time, best size and run."""
    import torch
    best = 0.0
    for mib in (4, 8, 16):
        a = torch.empty(mib << 20, dtype=torch.uint8, device=dev).fill_(1)
        b = torch.empty_like(a)
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            b.copy_(a)
        torch.cuda.current_stream(dev).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(copies):
                b.copy_(a)
        g.replay()
        torch.cuda.synchronize(dev)
        for _ in range(3):
            x, y = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x.record()
            g.replay()
            y.record()
            torch.cuda.synchronize(dev)
            best = max(best, 2.0 * a.numel() * copies / (x.elapsed_time(y) * 1e-3) / 1e9)
        del g
    return round(best, 1)


def run_peaks_only(binding, ctx, pid, keep, fs_hz, D, S, N, pairs, flops, fp32_peak, l2_gbs, dev, stream, reps=200):
    """The scan in peaks-only mode (no E-field or envelope written): ALU- and L2-bound, so it
    is reported against the FP32 peak and the measured L2 bandwidth. L2 bytes per pair: the
    station spectrum staged by a bulk copy (4N B) and the 28 B of results."""
    import torch
    es = binding.make_event(pid, *keep, fs_hz, 1.0)
    out, ost = binding.alloc_outputs(D, S, N, device=dev, traces=False)
    sp = stream.cuda_stream
    for _ in range(10):
        binding.ar_unfold(ctx.h, es, ost, sp)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        binding.ar_unfold(ctx.h, es, ost, sp)
    b.record(stream)
    binding.ar_sync(ctx.h, sp)
    s = a.elapsed_time(b) / reps * 1e-3
    l2_bytes = pairs * (4 * N + 28)
    return {"unfolds_per_s": round(pairs / s, 1), "ms_per_call": round(s * 1e3, 4),
            "fp32": {"achieved_tflops": round(flops / s / 1e12, 2), "peak": round(fp32_peak, 1),
                     "frac": round(flops / s / 1e12 / fp32_peak, 3)},
            "l2": {"achieved_gbs": round(l2_bytes / s / 1e9, 1), "peak_measured_gbs": l2_gbs,
                   "frac": round(l2_bytes / s / 1e9 / l2_gbs, 3) if l2_gbs else None},
            "note": "back to back, two kernels per call"}


def run_back_to_back(binding, ctx, es, ost, pairs, stream, reps=200):
    """The scan called back to back on one stream, no L2 flush between calls (a stream of
    events arriving faster than they are processed): device time per call."""
    import torch
    sp = stream.cuda_stream
    for _ in range(10):
        binding.ar_unfold(ctx.h, es, ost, sp)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        binding.ar_unfold(ctx.h, es, ost, sp)
    b.record(stream)
    binding.ar_sync(ctx.h, sp)
    ms = a.elapsed_time(b) / reps
    return {"unfolds_per_s": round(pairs / (ms * 1e-3), 1), "ms_per_call": round(ms, 4), "calls": reps,
            "note": "no L2 flush between calls"}


def run_trace_lengths(binding, synth, ctx, pid, dev, stream, hbm=None, reps=100):
    """The scan's geometry (124 stations x 64 directions) at the other supported trace
    lengths, 1024 and 4096 samples: device time per call back to back, unfolds/s and the
    unfold kernel's HBM fraction (algorithmic bytes over the kernel's CUDA-event time)."""
    import torch
    res = {}
    for n in (1024, 4096):
        ev = synth.direction_scan(n_samples=n)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        keep = (t(ev.traces), t(ev.pos_m), t(ev.t_start_ns), t(ev.dirs_rad))
        es = binding.make_event(pid, *keep, ev.fs_hz)
        out, ost = binding.alloc_outputs(ev.n_dirs, ev.n_stations, n, device=dev)
        fn = lambda: binding.ar_unfold(ctx.h, es, ost, stream.cuda_stream)
        for _ in range(10):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        ctx.sync(stream)
        ms = a.elapsed_time(b) / reps
        binding.ar_set_profiling(ctx.h, 1)
        kk = []
        for _ in range(20):
            fn()
            ctx.sync(stream)
            kk.append(binding.ar_kernel_times(ctx.h)[1])
        binding.ar_set_profiling(ctx.h, 0)
        k_ms = statistics.mean(kk)
        pairs = ev.n_stations * ev.n_dirs
        row = {"unfolds_per_s": round(pairs / (ms * 1e-3), 1), "ms_per_call": round(ms, 4),
               "unfold_kernel_ms": round(k_ms, 4)}
        if hbm:
            nbytes = unfold_bytes_per_launch(ev.n_stations, ev.n_dirs, n, 51)
            row["hbm_frac"] = round(nbytes / (k_ms * 1e-3) / 1e9 / hbm, 3)
        res[str(n)] = row
        del keep, out, ost
    return res


def run_mixed_antennas(binding, synth, ctx, dev, stream, hbm=None, reps=100):
    """Mixed-antenna scan: the scan event with three antenna types (two on the standard grid,
    one on the paper's largest grid) assigned per station, grouped by type and mixed; device
    time per call with CUDA events, in unfolds/s."""
    import torch
    ev = synth.mixed_antenna_scan()
    ids = [ctx.load_pattern(p) for p in synth.mixed_antenna_patterns()]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    args = (ids[0], t(ev.traces), t(ev.pos_m), t(ev.t_start_ns), t(ev.dirs_rad))
    out, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device=dev)
    pairs = ev.n_stations * ev.n_dirs
    res = {"workload": "124 stations x 64 directions x 2048 samples, antenna types 0/1 (19x72x51) and 2 "
                       "(31x48x98, the paper's largest grid)"}
    ost = binding.outputs_struct(out)
    for name, grouped in (("grouped", True), ("mixed", False)):
        types = synth.station_antenna_types(ev.n_stations, sort=grouped)
        sp = t(np.asarray(ids, np.int32)[types])
        es = binding.make_event(*args, ev.fs_hz, 1.0, sp)
        fn = lambda: binding.ar_unfold(ctx.h, es, ost, stream.cuda_stream)
        for _ in range(5):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        ctx.sync(stream)
        ms = a.elapsed_time(b) / reps
        nbytes = unfold_bytes_per_launch(ev.n_stations, ev.n_dirs, ev.n_samples, 98)
        res[name] = {"unfolds_per_s": round(pairs / (ms * 1e-3), 1), "ms_per_call": round(ms, 4),
                     "types": [int((types == k).sum()) for k in range(3)],
                     "hbm_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                     "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 3) if hbm else None}
    return res


def run_output_variant(binding, synth, ctx, pid, dev, stream, hbm=None, variant="fine", reps=100):
    """The scan with a variant output requested, full outputs and peaks only; device time per
    call with CUDA events, in unfolds/s. ``fine``: sub-sample peak times (the residual then
    uses them); ``snr``: pulse SNRs (the residual then weights stations by them)."""
    import torch
    ev = synth.direction_scan()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    args = (pid, t(ev.traces), t(ev.pos_m), t(ev.t_start_ns), t(ev.dirs_rad))
    pairs = ev.n_stations * ev.n_dirs
    what = {"fine": ("parabolic sub-sample peak times", 8), "snr": ("pulse SNR and SNR-weighted residuals", 4)}
    text, extra = what[variant]
    res = {"workload": "124 stations x 64 directions x 2048 samples, " + text}
    es = binding.make_event(*args, ev.fs_hz, 1.0)
    for name, traces in (("full_outputs", True), ("peaks_only", False)):
        out, ost = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device=dev, traces=traces,
                                         **{variant: True})
        fn = lambda: binding.ar_unfold(ctx.h, es, ost, stream.cuda_stream)
        for _ in range(5):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        ctx.sync(stream)
        ms = a.elapsed_time(b) / reps
        row = {"unfolds_per_s": round(pairs / (ms * 1e-3), 1), "ms_per_call": round(ms, 4)}
        if traces and hbm:
            nbytes = unfold_bytes_per_launch(ev.n_stations, ev.n_dirs, ev.n_samples, 51) + extra * pairs
            row.update({"hbm_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                        "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 3)})
        res[name] = row
    return res


def run_tensor_core(binding, synth, ctx, pid, dev, stream, peaks, reps=20):
    """Throughput of the tensor-core variant on the scan workload (124 stations x 64
    directions x 2048 samples): unfolds/s per call, and the inverse GEMM's tensor rate
    (split products counted: 2 x rows x K x 1024 x terms, rows = 2 x pairs x 4) against the
    measured dense BF16 peak."""
    import torch
    ev = synth.direction_scan()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    args = (pid, t(ev.traces), t(ev.pos_m), t(ev.t_start_ns), t(ev.dirs_rad))
    pairs = ev.n_stations * ev.n_dirs
    A = ev.n_samples // 512
    out, _ = binding.alloc_outputs(ev.n_dirs, ev.n_stations, ev.n_samples, device=dev)
    res = {"workload": "124 stations x 64 directions x 2048 samples"}
    peak = peaks.get("bf16_tflops")
    for terms in (3, 6):
        fn = lambda: ctx.unfold_tc(*args, split_terms=terms, fs_hz=ev.fs_hz, out=out, stream=stream)
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        ctx.sync(stream)
        ms = a.elapsed_time(b) / reps
        binding.ar_set_profiling(ctx.h, 1)
        fn()
        ctx.sync(stream)
        kt = binding.ar_kernel_times(ctx.h)
        binding.ar_set_profiling(ctx.h, 0)
        flops = 2.0 * (2 * pairs * A) * 256 * 1024 * terms
        tflops = flops / (kt[1] * 1e-3) / 1e12
        res[f"x{terms}"] = {"unfolds_per_s": round(pairs / (ms * 1e-3), 1), "ms_per_call": round(ms, 4),
                            "inverse_gemm_ms": round(kt[1], 4), "inverse_gemm_tflops": round(tflops, 1),
                            "inverse_gemm_frac_of_measured_bf16": round(tflops / peak, 4) if peak else None}
    return res


def run_batched(args, binding, synth, ctx, pid, dev, stream):
    """The 256-event uneven workload: 256 plain ar_unfold calls vs one batch graph launch
    (autotuned plan), same outputs buffers, device time with CUDA events."""
    import torch
    descs = synth.uneven_stream(256)
    evs = [synth.materialise(d) for d in descs]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    outs = [binding.alloc_outputs(e.n_dirs, e.n_stations, e.n_samples, device=dev)[0] for e in evs]
    keep = [(t(e.traces), t(e.pos_m), t(e.t_start_ns), t(e.dirs_rad)) for e in evs]   # device inputs
    structs = [binding.make_event(pid, *k, e.fs_hz) for k, e in zip(keep, evs)]
    ostructs = [binding.outputs_struct(o) for o in outs]
    pairs = sum(e.n_stations * e.n_dirs for e in evs)
    sp = stream.cuda_stream
    for e in evs:   # tables and workspace for every shape before timing
        ctx.prepare(e.n_samples, e.fs_hz, pid, max(x.n_stations for x in evs))
    reps = max(3, min(args.steps // 100, 10))

    def timed(fn, n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize(dev)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / n

    def plain():
        for es, os_ in zip(structs, ostructs):
            binding.ar_unfold(ctx.h, es, os_, sp)

    plain_ms = timed(plain, reps)
    bctx = binding.Context(dev.index if dev.index is not None else 0, autotune=True)
    bpid = bctx.load_pattern(synth.make_pattern())
    bstructs = [binding.make_event(bpid, *k, e.fs_hz) for k, e in zip(keep, evs)]
    plan = bctx.batch(256, sum(e.n_stations for e in evs), sum(e.n_dirs for e in evs), 51)
    plan.run(bstructs, ostructs)      # first run: autotune
    torch.cuda.synchronize(dev)
    batch_ms = timed(lambda: plan.run(bstructs, ostructs), reps)
    ctas, tune_ms = plan.tuning()
    plan_info = plan.tuning_info()
    binding.ar_sync(ctx.h, sp)
    binding.ar_sync(bctx.h, sp)
    plan.close()
    bctx.close()
    out_bytes = sum(v.numel() * v.element_size() for o in outs for v in o.values() if v is not None)
    del outs, keep
    torch.cuda.empty_cache()
    return {"workload": "256 events: stations U{3..124}, samples {1024, 2048, 4096}, directions U{16..256}",
            "pairs": pairs, "output_bytes": out_bytes, "reps": reps,
            "plain_ms": round(plain_ms, 3), "plain_unfolds_per_s": round(pairs / plain_ms * 1e3, 1),
            "batched_ms": round(batch_ms, 3), "batched_unfolds_per_s": round(pairs / batch_ms * 1e3, 1),
            "speedup": round(plain_ms / batch_ms, 3), "batched_GBps": round(out_bytes / batch_ms / 1e6, 1),
            "ctas_per_sm": list(ctas), "autotune_graph_ms": [round(x, 3) for x in tune_ms],
            "plan_per_class": {"classes": ["1024", "2048", "4096"], **plan_info}}


def run_serving(args, binding, synth, dev):
    """The continuous-batching server against the plain one (one event per launch, one in
    flight) on streams of the uneven size distribution, in two output modes:
      peaks  peaks, residuals, t0, chi2 and status returned to pinned host buffers;
      full   the E-field and envelope traces as well (on average about 240 MB per event, so
             the device-to-host link, about 190 GB/s, bounds throughput near 800 events/s).
    Per mode: Poisson arrivals at offered rates, each run for min(5 s of arrivals, 5,000
    events) -- so at least 5 s or 5,000 events -- and a closed loop that keeps `depth` requests
    outstanding for 5 s, which measures each server's ceiling. Latency runs from the scheduled
    arrival (closed loop: the submit stamp) to the server's completion stamp, same clock."""
    import torch
    ctx = binding.Context(dev.index if dev.index is not None else 0)
    pid = ctx.load_pattern(synth.make_pattern())
    pool = [synth.materialise(d) for d in synth.uneven_stream(64, seed_key=9)]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    keep = [tuple(pin(a) for a in (e.traces, e.pos_m, e.t_start_ns, e.dirs_rad)) for e in pool]
    evs = [binding.make_event(pid, *k, e.fs_hz) for k, e in zip(keep, pool)]
    pairs_of = [e.n_stations * e.n_dirs for e in pool]
    smax, dmax = 124, 256

    def peak_slots(R):
        slots = []
        for _ in range(R):
            o = {"efield": None, "envelope": None,
                 "peak_idx": torch.empty(dmax * smax, dtype=torch.int32).pin_memory(),
                 "peak_amp": torch.empty(dmax * smax, dtype=torch.float32).pin_memory(),
                 "peak_time_ns": torch.empty(dmax * smax, dtype=torch.float64).pin_memory(),
                 "residual_ns": torch.empty(dmax * smax, dtype=torch.float64).pin_memory(),
                 "t0_ns": torch.empty(dmax, dtype=torch.float64).pin_memory(),
                 "chi2": torch.empty(dmax, dtype=torch.float64).pin_memory(),
                 "status": torch.empty(dmax * smax, dtype=torch.int32).pin_memory()}
            s = binding.outputs_struct(o)
            s._t = o
            slots.append(s)
        return slots

    # full outputs: one pinned output set per pool event (the events up to ~12 GB of outputs)
    full_n = 0
    full_bytes = 0
    for e in pool:
        b = e.n_dirs * e.n_stations * (12 * e.n_samples + 40)
        if full_bytes + b > (12 << 30):
            break
        full_bytes += b
        full_n += 1
    result = {"event_pool": "64 events of the uneven distribution (S U{3..124}, N {1024,2048,4096}, D U{16..256})",
              "state_budget_bytes": 4 << 30, "modes": {}}
    modes = {
        "peaks": dict(desc="peaks, residuals, t0, chi2, status returned to pinned host buffers",
                      rates=[200, 1000, 5000, 20000, 50000], n_pool=len(pool)),
        "full": dict(desc=f"E-field and envelope returned as well (the first {full_n} pool events, "
                          f"{full_bytes / 2**30:.1f} GiB of pinned outputs, {full_bytes / max(full_n, 1) / 1e6:.0f} MB "
                          "per event on average)",
                     rates=[100, 300, 600], n_pool=full_n),
    }
    for mode, spec in modes.items():
        n_pool = spec["n_pool"]
        if mode == "peaks":
            R = 256
            slots = peak_slots(R)
            slot_of = lambda i: i % R
        else:
            R = n_pool
            slots = [binding.alloc_outputs(pool[k].n_dirs, pool[k].n_stations, pool[k].n_samples, device="cpu",
                                           pin_memory=True)[1] for k in range(n_pool)]
            slot_of = lambda i: i % n_pool
        mres = {"mode": spec["desc"], "rates": {}, "closed_loop": {}}
        for kind, cfg in (("batched", dict(max_batch_events=32, max_inflight=2)),
                          ("plain", dict(max_batch_events=1, max_inflight=1))):
            srv = binding.Server(ctx, state_budget_bytes=4 << 30, max_stations_per_event=124, max_n_freq=51, **cfg)
            warm = [srv.submit(evs[i], slots[slot_of(i)]) for i in range(n_pool)]   # tables, graphs
            for t in warm:
                srv.wait(t)
                srv.release(t)

            def stream(n, arrival):
                """Submit n requests (arrival(i) -> absolute target time or None), return stats."""
                owner = [None] * R
                tickets = []
                pairs = 0
                t0 = time.perf_counter()
                for i in range(n):
                    target = arrival(i, t0)
                    if target is not None:
                        while time.perf_counter() < target:
                            pass
                    j = slot_of(i)
                    if owner[j] is not None:
                        srv.wait(owner[j])
                    k = i % n_pool
                    tk = srv.submit(evs[k], slots[j])
                    owner[j] = tk
                    tickets.append((tk, target))
                    pairs += pairs_of[k]
                lat, last = [], 0.0
                for tk, target in tickets:
                    srv.wait(tk, 600000)
                    _, sub, done = srv.times(tk)
                    lat.append(done / 1e9 - (target if target is not None else sub / 1e9))
                    last = max(last, done / 1e9)
                    srv.release(tk)
                span = last - t0
                lat_ms = np.array(lat) * 1e3
                return {"events": n, "seconds": round(span, 3), "throughput_events_per_s": round(n / span, 1),
                        "unfolds_per_s": round(pairs / span, 1),
                        "p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                        "p99_ms": round(float(np.percentile(lat_ms, 99)), 3)}

            for lam in spec["rates"]:
                n = int(min(5000, 5 * lam))
                arr = synth.poisson_arrivals(lam, n, seed_key=lam)
                r = stream(n, lambda i, t0: t0 + arr[i])
                r["offered_events_per_s"] = lam
                mres["rates"].setdefault(str(lam), {})[kind] = r
            # closed loop: `depth` requests outstanding, for 5 s
            depth = min(R, 64)
            owner = [None] * R
            done_n, pairs, lat = 0, 0, []
            t0 = time.perf_counter()
            i = 0
            inflight = []
            while time.perf_counter() - t0 < 5.0 or inflight:
                if time.perf_counter() - t0 < 5.0 and len(inflight) < depth:
                    j = slot_of(i)
                    if owner[j] is not None and owner[j] in inflight:
                        pass
                    else:
                        k = i % n_pool
                        tk = srv.submit(evs[k], slots[j])
                        owner[j] = tk
                        inflight.append(tk)
                        pairs += pairs_of[k]
                        i += 1
                        continue
                tk = inflight.pop(0)
                srv.wait(tk, 600000)
                _, sub, done = srv.times(tk)
                lat.append((done - sub) / 1e6)
                srv.release(tk)
                done_n += 1
            span = time.perf_counter() - t0
            lat_ms = np.array(lat)
            mres["closed_loop"][kind] = {
                "depth": depth, "events": done_n, "seconds": round(span, 3),
                "throughput_events_per_s": round(done_n / span, 1), "unfolds_per_s": round(pairs / span, 1),
                "p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                "p99_ms": round(float(np.percentile(lat_ms, 99)), 3)}
            srv.close()
        result["modes"][mode] = mres
        del slots
    ctx.close()
    return result


# ---- the reference arm (the oracle, on the host cores) ---------------------------------

def run_reference(args):
    world, rank, _ = dist_setup(False)
    if rank != 0:
        return
    from paper_1507_07733_gb300 import synth
    pat = synth.make_pattern()
    ev = synth.direction_scan()
    pairs, dt, threads = time_oracle(pat, ev, steps=args.steps, warmup=args.warmup)
    value = pairs / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "stations": ev.n_stations, "samples": ev.n_samples,
                   "directions": ev.n_dirs, "sample_per_step": "1 station x 16 directions"},
        "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps x (1 station x 16 directions), FP64 oracle, "
                                   f"OpenMP over pairs"},
        "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--cpu-steps", type=int, default=40, help="oracle sample steps for cpu_baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-event batched-vs-plain comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the Poisson serving comparison")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
