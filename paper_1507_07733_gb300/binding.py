"""Thin ctypes binding of ``libaerafold.so`` (the C ABI of include/aerafold.h).

Argument marshalling only: every step of the unfolding runs in the library's CUDA kernels.
Function names match the C ABI (``ar_create``, ``ar_load_pattern``, ``ar_unfold``, ...).
``Context`` wraps them for PyTorch users: tensors supply device memory and streams, and
are passed to the library as raw pointers.

Loading fails loudly (``LibraryMissing``) when the library has not been built: there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libaerafold.so")

AR_OK = 0
STATUS_NAMES = ["AR_OK", "AR_ERR_INVALID_ARG", "AR_ERR_UNSUPPORTED_N", "AR_ERR_NO_PATTERN",
                "AR_ERR_OUT_OF_MEMORY", "AR_ERR_BUDGET", "AR_ERR_CUDA", "AR_ERR_TIMEOUT",
                "AR_ERR_NOT_READY", "AR_ERR_DEVICE"]
AR_ERR_TIMEOUT = STATUS_NAMES.index("AR_ERR_TIMEOUT")
AR_ERR_NOT_READY = STATUS_NAMES.index("AR_ERR_NOT_READY")
AR_STATUS_SINGULAR = 1
AR_STATUS_ZEN_CLAMP = 2
AR_STATUS_BAD_DIR = 4
AR_STATUS_BAD_PATTERN = 8

#: every symbol include/aerafold.h declares
EXPORTED = ["ar_create", "ar_destroy", "ar_last_error", "ar_status_string", "ar_load_pattern",
            "ar_prepare", "ar_unfold", "ar_sync", "ar_unfold_host", "ar_set_profiling", "ar_kernel_times",
            "ar_set_test_fault",
            "ar_unfold_noalloc", "ar_batch_create", "ar_batch_run", "ar_batch_tuning", "ar_batch_tuning_info",
            "ar_batch_destroy",
            "ar_server_create", "ar_submit", "ar_poll", "ar_wait", "ar_ticket_times", "ar_ticket_release",
            "ar_server_destroy", "ar_reconstruct", "ar_unfold_tc"]


class LibraryMissing(RuntimeError):
    pass


class ArError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class ar_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("state_budget_bytes", ctypes.c_uint64)]


class ar_pattern_desc(ctypes.Structure):
    _fields_ = [("n_zen", ctypes.c_int32), ("zen0_rad", ctypes.c_double), ("dzen_rad", ctypes.c_double),
                ("n_az", ctypes.c_int32), ("az0_rad", ctypes.c_double), ("daz_rad", ctypes.c_double),
                ("n_freq", ctypes.c_int32), ("f0_hz", ctypes.c_double), ("df_hz", ctypes.c_double)]


class ar_event(ctypes.Structure):
    _fields_ = [("n_stations", ctypes.c_int32), ("n_samples", ctypes.c_int32), ("n_dirs", ctypes.c_int32),
                ("pattern_id", ctypes.c_int32), ("fs_hz", ctypes.c_double),
                ("refractive_index", ctypes.c_double), ("traces", ctypes.c_void_p),
                ("pos_m", ctypes.c_void_p), ("t_start_ns", ctypes.c_void_p), ("dirs_rad", ctypes.c_void_p),
                ("station_pattern", ctypes.c_void_p)]


class ar_batch_limits(ctypes.Structure):
    _fields_ = [("max_events", ctypes.c_int32), ("max_stations", ctypes.c_int32), ("max_dirs", ctypes.c_int32),
                ("max_n_freq", ctypes.c_int32)]


class ar_batch_plan_info(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32 * 3), ("slabs_staged", ctypes.c_int32 * 3),
                ("max_ctas_per_sm", ctypes.c_int32 * 3), ("tuned", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("default_ms", ctypes.c_float), ("tuned_ms", ctypes.c_float)]


class ar_outputs(ctypes.Structure):
    _fields_ = [("efield", ctypes.c_void_p), ("envelope", ctypes.c_void_p), ("peak_idx", ctypes.c_void_p),
                ("peak_amp", ctypes.c_void_p), ("peak_time_ns", ctypes.c_void_p),
                ("residual_ns", ctypes.c_void_p), ("t0_ns", ctypes.c_void_p), ("chi2", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("peak_time_fine_ns", ctypes.c_void_p), ("snr", ctypes.c_void_p)]


class ar_recon_out(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_void_p), ("t0_ns", ctypes.c_void_p), ("chi2", ctypes.c_void_p),
                ("iterations", ctypes.c_void_p), ("history", ctypes.c_void_p), ("last", ar_outputs)]


class ar_server_config(ctypes.Structure):
    _fields_ = [("state_budget_bytes", ctypes.c_uint64), ("max_batch_events", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("max_stations_per_event", ctypes.c_int32),
                ("max_n_freq", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load the library once; raises ``LibraryMissing`` if it is not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # AERAFOLD_LIB selects another build of the library (the debug build in the tests)
        p = path or os.environ.get("AERAFOLD_LIB") or LIB_PATH
        if not os.path.exists(p):
            raise LibraryMissing(f"{p} not found: build it with __graft_entry__.build()")
        L = ctypes.CDLL(p)
        vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        L.ar_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ar_config)]
        L.ar_destroy.argtypes = [vp]
        L.ar_last_error.argtypes = [vp]
        L.ar_last_error.restype = ctypes.c_char_p
        L.ar_status_string.argtypes = [ctypes.c_int]
        L.ar_status_string.restype = ctypes.c_char_p
        L.ar_load_pattern.argtypes = [vp, ctypes.POINTER(ar_pattern_desc), vp, ctypes.POINTER(i32)]
        L.ar_prepare.argtypes = [vp, i32, dbl, i32, i32]
        L.ar_unfold.argtypes = [vp, ctypes.POINTER(ar_event), ctypes.POINTER(ar_outputs), vp]
        L.ar_unfold_tc.argtypes = [vp, ctypes.POINTER(ar_event), ctypes.POINTER(ar_outputs), ctypes.c_int32, vp]
        L.ar_sync.argtypes = [vp, vp]
        L.ar_unfold_host.argtypes = [vp, ctypes.POINTER(ar_event), ctypes.POINTER(ar_outputs), vp]
        L.ar_set_profiling.argtypes = [vp, i32]
        L.ar_set_test_fault.argtypes = [vp, i32]
        L.ar_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        L.ar_batch_create.argtypes = [vp, ctypes.POINTER(ar_batch_limits), ctypes.POINTER(vp)]
        L.ar_batch_run.argtypes = [vp, vp, vp, i32, vp]
        L.ar_batch_tuning.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]
        L.ar_batch_tuning_info.argtypes = [vp, ctypes.POINTER(ar_batch_plan_info)]
        L.ar_batch_destroy.argtypes = [vp]
        u64, i64 = ctypes.c_uint64, ctypes.c_int64
        L.ar_server_create.argtypes = [vp, ctypes.POINTER(ar_server_config), ctypes.POINTER(vp)]
        L.ar_submit.argtypes = [vp, ctypes.POINTER(ar_event), ctypes.POINTER(ar_outputs), ctypes.POINTER(u64)]
        L.ar_poll.argtypes = [vp, u64]
        L.ar_wait.argtypes = [vp, u64, i32]
        L.ar_ticket_times.argtypes = [vp, u64, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.ar_ticket_release.argtypes = [vp, u64]
        L.ar_server_destroy.argtypes = [vp]
        L.ar_reconstruct.argtypes = [vp, ctypes.POINTER(ar_event), i32, dbl, ctypes.POINTER(ar_recon_out), vp]
        L.ar_unfold_noalloc.argtypes = [ctypes.POINTER(ar_pattern_desc), vp, ctypes.POINTER(ar_event),
                                        ctypes.POINTER(ar_outputs), vp]
        for name in EXPORTED:
            if name not in ("ar_last_error", "ar_status_string"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


# ---- raw C-ABI wrappers (same names) ---------------------------------------------------

def _check(ctx, st):
    if st != AR_OK:
        msg = load().ar_last_error(ctx).decode()
        raise ArError(st, msg)


def ar_create(device: int = 0, autotune: bool = False, state_budget_bytes: int = 0):
    L = load()
    h = ctypes.c_void_p()
    cfg = ar_config(device, int(autotune), state_budget_bytes)
    _check(None, L.ar_create(ctypes.byref(h), ctypes.byref(cfg)))
    return h


def ar_destroy(ctx) -> None:
    load().ar_destroy(ctx)


def ar_last_error(ctx) -> str:
    return load().ar_last_error(ctx).decode()


def ar_status_string(st: int) -> str:
    return load().ar_status_string(st).decode()


def ar_load_pattern(ctx, pattern) -> int:
    """``pattern`` has ``desc()`` (axes) and ``table`` ([nz][na][nf][2][2] complex64)."""
    d = ar_pattern_desc(**pattern.desc())
    tab = np.ascontiguousarray(pattern.table, dtype=np.complex64)
    pid = ctypes.c_int32()
    _check(ctx, load().ar_load_pattern(ctx, ctypes.byref(d), tab.ctypes.data, ctypes.byref(pid)))
    return pid.value


def ar_prepare(ctx, n_samples: int, fs_hz: float, pattern_id: int, max_stations: int) -> None:
    _check(ctx, load().ar_prepare(ctx, n_samples, fs_hz, pattern_id, max_stations))


def ar_unfold(ctx, ev: ar_event, out: ar_outputs, stream: int = 0) -> None:
    _check(ctx, load().ar_unfold(ctx, ctypes.byref(ev), ctypes.byref(out), ctypes.c_void_p(stream)))


def ar_unfold_tc(ctx, ev: ar_event, out: ar_outputs, split_terms: int = 3, stream: int = 0) -> None:
    _check(ctx, load().ar_unfold_tc(ctx, ctypes.byref(ev), ctypes.byref(out), int(split_terms),
                                    ctypes.c_void_p(stream)))


def ar_set_test_fault(ctx, mode: int) -> None:
    """Test of the bounded-wait error path (see include/aerafold.h)."""
    _check(ctx, load().ar_set_test_fault(ctx, int(mode)))


def ar_sync(ctx, stream: int = 0) -> None:
    _check(ctx, load().ar_sync(ctx, ctypes.c_void_p(stream)))


def ar_unfold_host(ctx, ev: ar_event, out: ar_outputs, stream: int = 0) -> None:
    _check(ctx, load().ar_unfold_host(ctx, ctypes.byref(ev), ctypes.byref(out), ctypes.c_void_p(stream)))


def ar_set_profiling(ctx, enable: bool) -> None:
    _check(ctx, load().ar_set_profiling(ctx, int(enable)))


def ar_kernel_times(ctx):
    """(spectrum, unfold, residual) durations in ms of the last profiled ar_unfold."""
    ms = (ctypes.c_float * 3)()
    _check(ctx, load().ar_kernel_times(ctx, ms))
    return tuple(ms)


def ar_unfold_noalloc(desc: dict, device_table_ptr: int, ev: ar_event, out: ar_outputs, stream: int = 0) -> None:
    """The allocation-free entry point: ``device_table_ptr`` is the caller's device copy of the
    VEL table; no context is involved."""
    d = ar_pattern_desc(**desc)
    _check(None, load().ar_unfold_noalloc(ctypes.byref(d), ctypes.c_void_p(device_table_ptr), ctypes.byref(ev),
                                          ctypes.byref(out), ctypes.c_void_p(stream)))


def ar_batch_create(ctx, max_events: int, max_stations: int, max_dirs: int, max_n_freq: int = 64):
    h = ctypes.c_void_p()
    lim = ar_batch_limits(max_events, max_stations, max_dirs, max_n_freq)
    _check(ctx, load().ar_batch_create(ctx, ctypes.byref(lim), ctypes.byref(h)))
    return h


def ar_batch_run(ctx, plan, events, outs, stream: int = 0) -> None:
    """``events``/``outs``: sequences of ``ar_event`` / ``ar_outputs`` (device pointers)."""
    n = len(events)
    ev_arr = (ar_event * n)(*events)
    out_arr = (ar_outputs * n)(*outs)
    _check(ctx, load().ar_batch_run(plan, ctypes.cast(ev_arr, ctypes.c_void_p), ctypes.cast(out_arr, ctypes.c_void_p),
                                    n, ctypes.c_void_p(stream)))


def ar_batch_tuning(plan):
    """(CTAs per SM for the 1024/2048/4096 classes, autotuner graph ms for 1..6 CTAs per SM)."""
    c = (ctypes.c_int32 * 3)()
    ms = (ctypes.c_float * 6)()
    st = load().ar_batch_tuning(plan, c, ms)
    if st != AR_OK:
        raise ArError(st, "ar_batch_tuning")
    return tuple(c), tuple(ms)


def ar_batch_tuning_info(h) -> dict:
    """The plan per length class (1024, 2048, 4096 samples) and the autotuner's timings."""
    i = ar_batch_plan_info()
    _check(None, load().ar_batch_tuning_info(h, ctypes.byref(i)))
    return {"ctas_per_sm": list(i.ctas_per_sm), "slabs_staged": list(i.slabs_staged),
            "max_ctas_per_sm": list(i.max_ctas_per_sm), "tuned": bool(i.tuned), "candidates": i.candidates,
            "default_ms": round(i.default_ms, 4), "tuned_ms": round(i.tuned_ms, 4)}


def ar_batch_destroy(plan) -> None:
    load().ar_batch_destroy(plan)


def ar_server_create(ctx, state_budget_bytes: int = 0, max_batch_events: int = 32, max_inflight: int = 2,
                     max_stations_per_event: int = 124, max_n_freq: int = 64):
    h = ctypes.c_void_p()
    cfg = ar_server_config(state_budget_bytes, max_batch_events, max_inflight, max_stations_per_event, max_n_freq)
    _check(ctx, load().ar_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return h


def ar_submit(ctx, server, ev: ar_event, out: ar_outputs) -> int:
    t = ctypes.c_uint64()
    _check(ctx, load().ar_submit(server, ctypes.byref(ev), ctypes.byref(out), ctypes.byref(t)))
    return t.value


def ar_poll(server, ticket: int) -> int:
    """Status code: 0 done, 8 (AR_ERR_NOT_READY) in flight, else the request's error."""
    return load().ar_poll(server, ticket)


def ar_wait(server, ticket: int, timeout_ms: int) -> int:
    return load().ar_wait(server, ticket, timeout_ms)


def ar_ticket_times(server, ticket: int):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    st = load().ar_ticket_times(server, ticket, ctypes.byref(a), ctypes.byref(b))
    return st, a.value, b.value


def ar_ticket_release(server, ticket: int) -> int:
    return load().ar_ticket_release(server, ticket)


def ar_server_destroy(server) -> None:
    load().ar_server_destroy(server)


def ar_reconstruct(ctx, ev: ar_event, max_iter: int, tol_rad: float, out: ar_recon_out, stream: int = 0) -> None:
    _check(ctx, load().ar_reconstruct(ctx, ctypes.byref(ev), max_iter, tol_rad, ctypes.byref(out),
                                      ctypes.c_void_p(stream)))


# ---- PyTorch-facing helpers ----------------------------------------------------------

def _ptr(t):
    return None if t is None else t.data_ptr()


def make_event(pattern_id: int, traces, pos_m, t_start_ns, dirs_rad, fs_hz: float = 200e6,
               refractive_index: float = 1.0, station_pattern=None) -> ar_event:
    """Build an ``ar_event`` from tensors (device or host, matching the call used);
    ``station_pattern`` is an optional int32 tensor of pattern ids, one per station. The
    struct keeps references to the tensors, so they live at least as long as it does."""
    S, two, N = traces.shape
    assert two == 2
    if station_pattern is not None:
        assert station_pattern.dtype.itemsize == 4 and station_pattern.numel() == S
    ev = ar_event(S, N, dirs_rad.shape[0], pattern_id, fs_hz, refractive_index,
                  _ptr(traces), _ptr(pos_m), _ptr(t_start_ns), _ptr(dirs_rad),
                  _ptr(station_pattern) if station_pattern is not None else None)
    ev._tensors = (traces, pos_m, t_start_ns, dirs_rad, station_pattern)
    return ev


def alloc_outputs(n_dirs: int, n_stations: int, n_samples: int, device="cuda", traces: bool = True,
                  pin_memory: bool = False, fine: bool = False, snr: bool = False):
    """Allocate output tensors with the library's layouts; returns (dict, ar_outputs). With
    ``fine`` the dict also holds ``peak_time_fine_ns`` (sub-sample peak times; the residual
    then uses them); with ``snr`` it holds ``snr`` (pulse SNRs; the residual then weights
    stations by them)."""
    import torch
    D, S, N = n_dirs, n_stations, n_samples
    kw = dict(device=device)
    if device == "cpu" and pin_memory:
        kw["pin_memory"] = True
    o = dict(
        efield=torch.empty((D, S, 2, N), dtype=torch.float32, **kw) if traces else None,
        envelope=torch.empty((D, S, N), dtype=torch.float32, **kw) if traces else None,
        peak_idx=torch.empty((D, S), dtype=torch.int32, **kw),
        peak_amp=torch.empty((D, S), dtype=torch.float32, **kw),
        peak_time_ns=torch.empty((D, S), dtype=torch.float64, **kw),
        residual_ns=torch.empty((D, S), dtype=torch.float64, **kw),
        t0_ns=torch.empty((D,), dtype=torch.float64, **kw),
        chi2=torch.empty((D,), dtype=torch.float64, **kw),
        status=torch.empty((D, S), dtype=torch.int32, **kw),
    )
    if fine:
        o["peak_time_fine_ns"] = torch.empty((D, S), dtype=torch.float64, **kw)
    if snr:
        o["snr"] = torch.empty((D, S), dtype=torch.float32, **kw)
    return o, outputs_struct(o)


def outputs_struct(o: dict) -> ar_outputs:
    return ar_outputs(*[_ptr(o.get(k)) for k in ("efield", "envelope", "peak_idx", "peak_amp", "peak_time_ns",
                                                  "residual_ns", "t0_ns", "chi2", "status", "peak_time_fine_ns",
                                                  "snr")])


class Context:
    """One library context on one device (PyTorch tensors in, tensors out)."""

    def __init__(self, device: int = 0, autotune: bool = False, state_budget_bytes: int = 0):
        self.device = device
        self.h = ar_create(device, autotune, state_budget_bytes)

    def close(self):
        if self.h:
            ar_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_pattern(self, pattern) -> int:
        return ar_load_pattern(self.h, pattern)

    def prepare(self, n_samples: int, fs_hz: float, pattern_id: int, max_stations: int) -> None:
        ar_prepare(self.h, n_samples, fs_hz, pattern_id, max_stations)

    def unfold(self, pattern_id: int, traces, pos_m, t_start_ns, dirs_rad, fs_hz: float = 200e6,
               refractive_index: float = 1.0, out: dict | None = None, traces_out: bool = True,
               stream=None, sync: bool = False, station_pattern=None) -> dict:
        """Unfold an event held in device tensors; returns the output tensors (async unless sync)."""
        import torch
        S, _, N = traces.shape
        D = dirs_rad.shape[0]
        if out is None:
            out, _ = alloc_outputs(D, S, N, device=traces.device, traces=traces_out)
        ev = make_event(pattern_id, traces, pos_m, t_start_ns, dirs_rad, fs_hz, refractive_index, station_pattern)
        st = stream if stream is not None else torch.cuda.current_stream(traces.device)
        ar_unfold(self.h, ev, outputs_struct(out), st.cuda_stream)
        if sync:
            ar_sync(self.h, st.cuda_stream)
        return out

    def unfold_tc(self, pattern_id: int, traces, pos_m, t_start_ns, dirs_rad, split_terms: int = 3,
                  fs_hz: float = 200e6, refractive_index: float = 1.0, out: dict | None = None,
                  traces_out: bool = True, stream=None, sync: bool = False, station_pattern=None) -> dict:
        """ar_unfold_tc: the tensor-core DFT variant (split-BF16 x3 or x6) on device tensors."""
        import torch
        S, _, N = traces.shape
        D = dirs_rad.shape[0]
        if out is None:
            out, _ = alloc_outputs(D, S, N, device=traces.device, traces=traces_out)
        ev = make_event(pattern_id, traces, pos_m, t_start_ns, dirs_rad, fs_hz, refractive_index, station_pattern)
        st = stream if stream is not None else torch.cuda.current_stream(traces.device)
        ar_unfold_tc(self.h, ev, outputs_struct(out), split_terms, st.cuda_stream)
        if sync:
            ar_sync(self.h, st.cuda_stream)
        return out

    def batch(self, max_events: int, max_stations: int, max_dirs: int, max_n_freq: int = 64) -> "Batch":
        return Batch(self, max_events, max_stations, max_dirs, max_n_freq)

    def reconstruct(self, pattern_id: int, traces, pos_m, t_start_ns, fs_hz: float = 200e6,
                    refractive_index: float = 1.0, max_iter: int = 8, tol_rad: float = 1e-6, traces_out: bool = True,
                    stream=None, sync: bool = True) -> dict:
        """The iterative reconstruction of one event held in device tensors."""
        import torch
        S, _, N = traces.shape
        dev = traces.device
        last, _ = alloc_outputs(1, S, N, device=dev, traces=traces_out)
        res = dict(direction=torch.empty(2, dtype=torch.float64, device=dev),
                   t0_ns=torch.empty(1, dtype=torch.float64, device=dev),
                   chi2=torch.empty(1, dtype=torch.float64, device=dev),
                   iterations=torch.empty(1, dtype=torch.int32, device=dev),
                   history=torch.empty((max_iter + 1, 2), dtype=torch.float64, device=dev))
        dummy = torch.empty((1, 2), dtype=torch.float64, device=dev)
        ev = make_event(pattern_id, traces, pos_m, t_start_ns, dummy, fs_hz, refractive_index)
        out = ar_recon_out(_ptr(res["direction"]), _ptr(res["t0_ns"]), _ptr(res["chi2"]), _ptr(res["iterations"]),
                           _ptr(res["history"]), outputs_struct(last))
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        ar_reconstruct(self.h, ev, max_iter, tol_rad, out, st.cuda_stream)
        if sync:
            ar_sync(self.h, st.cuda_stream)
        res["last"] = last
        return res

    def sync(self, stream=None) -> None:
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        ar_sync(self.h, st.cuda_stream)

    def unfold_host(self, pattern_id: int, traces, pos_m, t_start_ns, dirs_rad, fs_hz: float = 200e6,
                    refractive_index: float = 1.0, out: dict | None = None, traces_out: bool = True,
                    stream=None, station_pattern=None) -> dict:
        """ar_unfold_host: inputs and outputs are host (CPU) tensors; returns when done."""
        import torch
        S, _, N = traces.shape
        D = dirs_rad.shape[0]
        if out is None:
            out, _ = alloc_outputs(D, S, N, device="cpu", traces=traces_out)
        ev = make_event(pattern_id, traces, pos_m, t_start_ns, dirs_rad, fs_hz, refractive_index, station_pattern)
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        ar_unfold_host(self.h, ev, outputs_struct(out), st.cuda_stream)
        return out


class Batch:
    """A batch plan (ar_batch_*) bound to a Context."""

    def __init__(self, ctx: Context, max_events: int, max_stations: int, max_dirs: int, max_n_freq: int = 64):
        self.ctx = ctx
        self.h = ar_batch_create(ctx.h, max_events, max_stations, max_dirs, max_n_freq)

    def run(self, events, outs, stream=None) -> None:
        """events: list of ``ar_event``; outs: list of output dicts (tensors) or ``ar_outputs``."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(self.ctx.device)
        structs = [o if isinstance(o, ar_outputs) else outputs_struct(o) for o in outs]
        ar_batch_run(self.ctx.h, self.h, events, structs, st.cuda_stream)

    def tuning(self):
        return ar_batch_tuning(self.h)

    def tuning_info(self) -> dict:
        """The plan per length class (1024, 2048, 4096 samples) and the autotuner's timings."""
        return ar_batch_tuning_info(self.h)

    def close(self):
        if self.h:
            ar_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A continuous-batching server (ar_server_*) on a Context: events and outputs in host
    (preferably pinned) tensors."""

    def __init__(self, ctx: Context, state_budget_bytes: int = 0, max_batch_events: int = 32, max_inflight: int = 2,
                 max_stations_per_event: int = 124, max_n_freq: int = 64):
        self.ctx = ctx
        self.h = ar_server_create(ctx.h, state_budget_bytes, max_batch_events, max_inflight, max_stations_per_event,
                                  max_n_freq)
        self._live = {}   # ticket -> (event, outputs): their memory must outlive the request

    def submit(self, ev: ar_event, out) -> int:
        t = ar_submit(self.ctx.h, self.h, ev, out if isinstance(out, ar_outputs) else outputs_struct(out))
        self._live[t] = (ev, out)
        return t

    def _settled(self, ticket: int, st: int) -> int:
        if st not in (AR_ERR_NOT_READY, AR_ERR_TIMEOUT):
            self._live.pop(ticket, None)
        return st

    def poll(self, ticket: int) -> int:
        return self._settled(ticket, ar_poll(self.h, ticket))

    def wait(self, ticket: int, timeout_ms: int = 60000) -> int:
        return self._settled(ticket, ar_wait(self.h, ticket, timeout_ms))

    def times(self, ticket: int):
        return ar_ticket_times(self.h, ticket)

    def release(self, ticket: int) -> int:
        st = ar_ticket_release(self.h, ticket)
        if st == AR_OK:
            self._live.pop(ticket, None)
        return st

    def close(self):
        if self.h:
            ar_server_destroy(self.h)   # finishes every queued and running request
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
