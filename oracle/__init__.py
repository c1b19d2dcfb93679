"""Python access to the FP64 CPU oracle (``aera_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg. The product library never imports it and shares no
code with it. ``build()`` compiles the C source with gcc (OpenMP over pairs,
``-ffp-contract=off`` so that no host fuses multiply-adds).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aera_oracle.c")
_LIB = os.path.join(_HERE, "libaera_oracle.so")
_lock = threading.Lock()
_lib = None

ST_SINGULAR = 1
ST_ZEN_CLAMP = 2
ST_BAD_DIR = 4


class _Pattern(ctypes.Structure):
    _fields_ = [("n_zen", ctypes.c_int32), ("zen0_rad", ctypes.c_double), ("dzen_rad", ctypes.c_double),
                ("n_az", ctypes.c_int32), ("az0_rad", ctypes.c_double), ("daz_rad", ctypes.c_double),
                ("n_freq", ctypes.c_int32), ("f0_hz", ctypes.c_double), ("df_hz", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``libaera_oracle.so`` next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P, D, I, U, F = (ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_float))
            I32 = ctypes.POINTER(ctypes.c_int32)
            PP = ctypes.POINTER(_Pattern)
            L.orc_in_band.argtypes = [I, D, I]
            L.orc_dft.argtypes = [I, I, P, P]
            L.orc_station_spectrum.argtypes = [I, F, P]
            L.orc_vel.argtypes = [PP, F, D, D, D, P, U]
            L.orc_solve.argtypes = [P, P, P, P]
            L.orc_solve.restype = I
            L.orc_unfold_pair.argtypes = [PP, F, I, D, P, D, D, P, P, I32, P, U, P]
            L.orc_residual.argtypes = [I, P, P, D, D, D, P, P, P]
            L.orc_peak_offset.argtypes = [I, P, I]
            L.orc_peak_offset.restype = D
            L.orc_snr.argtypes = [I, P, I]
            L.orc_snr.restype = D
            L.orc_residual_weighted.argtypes = [I, P, P, P, D, D, D, P, P, P]
            L.orc_unfold_event.argtypes = [PP, F, I, I, D, D, F, P, P, I, P,
                                           P, P, I32, P, P, P, P, P, U, P]
            L.orc_unfold_sample.argtypes = [PP, F, I, D, F, P, P, I, I32, I32,
                                            P, P, I32, P, P, U, P]
            L.orc_voltage_peaks.argtypes = [I, I, D, F, P, I32, P]
            L.orc_plane_fit.argtypes = [I, P, P, D, P, P, P]
            L.orc_plane_fit.restype = I
            L.orc_reconstruct.argtypes = [PP, F, I, I, D, D, F, P, P, I, D, P, I32, P, P, P, P,
                                          P, P, I32, P, P, U]
            L.orc_reconstruct.restype = I
            _lib = L
    return _lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _pat(pattern) -> tuple:
    d = pattern.desc()
    table = np.ascontiguousarray(pattern.table, dtype=np.complex64).view(np.float32)
    return _Pattern(**d), table


def set_threads(n: int) -> None:
    """Set the OpenMP thread count used by later oracle calls in this process."""
    os.environ["OMP_NUM_THREADS"] = str(n)
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
    except OSError:
        pass


def in_band(n: int, fs_hz: float, k: int) -> bool:
    return bool(lib().orc_in_band(n, fs_hz, k))


def dft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Naive unnormalised DFT of a complex vector; sign -1 forward, +1 inverse."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    lib().orc_dft(x.size, sign, _p(x.view(np.float64)), _p(out.view(np.float64)))
    return out


def station_spectrum(trace: np.ndarray) -> np.ndarray:
    """[2][N] float32 trace -> [2][N] complex128 spectra (each channel on its own)."""
    trace = np.ascontiguousarray(trace, dtype=np.float32)
    n = trace.shape[-1]
    out = np.empty((2, n), dtype=np.complex128)
    lib().orc_station_spectrum(n, _p(trace, ctypes.c_float), _p(out.view(np.float64)))
    return out


def vel(pattern, zen: float, az: float, f_hz: float):
    """Interpolated VEL H[c][p] (complex128 2x2) and status bits."""
    pd, table = _pat(pattern)
    H = np.empty(8)
    st = np.zeros(1, dtype=np.uint32)
    lib().orc_vel(ctypes.byref(pd), _p(table, ctypes.c_float), zen, az, f_hz, _p(H), _p(st, ctypes.c_uint32))
    return H.view(np.complex128).reshape(2, 2), int(st[0])


def solve(H: np.ndarray, V: np.ndarray):
    """Closed-form E for V = H E; returns (E complex[2], singular flag, margin)."""
    Hf = np.ascontiguousarray(np.asarray(H, dtype=np.complex128).reshape(4)).view(np.float64)
    Vf = np.ascontiguousarray(np.asarray(V, dtype=np.complex128).reshape(2)).view(np.float64)
    E = np.empty(4)
    mg = np.empty(1)
    sing = lib().orc_solve(_p(Hf), _p(Vf), _p(E), _p(mg))
    return E.view(np.complex128), int(sing), float(mg[0])


def unfold_pair(pattern, trace: np.ndarray, zen: float, az: float, fs_hz: float = 200e6):
    """One pair from a [2][N] float32 trace: dict(efield [2][N], env [N], peak_idx, peak_amp,
    status, min_margin)."""
    pd, table = _pat(pattern)
    spec = station_spectrum(trace)
    n = spec.shape[1]
    ef = np.empty((2, n))
    env = np.empty(n)
    pi = np.zeros(1, dtype=np.int32)
    pa = np.empty(1)
    st = np.zeros(1, dtype=np.uint32)
    mm = np.empty(1)
    lib().orc_unfold_pair(ctypes.byref(pd), _p(table, ctypes.c_float), n, fs_hz, _p(spec.view(np.float64)),
                          zen, az, _p(ef), _p(env), _p(pi, ctypes.c_int32), _p(pa),
                          _p(st, ctypes.c_uint32), _p(mm))
    return dict(efield=ef, env=env, peak_idx=int(pi[0]), peak_amp=float(pa[0]), status=int(st[0]),
                min_margin=float(mm[0]))


def residual(pos: np.ndarray, peak_time: np.ndarray, zen: float, az: float, n_refr: float = 1.0):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    pt = np.ascontiguousarray(peak_time, dtype=np.float64)
    res = np.empty(pos.shape[0])
    t0 = np.empty(1)
    chi2 = np.empty(1)
    lib().orc_residual(pos.shape[0], _p(pos), _p(pt), zen, az, n_refr, _p(res), _p(t0), _p(chi2))
    return res, float(t0[0]), float(chi2[0])


def peak_offset(env: np.ndarray, k: int) -> float:
    """Sub-sample offset of the envelope maximum at sample k (parabola through k-1, k, k+1)."""
    e = np.ascontiguousarray(env, dtype=np.float64)
    return float(lib().orc_peak_offset(e.size, _p(e), int(k)))


def snr(env: np.ndarray, k: int) -> float:
    """(env[k] / noise)^2, noise^2 = mean of env^2 more than N/16 samples from k (0 if none)."""
    e = np.ascontiguousarray(env, dtype=np.float64)
    return float(lib().orc_snr(e.size, _p(e), int(k)))


def event_snr(envelope: np.ndarray, peak_idx: np.ndarray) -> np.ndarray:
    """SNR [D][S] of an event's envelopes [D][S][N] at the given peak indices [D][S]."""
    D, S, _ = envelope.shape
    return np.array([[snr(envelope[d, s], int(peak_idx[d, s])) for s in range(S)] for d in range(D)])


def residual_weighted(pos: np.ndarray, peak_time: np.ndarray, w: np.ndarray, zen: float, az: float,
                      n_refr: float = 1.0):
    """Plane-wave residual with per-station weights (the unweighted fit when they sum to 0)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    pt = np.ascontiguousarray(peak_time, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    res = np.empty(pos.shape[0])
    t0 = np.empty(1)
    chi2 = np.empty(1)
    lib().orc_residual_weighted(pos.shape[0], _p(pos), _p(pt), _p(ww), zen, az, n_refr, _p(res), _p(t0), _p(chi2))
    return res, float(t0[0]), float(chi2[0])


def fine_peak_times(envelope: np.ndarray, peak_idx: np.ndarray, t_start_ns: np.ndarray, fs_hz: float) -> np.ndarray:
    """Refined peak times [D][S] from an event's envelopes [D][S][N] and peak indices [D][S]."""
    D, S, N = envelope.shape
    out = np.empty((D, S))
    for d in range(D):
        for s in range(S):
            k = int(peak_idx[d, s])
            out[d, s] = t_start_ns[s] + (k + peak_offset(envelope[d, s], k)) * (1e9 / fs_hz)
    return out


def unfold_event(pattern, ev, n_refr: float = 1.0, traces_out: bool = True) -> dict:
    """Every pair of an event (``synth.Event``), with the output layouts of the library."""
    pd, table = _pat(pattern)
    S, N, D = ev.n_stations, ev.n_samples, ev.n_dirs
    tr = np.ascontiguousarray(ev.traces, dtype=np.float32)
    pos = np.ascontiguousarray(ev.pos_m, dtype=np.float64)
    ts = np.ascontiguousarray(ev.t_start_ns, dtype=np.float64)
    dirs = np.ascontiguousarray(ev.dirs_rad, dtype=np.float64)
    o = dict(efield=np.empty((D, S, 2, N)) if traces_out else None,
             envelope=np.empty((D, S, N)) if traces_out else None,
             peak_idx=np.zeros((D, S), dtype=np.int32), peak_amp=np.empty((D, S)),
             peak_time_ns=np.empty((D, S)), residual_ns=np.empty((D, S)), t0_ns=np.empty(D),
             chi2=np.empty(D), status=np.zeros((D, S), dtype=np.uint32), min_margin=np.empty((D, S)))
    lib().orc_unfold_event(ctypes.byref(pd), _p(table, ctypes.c_float), S, N, ev.fs_hz, n_refr,
                           _p(tr, ctypes.c_float), _p(pos), _p(ts), D, _p(dirs),
                           _p(o["efield"]), _p(o["envelope"]), _p(o["peak_idx"], ctypes.c_int32),
                           _p(o["peak_amp"]), _p(o["peak_time_ns"]), _p(o["residual_ns"]),
                           _p(o["t0_ns"]), _p(o["chi2"]), _p(o["status"], ctypes.c_uint32),
                           _p(o["min_margin"]))
    return o


def unfold_sample(pattern, ev, st_idx, dir_idx, traces_out: bool = True) -> dict:
    """A sample of pairs (station index, direction index) of an event."""
    pd, table = _pat(pattern)
    N = ev.n_samples
    si = np.ascontiguousarray(st_idx, dtype=np.int32)
    di = np.ascontiguousarray(dir_idx, dtype=np.int32)
    n = si.size
    tr = np.ascontiguousarray(ev.traces, dtype=np.float32)
    ts = np.ascontiguousarray(ev.t_start_ns, dtype=np.float64)
    dirs = np.ascontiguousarray(ev.dirs_rad, dtype=np.float64)
    o = dict(efield=np.empty((n, 2, N)) if traces_out else None,
             envelope=np.empty((n, N)) if traces_out else None,
             peak_idx=np.zeros(n, dtype=np.int32), peak_amp=np.empty(n), peak_time_ns=np.empty(n),
             status=np.zeros(n, dtype=np.uint32), min_margin=np.empty(n))
    lib().orc_unfold_sample(ctypes.byref(pd), _p(table, ctypes.c_float), N, ev.fs_hz,
                            _p(tr, ctypes.c_float), _p(ts), _p(dirs), n,
                            _p(si, ctypes.c_int32), _p(di, ctypes.c_int32),
                            _p(o["efield"]), _p(o["envelope"]), _p(o["peak_idx"], ctypes.c_int32),
                            _p(o["peak_amp"]), _p(o["peak_time_ns"]), _p(o["status"], ctypes.c_uint32),
                            _p(o["min_margin"]))
    return o


def voltage_peaks(ev):
    """Initial timing of the reconstruction loop: per station argmax_n v0^2 + v1^2."""
    tr = np.ascontiguousarray(ev.traces, dtype=np.float32)
    idx = np.zeros(ev.n_stations, dtype=np.int32)
    t = np.empty(ev.n_stations)
    lib().orc_voltage_peaks(ev.n_stations, ev.n_samples, ev.fs_hz, _p(tr, ctypes.c_float),
                            _p(np.ascontiguousarray(ev.t_start_ns, dtype=np.float64)), _p(idx, ctypes.c_int32), _p(t))
    return idx, t


def plane_fit(pos, t_ns, n_refr: float = 1.0):
    """Least-squares plane-wave direction: (zenith, azimuth, t0) or None if undetermined."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    t = np.ascontiguousarray(t_ns, dtype=np.float64)
    z, a, t0 = np.empty(1), np.empty(1), np.empty(1)
    if lib().orc_plane_fit(pos.shape[0], _p(pos), _p(t), n_refr, _p(z), _p(a), _p(t0)):
        return None
    return float(z[0]), float(a[0]), float(t0[0])


def reconstruct(pattern, ev, max_iter: int = 8, tol_rad: float = 1e-6, n_refr: float = 1.0) -> dict:
    """The iterative loop of Sec. 2 on one event (directions of ``ev`` are ignored)."""
    pd, table = _pat(pattern)
    S, N = ev.n_stations, ev.n_samples
    tr = np.ascontiguousarray(ev.traces, dtype=np.float32)
    pos = np.ascontiguousarray(ev.pos_m, dtype=np.float64)
    ts = np.ascontiguousarray(ev.t_start_ns, dtype=np.float64)
    hist = np.full((max_iter + 1, 2), np.nan)
    ihist = np.full((max_iter + 1, S), -1, dtype=np.int32)
    zen, az, t0, chi2 = np.empty(1), np.empty(1), np.empty(1), np.full(1, np.nan)
    ef, env = np.empty((S, 2, N)), np.empty((S, N))
    pi, pa, pt = np.zeros(S, dtype=np.int32), np.empty(S), np.empty(S)
    st = np.zeros(S, dtype=np.uint32)
    it = lib().orc_reconstruct(ctypes.byref(pd), _p(table, ctypes.c_float), S, N, ev.fs_hz, n_refr,
                               _p(tr, ctypes.c_float), _p(pos), _p(ts), max_iter, tol_rad, _p(hist),
                               _p(ihist, ctypes.c_int32), _p(zen), _p(az), _p(t0), _p(chi2), _p(ef), _p(env),
                               _p(pi, ctypes.c_int32), _p(pa), _p(pt), _p(st, ctypes.c_uint32))
    return dict(iterations=it, zenith=float(zen[0]), azimuth=float(az[0]), t0_ns=float(t0[0]), chi2=float(chi2[0]),
                history=hist, peak_idx_history=ihist, efield=ef, envelope=env, peak_idx=pi, peak_amp=pa,
                peak_time_ns=pt, status=st)
