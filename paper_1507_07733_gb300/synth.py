"""Seeded synthetic AERA-like inputs: antenna pattern, station layout, traces, directions.

This module only *generates inputs*. It holds none of the unfolding arithmetic
(no transforms, no interpolation, no 2x2 solve, no envelope, no residual), so the
FP64 oracle and the CUDA path can both be fed from it without sharing code.

Shapes follow the paper's detector description (Sec. 1: 124 stations on a hexagonal
grid of about 6 km^2, each with a two-channel antenna for polarised measurements from
30 to 80 MHz; Sec. 3: the antenna vector effective length tabulated over frequency,
zenith and azimuth). No real AERA data or antenna pattern exists here, so every array
is synthetic and derived from one master seed.

Pattern model (a smooth, invertible stand-in for a measured VEL table):

    H[c,p](zen, az, f) = R_c(f) * M_c(zen, az) * G[c,p](zen, az) * (1 + 0.01 (n1 + i n2))

    G[0,:] = (cos zen cos az, -sin az)    east-west arm
    G[1,:] = (cos zen sin az,  cos az)    north-south arm       (det G = cos zen)
    M_c    = (1 + a1 cos zen + a2 cos 2az + a3 sin zen sin az) * exp(i b (1 - cos zen))
    R_c(f) = L0 / (1 + i Q_c (f/f0c - f0c/f))                  resonant response
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASTER_SEED = 1507077330

C_M_PER_NS = 0.299792458  # speed of light in vacuum [m/ns]

#: pattern grid of the synthetic table: zenith 0..90 deg step 5, azimuth 0..355 step 5,
#: frequency 30..80 MHz step 1 MHz
PATTERN_GRID = dict(n_zen=19, zen0_deg=0.0, dzen_deg=5.0,
                    n_az=72, az0_deg=0.0, daz_deg=5.0,
                    n_freq=51, f0_hz=30e6, df_hz=1e6)

#: the paper's largest pattern (Sec. 3): 98 frequencies x 31 zenith x 49 azimuth angles. Read
#: as zenith 0..90 deg step 3, azimuth 0..360 deg step 7.5 with the 360-degree node equal to
#: the 0-degree one (48 distinct periodic nodes), and 98 frequencies spanning 30..80 MHz.
LARGE_PATTERN_GRID = dict(n_zen=31, zen0_deg=0.0, dzen_deg=3.0,
                          n_az=48, az0_deg=0.0, daz_deg=7.5,
                          n_freq=98, f0_hz=30e6, df_hz=50e6 / 97)

FS_HZ = 200e6           # AERA digitiser rate used by every workload
STATION_SPACING_M = 236.0


def _rng(*keys: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([MASTER_SEED, *keys])))


@dataclasses.dataclass
class Pattern:
    """A complex VEL table with its axes.

    ``table`` is complex64 with shape [n_zen][n_az][n_freq][2 channels][2 polarisations]
    (polarisation 0 = theta, 1 = phi). Axis origins and steps are in radians and Hz.
    """
    n_zen: int
    zen0_rad: float
    dzen_rad: float
    n_az: int
    az0_rad: float
    daz_rad: float
    n_freq: int
    f0_hz: float
    df_hz: float
    table: np.ndarray

    def desc(self) -> dict:
        return {k: getattr(self, k) for k in (
            "n_zen", "zen0_rad", "dzen_rad", "n_az", "az0_rad", "daz_rad",
            "n_freq", "f0_hz", "df_hz")}


def make_pattern(seed_key: int = 0, noise: float = 0.01, grid: dict | None = None) -> Pattern:
    """Synthetic two-channel VEL table on ``grid`` (default ``PATTERN_GRID``)."""
    g = PATTERN_GRID if grid is None else grid
    rng = _rng(101, seed_key)
    zen = np.deg2rad(g["zen0_deg"] + g["dzen_deg"] * np.arange(g["n_zen"]))
    az = np.deg2rad(g["az0_deg"] + g["daz_deg"] * np.arange(g["n_az"]))
    f = g["f0_hz"] + g["df_hz"] * np.arange(g["n_freq"])
    Z, A = np.meshgrid(zen, az, indexing="ij")             # [zen][az]
    cz, sz, ca, sa = np.cos(Z), np.sin(Z), np.cos(A), np.sin(A)
    G = np.empty(Z.shape + (2, 2), dtype=np.float64)
    G[..., 0, 0] = cz * ca
    G[..., 0, 1] = -sa
    G[..., 1, 0] = cz * sa
    G[..., 1, 1] = ca
    table = np.empty((g["n_zen"], g["n_az"], g["n_freq"], 2, 2), dtype=np.complex128)
    for c in range(2):
        a1, a2, a3 = rng.uniform(-0.2, 0.2, size=3)
        b = rng.uniform(-0.5, 0.5)
        f0c = rng.uniform(52e6, 58e6)
        qc = rng.uniform(1.5, 3.0)
        M = (1 + a1 * cz + a2 * np.cos(2 * A) + a3 * sz * sa) * np.exp(1j * b * (1 - cz))
        R = 1.0 / (1 + 1j * qc * (f / f0c - f0c / f))       # L0 = 1 m
        for p in range(2):
            table[:, :, :, c, p] = (M * G[..., c, p])[:, :, None] * R[None, None, :]
    n1 = rng.standard_normal(table.shape)
    n2 = rng.standard_normal(table.shape)
    table *= 1 + noise * (n1 + 1j * n2)
    return Pattern(g["n_zen"], math.radians(g["zen0_deg"]), math.radians(g["dzen_deg"]),
                   g["n_az"], math.radians(g["az0_deg"]), math.radians(g["daz_deg"]),
                   g["n_freq"], g["f0_hz"], g["df_hz"], table.astype(np.complex64))


def make_flat_pattern(matrix: np.ndarray, grid: dict | None = None) -> Pattern:
    """A pattern whose every node holds the same 2x2 complex ``matrix`` [c][p]."""
    g = dict(PATTERN_GRID if grid is None else grid)
    shape = (g["n_zen"], g["n_az"], g["n_freq"], 2, 2)
    table = np.broadcast_to(np.asarray(matrix, dtype=np.complex64), shape).copy()
    return Pattern(g["n_zen"], math.radians(g["zen0_deg"]), math.radians(g["dzen_deg"]),
                   g["n_az"], math.radians(g["az0_deg"]), math.radians(g["daz_deg"]),
                   g["n_freq"], g["f0_hz"], g["df_hz"], table)


def hex_lattice(n: int, spacing: float = STATION_SPACING_M) -> np.ndarray:
    """The ``n`` triangular-lattice nodes nearest the origin, [n][2] metres (deterministic)."""
    r = int(math.ceil(math.sqrt(n))) + 3
    pts = []
    for j in range(-r, r + 1):
        for i in range(-r, r + 1):
            x = spacing * (i + 0.5 * j)
            y = spacing * (math.sqrt(3) / 2) * j
            pts.append((x * x + y * y, math.atan2(y, x), x, y))
    pts.sort()
    return np.array([(p[2], p[3]) for p in pts[:n]], dtype=np.float64)


def make_stations(n: int = 124, seed_key: int = 0) -> np.ndarray:
    """Station positions [n][3] in metres: the 124-node hexagonal array, jittered.

    For ``n`` < 124 a seeded subset of the full array is returned.
    """
    rng = _rng(202, seed_key)
    xy = hex_lattice(124)
    xy = xy + rng.uniform(-5.0, 5.0, size=xy.shape)
    z = rng.normal(0.0, 2.0, size=(124, 1))
    pos = np.concatenate([xy, z], axis=1)
    if n < 124:
        idx = np.sort(rng.choice(124, size=n, replace=False))
        pos = pos[idx]
    elif n > 124:
        raise ValueError("the synthetic array has 124 stations")
    return np.ascontiguousarray(pos)


def _pulse(n: int, pos_samples: float, dt_ns: float, amp: float, tau_ns: float = 5.0) -> np.ndarray:
    """Bipolar Gaussian-derivative pulse peaking at ``amp`` near ``pos_samples``."""
    t = (np.arange(n) - pos_samples) * dt_ns
    return amp * (-t / tau_ns) * np.exp(0.5 - t * t / (2 * tau_ns * tau_ns))


@dataclasses.dataclass
class Event:
    """One radio event: traces [S][2][N] float32, positions [S][3] m, window starts [S] ns,
    candidate directions [D][2] (zenith, azimuth) rad."""
    traces: np.ndarray
    pos_m: np.ndarray
    t_start_ns: np.ndarray
    dirs_rad: np.ndarray
    fs_hz: float = FS_HZ
    true_dir: tuple | None = None

    @property
    def n_stations(self) -> int:
        return self.traces.shape[0]

    @property
    def n_samples(self) -> int:
        return self.traces.shape[2]

    @property
    def n_dirs(self) -> int:
        return self.dirs_rad.shape[0]


def scan_directions(n_zen: int = 8, n_az: int = 8, zen_max_deg: float = 60.0) -> np.ndarray:
    """Grid scan: zenith linspace(0, zen_max, n_zen) x azimuth 0, 360/n_az, ... [D][2] rad."""
    zz = np.deg2rad(np.linspace(0.0, zen_max_deg, n_zen))
    aa = np.deg2rad(np.arange(n_az) * (360.0 / n_az))
    Z, A = np.meshgrid(zz, aa, indexing="ij")
    return np.ascontiguousarray(np.stack([Z.ravel(), A.ravel()], axis=1))


def random_directions(n: int, rng: np.random.Generator, zen_max_deg: float = 60.0) -> np.ndarray:
    zz = np.deg2rad(rng.uniform(0.0, zen_max_deg, size=n))
    aa = np.deg2rad(rng.uniform(0.0, 360.0, size=n))
    return np.ascontiguousarray(np.stack([zz, aa], axis=1))


def make_event(n_stations: int, n_samples: int, dirs_rad: np.ndarray, seed_key: int = 0,
               plane_wave: bool = True, fs_hz: float = FS_HZ, noise_sigma: float = 1.0) -> Event:
    """Noise plus one bipolar pulse per station.

    With ``plane_wave`` the pulse arrival follows a seeded true direction (zenith <= 60 deg)
    and each station's window start is set so the pulse falls in [0.2 N, 0.8 N); otherwise
    the pulse sits uniformly in [N/8, 7N/8) and windows start at 0.
    """
    rng = _rng(303, seed_key, n_stations, n_samples)
    S, N = n_stations, n_samples
    dt_ns = 1e9 / fs_hz
    pos = make_stations(S, seed_key)
    traces = (noise_sigma * rng.standard_normal((S, 2, N))).astype(np.float64)
    amp = rng.uniform(5.0, 50.0, size=S) * noise_sigma
    alpha = rng.uniform(0.0, 2 * math.pi, size=S)
    if plane_wave:
        zt = math.radians(rng.uniform(0.0, 60.0))
        at = math.radians(rng.uniform(0.0, 360.0))
        k = np.array([math.sin(zt) * math.cos(at), math.sin(zt) * math.sin(at), math.cos(zt)])
        # arrival time of a plane front coming from direction k (earlier where k.x is larger)
        t_arr = -(pos @ k) / C_M_PER_NS
        p = rng.uniform(0.2 * N, 0.8 * N, size=S)
        t_start = t_arr - p * dt_ns
        true_dir = (zt, at)
    else:
        p = rng.uniform(N / 8, 7 * N / 8, size=S)
        t_start = np.zeros(S)
        true_dir = None
    for s in range(S):
        pul = _pulse(N, p[s], dt_ns, amp[s])
        traces[s, 0] += math.cos(alpha[s]) * pul
        traces[s, 1] += math.sin(alpha[s]) * pul
    return Event(np.ascontiguousarray(traces.astype(np.float32)), pos,
                 np.ascontiguousarray(t_start), np.ascontiguousarray(dirs_rad, dtype=np.float64),
                 fs_hz, true_dir)


# ---- the workloads -----------------------------------------------------------------

def single_event(n_samples: int = 2048) -> Event:
    """Plain single event: 10 stations x 2 x N samples, 1 direction (zenith 30, azimuth 45)."""
    dirs = np.deg2rad(np.array([[30.0, 45.0]]))
    return make_event(10, n_samples, dirs, seed_key=1, plane_wave=False)


def direction_scan(n_stations: int = 124, n_samples: int = 2048) -> Event:
    """Direction scan: 124 stations x 2 x 2048 samples, 8 zenith x 8 azimuth directions."""
    return make_event(n_stations, n_samples, scan_directions(8, 8), seed_key=2, plane_wave=True)


def mixed_antenna_patterns() -> list:
    """The antenna types of the mixed-antenna workload: two on the standard grid (different
    seeds) and one on the paper's largest grid (``LARGE_PATTERN_GRID``)."""
    return [make_pattern(seed_key=0), make_pattern(seed_key=7), make_pattern(seed_key=8, grid=LARGE_PATTERN_GRID)]


def station_antenna_types(n_stations: int, n_types: int = 3, seed_key: int = 9, sort: bool = True) -> np.ndarray:
    """A seeded antenna type per station (about half type 0, 30 % type 1, 20 % type 2).

    With ``sort`` the types are non-decreasing along the station index (stations grouped by
    antenna type, the order the unfolding walks most efficiently); otherwise they are mixed.
    """
    rng = _rng(707, seed_key, n_stations)
    p = np.array([0.5, 0.3, 0.2][:n_types])
    t = rng.choice(n_types, size=n_stations, p=p / p.sum()).astype(np.int32)
    return np.sort(t) if sort else t


def mixed_antenna_scan(n_stations: int = 124, n_samples: int = 2048) -> Event:
    """Mixed-antenna direction scan: the direction-scan event (124 stations x 2 x 2048
    samples, 8 x 8 directions); ``station_antenna_types`` gives each station's antenna."""
    return direction_scan(n_stations, n_samples)


def uneven_stream(n_events: int = 256, seed_key: int = 4):
    """Batched uneven workload: per event S ~ U{3..124}, N ~ U{1024,2048,4096}, D ~ U{16..256}.

    Returns a list of (n_stations, n_samples, n_dirs, event_seed) descriptors; call
    ``materialise`` to build the arrays of one of them.
    """
    rng = _rng(404, seed_key)
    out = []
    for e in range(n_events):
        S = int(rng.integers(3, 125))
        N = int(rng.choice([1024, 2048, 4096]))
        D = int(rng.integers(16, 257))
        out.append((S, N, D, 1000 + e))
    return out


def materialise(desc) -> Event:
    S, N, D, key = desc
    rng = _rng(505, key)
    return make_event(S, N, random_directions(D, rng), seed_key=key, plane_wave=True)


def poisson_arrivals(rate_hz: float, n: int, seed_key: int = 5) -> np.ndarray:
    """Arrival offsets (seconds from t=0) of a Poisson stream of ``n`` events."""
    rng = _rng(606, seed_key, int(rate_hz))
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
