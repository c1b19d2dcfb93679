"""Synthetic-input generator checks against the detector facts the paper states."""
import json
import math
import os

import numpy as np

from paper_1507_07733_gb300 import synth

HERE = os.path.dirname(__file__)
FACTS = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))


def test_station_array_matches_paper():
    pos = synth.make_stations(124)
    assert pos.shape == (FACTS["n_stations"]["value"], 3)
    # each node of a triangular lattice owns a hexagon of area (sqrt 3 / 2) d^2
    area_km2 = 124 * (math.sqrt(3) / 2) * synth.STATION_SPACING_M ** 2 / 1e6
    assert abs(area_km2 - FACTS["array_area_km2"]["value"]) <= 0.05 * FACTS["array_area_km2"]["value"]
    d = np.sqrt(((pos[:, None, :2] - pos[None, :, :2]) ** 2).sum(-1)) + 1e9 * np.eye(124)
    assert np.all(abs(d.min(1) - synth.STATION_SPACING_M) <= 15.0)


def test_pattern_table_layout_size():
    # a 2-component complex VEL table in single precision at the paper's largest grid
    lp = FACTS["largest_pattern"]
    nbytes = lp["n_freq"] * lp["n_zen"] * lp["n_az"] * 2 * np.dtype(np.complex64).itemsize
    assert abs(nbytes - lp["approx_bytes_fp32"]) <= 0.05 * lp["approx_bytes_fp32"]
    p = synth.make_pattern()
    assert p.table.shape == (19, 72, 51, 2, FACTS["channels_per_station"]["value"])
    assert p.table.dtype == np.complex64 and p.table.nbytes == 2_232_576


def test_pattern_invertible_below_60_deg():
    p = synth.make_pattern()
    t = p.table.astype(np.complex128)
    det = t[..., 0, 0] * t[..., 1, 1] - t[..., 0, 1] * t[..., 1, 0]
    scale = abs(t[..., 0, 0]) * abs(t[..., 1, 1]) + abs(t[..., 0, 1]) * abs(t[..., 1, 0])
    assert np.all(abs(det[:13]) > 0.3 * scale[:13])         # zenith 0..60 deg


def test_seeded_and_shapes():
    a, b = synth.direction_scan(), synth.direction_scan()
    assert np.array_equal(a.traces, b.traces) and a.traces.shape == (124, 2, 2048)
    assert a.traces.dtype == np.float32 and a.dirs_rad.shape == (64, 2)
    e = synth.single_event()
    assert e.traces.shape == (10, 2, 2048) and e.n_dirs == 1
    s = synth.uneven_stream(256)
    assert len(s) == 256 and all(3 <= x[0] <= 124 and x[1] in (1024, 2048, 4096) and 16 <= x[2] <= 256 for x in s)


def test_large_grid_and_antenna_types():
    lp = FACTS["largest_pattern"]
    big = synth.mixed_antenna_patterns()[2]
    # the paper's 49 azimuth angles include 360 deg = 0 deg: 48 periodic nodes are stored
    assert big.table.shape == (lp["n_zen"], lp["n_az"] - 1, lp["n_freq"], 2, 2)
    assert abs(big.n_az * big.daz_rad - 2 * math.pi) <= 1e-12
    assert abs(big.f0_hz + (big.n_freq - 1) * big.df_hz - 80e6) <= 1e-3
    assert abs((big.n_zen - 1) * big.dzen_rad - math.pi / 2) <= 1e-12
    t = synth.station_antenna_types(124)
    assert t.dtype == np.int32 and t.shape == (124,) and set(np.unique(t)) == {0, 1, 2}
    assert np.all(np.diff(t) >= 0)
    u = synth.station_antenna_types(124, sort=False)
    assert np.array_equal(np.sort(u), t) and np.any(np.diff(u) < 0)
