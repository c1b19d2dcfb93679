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
