"""The seeded generators: deterministic, right sizes and ranges, and the
density structure each workload asks for (no GPU)."""

import numpy as np

from paper_1611_08494_gb300 import synth


def test_deterministic():
    a, b = synth.c1(), synth.c1()
    for k in ("a_lon", "a_lat", "b_lon", "b_lat"):
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(synth.c1(seed=5)["a_lon"], a["a_lon"])


def test_c1_shape():
    d = synth.c1()
    assert d["a_lon"].size == 10_000 and d["b_lon"].size == 10_000
    assert d["a_lon"].min() >= 150 and d["a_lon"].max() < 151
    assert d["a_lat"].min() >= 2 and d["a_lat"].max() <= 3
    assert d["truth"]["a_row"].size == 7_000
    assert np.unique(d["truth"]["b_row"]).size == 7_000


def test_c2_profile():
    d = synth.c2(scale=0.05)
    assert d["a_lon"].size == 10_000 and d["b_lon"].size == 250_000
    b = np.abs(d["b_lat"])
    assert b.max() <= 1.0 and d["b_lon"].max() <= 3.0
    # truncated exponential in |b| with scale 0.3 deg on [0, 1]
    x = 1.0 / 0.3
    mean = 0.3 * (1 - (1 + x) * np.exp(-x)) / (1 - np.exp(-x))
    assert abs(b.mean() - mean) < 0.005
    r = d["region"]
    assert r["a_col"].min() >= 5 and r["a_col"].max() <= 60
    ratio = r["b_col"] / r["a_col"]
    assert ratio.min() >= 0.3 and ratio.max() <= 1.0
    assert r["pa_col"].min() >= 0 and r["pa_col"].max() < 180


def test_c3_structure():
    d = synth.c3(scale=0.0004, special=500)
    n_a = d["a_lon"].size
    assert n_a == 20_000 and d["b_lon"].size == 80_000
    assert np.sum(d["a_lat"] > 89.5) >= 500 and np.sum(d["a_lat"] < -89.5) >= 500
    assert np.sum((d["a_lon"] < 0.5) | (d["a_lon"] > 359.5)) >= 500
    assert np.unique(d["a_id"]).size == n_a and np.unique(d["b_id"]).size == d["b_lon"].size
    # plane-to-pole contrast of 1 + 9 exp(-|b|/10 deg)
    lat = np.abs(d["b_lat"])
    dens_plane = np.sum(lat < 5) / np.sin(np.radians(5))
    dens_high = np.sum((lat > 60) & (lat < 85)) / (np.sin(np.radians(85)) - np.sin(np.radians(60)))
    assert 4.0 < dens_plane / dens_high < 9.0
