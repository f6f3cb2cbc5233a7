"""The bench's roofline object on CPU: the dominant kernel is the one with
the most time, achieved = algorithmic bytes per launch / its mean launch
time, frac = achieved / the peak, and a DRAM-traffic record is reported only
for the kernel sources it was taken on."""

import json

import pytest

import bench

REGION = dict(shape=0, a=2.0)  # fixed circles, as the all-sky workload


def test_dominant_kernel_and_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "load_peaks", lambda: {"hbm_gbs": 6000.0, "_source": "measured"})
    monkeypatch.setattr(bench, "traffic_record", lambda k: 1.5e7 if k == "k_onesweep" else None)
    steps, n_a, n_b = 2, 1000, 5_000_000
    # two steps, four planned passes over n_b keys each, five launches a step
    st = {"sort_key_passes": steps * 4 * n_b, "sort_pay_passes": steps * 4 * n_b,
          "candidates": 40_000}
    prof = {"k_onesweep": (0.5, 10), "k_scan_fp32_count": (0.3, 2), "k_gather_b": (0.1, 2)}
    r = bench.roofline(prof, st, steps, n_a, n_b, total_ms=2.0, region=REGION)
    assert r["kernel"] == "k_onesweep"
    # 8 B key + 4 B row + 8 B offsets, read and written, per key and pass
    alg = 40.0 * steps * 4 * n_b / 10
    assert r["algorithmic_bytes"] == pytest.approx(alg)
    assert r["ms_per_launch"] == pytest.approx(0.05)
    assert r["achieved"] == pytest.approx(alg / 0.05e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert r["share_of_step"] == pytest.approx(0.25)
    assert r["launches_per_step"] == pytest.approx(5.0)
    assert r["traffic"] == 1.5e7 and r["peak_source"] == "of measured"

    # the count pass dominating: per A 16 B position + 16 B best (fixed
    # circles: no region column), per candidate 12 B
    prof["k_scan_fp32_count"] = (0.9, 2)
    r = bench.roofline(prof, st, steps, n_a, n_b, total_ms=2.0, region=REGION)
    assert r["kernel"] == "k_scan_fp32_count"
    assert r["algorithmic_bytes"] == pytest.approx(n_a * 32 + 40_000 / steps * 12)
    assert r["traffic"] is None
    # per-source ellipses read three float64 columns more per A
    r = bench.roofline(prof, st, steps, n_a, n_b, total_ms=2.0,
                       region=dict(shape=1, a_col=[1.0], b_col=[1.0], pa_col=[0.0]))
    assert r["algorithmic_bytes"] == pytest.approx(n_a * 56 + 40_000 / steps * 12)

    # a kernel without an algorithmic figure: no fraction is claimed
    prof["k_other"] = (5.0, 1)
    r = bench.roofline(prof, st, steps, n_a, n_b, total_ms=8.0, region=REGION)
    assert r["kernel"] == "k_other" and r["achieved"] is None and r["frac"] is None
    assert bench.roofline({}, st, steps, n_a, n_b, 1.0, REGION) is None


def test_fallback_peak_is_named(monkeypatch):
    monkeypatch.setattr(bench, "load_peaks", lambda: {"hbm_gbs": 6800.0, "_source": "fallback"})
    r = bench.roofline({"k_gather_b": (0.2, 2)}, {"sort_key_passes": 0, "sort_pay_passes": 0,
                                                   "candidates": 0}, 2,
                       10, 1000, 1.0, REGION)
    assert r["peak_source"] == "of fallback" and r["peak"] == 6800.0
    assert r["algorithmic_bytes"] == 1000 * 36


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    h = bench.source_hash("k_onesweep")
    (prof_dir / "traffic.json").write_text(json.dumps({
        "k_onesweep": {"source_hash": h, "dram_bytes_per_launch": 123.0},
        "k_gather_b": {"source_hash": "0" * 16, "dram_bytes_per_launch": 456.0}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # (source_hash reads the kernel sources under ROOT: keep the real ones)
    monkeypatch.setattr(bench, "source_hash", lambda k: h if k == "k_onesweep" else "f" * 16)
    assert bench.traffic_record("k_onesweep") == 123.0
    assert bench.traffic_record("k_gather_b") is None  # taken on other sources
    assert bench.traffic_record("k_scan_fp32_count") is None  # no record
