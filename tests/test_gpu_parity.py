"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Member sets must be identical (bit-exact indices, canonical order), the
separations within 1e-4 arcsec, best pairs identical, join rows identical.
Both arithmetic paths are checked: FP32 with float64 recheck, and FP64.
Candidates the oracle flags as borderline (decision margin < 1e-9) would be
excluded; every fixed seed here has none, which the tests assert.
"""

import numpy as np
import pytest

import oracle
from paper_1611_08494_gb300 import synth

pytestmark = pytest.mark.gpu
SEP_TOL = 1e-4  # arcsec
PRECS = ["fp32", "fp64"]


@pytest.fixture(scope="module")
def xm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_08494_gb300 import xm as mod

    return mod


def _cuda(x):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _prec(xm, p):
    return xm.PREC_FP32 if p == "fp32" else xm.PREC_FP64


def _host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def _region_kw(region, xm_side):
    kw = dict(region)
    if xm_side:
        for k in ("a_col", "b_col", "pa_col"):
            if k in kw and kw[k] is not None:
                kw[k] = _cuda(kw[k])
    return kw


def check_pairs(res, ref, subset=None):
    a, b, s = _host(res.a_row), _host(res.b_row), _host(res.sep)
    if subset is not None:
        keep = np.isin(a, subset)
        a, b, s = a[keep], b[keep], s[keep]
    assert ref["border_a"].size == 0, "fixed seed has borderline candidates"
    np.testing.assert_array_equal(a, ref["a_row"])
    np.testing.assert_array_equal(b, ref["b_row"])
    if s.size:
        assert np.max(np.abs(s - ref["sep"])) <= SEP_TOL


def check_best(res, ref, n_a, subset=None):
    bb = oracle.best(ref, n_a)
    assert bb["near_tie"].size == 0
    got_b, got_s = _host(res.best_b), _host(res.best_sep)
    rows = np.arange(n_a) if subset is None else np.asarray(subset)
    np.testing.assert_array_equal(got_b[rows], bb["best_b"][rows])
    has = bb["best_b"][rows] >= 0
    assert np.all(np.isnan(got_s[rows][~has]))
    if has.any():
        assert np.max(np.abs(got_s[rows][has] - bb["best_sep"][rows][has])) <= SEP_TOL


def run(xm, d, prec, zone_height=0.0, fp64_index=True, selection=None, device_input=True,
        a_order=0):
    conv = _cuda if device_input else np.asarray
    idx = xm.Index(conv(d["b_lon"]), conv(d["b_lat"]), frame=d["b_frame"],
                   zone_height_arcsec=zone_height, build_fp64=fp64_index)
    kw = _region_kw(d["region"], device_input)
    res = xm.Result(idx, conv(d["a_lon"]), conv(d["a_lat"]), frame=d["a_frame"],
                    precision=_prec(xm, prec), a_order=a_order,
                    selection=selection or (xm.SEL_ALL | xm.SEL_BEST), **kw)
    return idx, res


def oracle_ref(d, subset=None):
    return oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], a_frame=d["a_frame"],
                        b_frame=d["b_frame"], subset=subset, **d["region"])


# ------------------------------------------------------------------ C1

@pytest.fixture(scope="module")
def c1():
    d = synth.c1()
    return d, oracle_ref(d)


@pytest.mark.parametrize("prec", PRECS)
def test_c1_all_and_best(xm, c1, prec):
    d, ref = c1
    _, res = run(xm, d, prec)
    assert res.n_pairs == ref["a_row"].size
    check_pairs(res, ref)
    check_best(res, ref, d["a_lon"].size)
    np.testing.assert_array_equal(_host(res.count),
                                  np.bincount(ref["a_row"], minlength=d["a_lon"].size))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("selection", ["all", "best"])
def test_c1_joins(xm, c1, prec, selection):
    d, ref = c1
    _, res = run(xm, d, prec)
    n_a, n_b = d["a_lon"].size, d["b_lon"].size
    sel = oracle.selected_pairs(ref, n_a, selection)
    for jt in oracle.JOINS:
        rows = res.join(jt, xm.SEL_ALL if selection == "all" else xm.SEL_BEST)
        exp = oracle.join(sel, n_a, n_b, jt)
        np.testing.assert_array_equal(_host(rows.a_row), exp["a_row"], err_msg=jt)
        np.testing.assert_array_equal(_host(rows.b_row), exp["b_row"], err_msg=jt)
        s, es = _host(rows.sep), exp["sep"]
        np.testing.assert_array_equal(np.isnan(s), np.isnan(es))
        ok = ~np.isnan(es)
        if ok.any():
            assert np.max(np.abs(s[ok] - es[ok])) <= SEP_TOL
        assert rows.n_unmatched_a == n_a - np.unique(sel["a_row"]).size
        assert rows.n_unmatched_b == n_b - np.unique(sel["b_row"]).size


def test_c1_host_input_equals_device_input(xm, c1):
    d, ref = c1
    _, res = run(xm, d, "fp32", device_input=False)
    check_pairs(res, ref)


@pytest.mark.parametrize("zone", [1.0, 3.0, 20.0, 600.0])
def test_c1_partition_independence(xm, c1, zone):
    d, ref = c1
    for prec in PRECS:
        _, res = run(xm, d, prec, zone_height=zone)
        check_pairs(res, ref)


# ------------------------------------------------------------------ C2

@pytest.fixture(scope="module")
def c2_small():
    d = synth.c2(scale=0.02)
    return d, oracle_ref(d)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("a_order", [1, 2])
def test_c2_small_ellipses_galactic(xm, c2_small, prec, a_order):
    d, ref = c2_small
    _, res = run(xm, d, prec, a_order=a_order)
    check_pairs(res, ref)
    check_best(res, ref, d["a_lon"].size)


def test_c2_small_without_fp64_index(xm, c2_small):
    d, ref = c2_small
    for prec in PRECS:
        _, res = run(xm, d, prec, fp64_index=False)
        check_pairs(res, ref)


@pytest.mark.slow
def test_c2_full_size_sampled(xm):
    """Full C2 (A = 200,000 ellipses, B = 5,000,000) in the bench's
    configuration; the oracle checks a seeded sample of 4,000 A sources."""
    d = synth.c2()
    n_a = d["a_lon"].size
    sub = np.sort(synth.rng(77).choice(n_a, 4000, replace=False))
    ref = oracle_ref(d, subset=sub)
    results = {}
    for prec in PRECS:
        _, res = run(xm, d, prec)
        check_pairs(res, ref, subset=sub)
        check_best(res, ref, n_a, subset=sub)
        results[prec] = (_host(res.a_row), _host(res.b_row), _host(res.best_b))
    # the two GPU paths agree on every A source, not just the sample
    for k in range(3):
        np.testing.assert_array_equal(results["fp32"][k], results["fp64"][k])


# ------------------------------------------------------- geometry breadth

def _mixed(seed, shape, a_frame=0, b_frame=0):
    g = synth.rng(seed)
    pa_, pb_ = [], []
    for lon0, lat0 in ((0.0, 90.0), (0.0, -90.0), (0.0, 10.0), (200.0, -45.0), (359.99, 0.0)):
        pa_.append(synth.cap(g, 80, lon0, lat0, 0.01))
        pb_.append(synth.cap(g, 160, lon0, lat0, 0.01))
    a_lon = np.concatenate([p[0] for p in pa_]); a_lat = np.concatenate([p[1] for p in pa_])
    b_lon = np.concatenate([p[0] for p in pb_]); b_lat = np.concatenate([p[1] for p in pb_])
    if a_frame == 1:
        a_lon, a_lat = oracle.from_equatorial(a_lon, a_lat, 1)
    if b_frame == 1:
        b_lon, b_lat = oracle.from_equatorial(b_lon, b_lat, 1)
    n = a_lon.size
    a_col = np.exp(g.uniform(np.log(2.0), np.log(40.0), n))
    region = dict(shape=shape, a_col=a_col, b_col=a_col * g.uniform(0.2, 1.0, n),
                  pa_col=g.uniform(-200.0, 400.0, n), pa_zero_deg=12.5, pa_dir=-1,
                  size_scale=0.5, size_unit_arcsec=2.0)
    return dict(a_lon=a_lon, a_lat=a_lat, b_lon=b_lon, b_lat=b_lat, a_frame=a_frame,
                b_frame=b_frame, region=region)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [0, 1, 2])
@pytest.mark.parametrize("frames", [(0, 0), (1, 1), (1, 0), (0, 1)])
def test_shapes_frames_poles_seam(xm, prec, shape, frames):
    d = _mixed(40 + shape, shape, *frames)
    ref = oracle_ref(d)
    assert ref["a_row"].size > 30
    for zone in (5.0, 60.0):
        for a_order in (1, 2):
            _, res = run(xm, d, prec, zone_height=zone, a_order=a_order)
            check_pairs(res, ref)
            check_best(res, ref, d["a_lon"].size)


def _region_points(lon0, lat0, theta_deg, xy):
    rho = np.hypot(xy[:, 0], xy[:, 1]) * synth.ARCSEC
    bearing = np.radians(theta_deg) + np.arctan2(xy[:, 1], xy[:, 0])
    return synth.destination(np.full(len(xy), lon0), np.full(len(xy), lat0), rho, bearing)


def _band_points(g, shape, a, b, n_ang=4):
    """Points at q = 1 +- {1e-3, 1e-5, 1e-7} on a region of semi-axes (a, b)
    (its frame: x along a)."""
    ang = g.uniform(0, 2 * np.pi, n_ang)
    pts = []
    for eps in (1e-3, 1e-5, 1e-7):
        for sgn in (-1, 1):
            f = 1 + sgn * eps
            if shape == 2:  # on the rectangle's edges
                pts += [[a * f, b * 0.5], [a * 0.3, -b * f], [a * f, b * f]]
            else:  # on the ellipse (q = f^2); a circle's points a hair apart in
                # radius, so no two separations tie
                pts += [[a * f * (1 + 1e-8 * k) * np.cos(t), b * f * (1 + 1e-8 * k) * np.sin(t)]
                        for k, t in enumerate(ang)]
    return np.array(pts)


@pytest.mark.parametrize("zone_height", [5.0, 30.0, 120.0])
@pytest.mark.parametrize("shape", [0, 1, 2])
def test_guard_band_stress_fixed_regions(xm, shape, zone_height):
    """The same near-boundary points around fixed regions (2.5 x 1.5 arcsec)
    at three zone heights: at 30 and 120 arcsec the regions are small
    against the zones and the count pass takes its one-lane-per-source form,
    whose guard band hands these cases to its float64 recheck; at 5 arcsec
    the warp-cooperative scan does."""
    g = synth.rng(700 + shape)
    n = 80
    lon0, lat0 = synth.uniform_box(g, n, 0.0, 360.0, -89.9, 89.9)
    a_sz, b_sz = 2.5, (1.5 if shape else 2.5)
    pa = 37.0
    b_lon, b_lat = [], []
    for i in range(n):
        lo, la = _region_points(lon0[i], lat0[i], pa, _band_points(g, shape, a_sz, b_sz))
        b_lon.append(lo); b_lat.append(la)
    d = dict(a_lon=lon0, a_lat=lat0, b_lon=np.concatenate(b_lon), b_lat=np.concatenate(b_lat),
             a_frame=0, b_frame=0, region=dict(shape=shape, a=a_sz, b=b_sz, pa=pa))
    ref = oracle_ref(d)
    xm.reset_stats()
    _, res = run(xm, d, "fp32", zone_height=zone_height)
    check_pairs(res, ref)
    check_best(res, ref, n)
    assert xm.stats()["rechecked"] > 0


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [0, 1, 2])
def test_guard_band_stress(xm, prec, shape):
    """B sources at q = 1 +- {1e-3, 1e-5, 1e-7} around every region: the FP32
    path must hand every near-boundary case to the FP64 recheck."""
    g = synth.rng(500 + shape)
    n = 60
    lon0, lat0 = synth.uniform_box(g, n, 0.0, 360.0, -89.9, 89.9)
    a_sz = np.exp(g.uniform(np.log(0.5), np.log(60.0), n))
    b_sz = a_sz * g.uniform(0.3, 1.0, n) if shape else a_sz
    pa = g.uniform(0.0, 180.0, n)
    b_lon, b_lat = [], []
    for i in range(n):
        ang = g.uniform(0, 2 * np.pi, 12)
        pts = []
        for eps in (1e-3, 1e-5, 1e-7):
            for sgn in (-1, 1):
                f = 1 + sgn * eps
                if shape == 2:  # on the rectangle's edges
                    pts += [[a_sz[i] * f, b_sz[i] * 0.5], [a_sz[i] * 0.3, -b_sz[i] * f],
                            [a_sz[i] * f, b_sz[i] * f]]
                else:  # on the ellipse (q = f^2)
                    pts += [[a_sz[i] * f * np.cos(t), b_sz[i] * f * np.sin(t)] for t in ang[:4]]
        lo, la = _region_points(lon0[i], lat0[i], pa[i], np.array(pts))
        b_lon.append(lo); b_lat.append(la)
    d = dict(a_lon=lon0, a_lat=lat0, b_lon=np.concatenate(b_lon), b_lat=np.concatenate(b_lat),
             a_frame=0, b_frame=0,
             region=dict(shape=shape, a_col=a_sz, b_col=b_sz, pa_col=pa))
    ref = oracle_ref(d)
    _, res = run(xm, d, prec, zone_height=30.0)
    check_pairs(res, ref)


# ------------------------------------------------------------ edge cases

def test_empty_catalogues(xm):
    import torch

    e = torch.empty(0, dtype=torch.float64, device="cuda")
    one = _cuda([10.0])
    for b_lon, b_lat, a_lon, a_lat in ((e, e, one, one), (one, one, e, e), (e, e, e, e)):
        idx = xm.Index(b_lon, b_lat)
        res = xm.Result(idx, a_lon, a_lat, shape=0, a=5.0)
        assert res.n_pairs == 0
        rows = res.join("or")
        assert rows.n == a_lon.numel() + b_lon.numel()


def test_single_source_and_duplicates(xm):
    # duplicates of one B position: every copy is a member; best = lowest row
    b_lon = _cuda([10.0001, 10.0001, 10.0001, 10.0009])
    b_lat = _cuda([0.0, 0.0, 0.0, 0.0])
    for prec in (xm.PREC_FP32, xm.PREC_FP64):
        idx = xm.Index(b_lon, b_lat)
        res = xm.Result(idx, _cuda([10.0]), _cuda([0.0]), precision=prec, shape=0, a=2.0)
        np.testing.assert_array_equal(_host(res.b_row), [0, 1, 2])
        assert _host(res.best_b)[0] == 0
        assert _host(res.best_sep)[0] == pytest.approx(0.36, abs=SEP_TOL)


def test_zero_size_region_matches_nothing(xm):
    idx = xm.Index(_cuda([10.0, 20.0]), _cuda([0.0, 0.0]))
    res = xm.Result(idx, _cuda([10.0, 20.0]), _cuda([0.0, 0.0]), shape=0, a_col=_cuda([0.0, 1.0]))
    np.testing.assert_array_equal(_host(res.a_row), [1])


@pytest.mark.parametrize("bad", ["nan_a", "lat_a", "lat_b", "size"])
def test_invalid_input_is_einval(xm, bad):
    good = _cuda([10.0, 11.0])
    lat = _cuda([0.0, 0.0])
    if bad == "lat_b":
        with pytest.raises(xm.XMError, match="EINVAL"):
            xm.Index(good, _cuda([0.0, 90.5]))
        return
    idx = xm.Index(good, lat)
    kw = dict(shape=0, a=1.0)
    a_lon, a_lat = good, lat
    if bad == "nan_a":
        a_lon = _cuda([np.nan, 1.0])
    elif bad == "lat_a":
        a_lat = _cuda([-91.0, 0.0])
    else:
        kw = dict(shape=0, a_col=_cuda([1.0, -2.0]))
    for a_order in (1, 2):  # found with and without the A sort
        with pytest.raises(xm.XMError, match="EINVAL"):
            xm.Result(idx, a_lon, a_lat, a_order=a_order, **kw)
    if bad == "nan_a":
        with pytest.raises(xm.XMError, match="a_order"):
            xm.Result(idx, good, lat, a_order=3, **dict(shape=0, a=1.0))


@pytest.mark.parametrize("prec", PRECS)
def test_many_members_overflow_and_long_segments(xm, prec):
    """Member lists of every size class reach the canonical order: more than
    2048 (long-segment radix sort), 513..2048 (block sort), 17..512 (warp
    sort) and up to 16 (per-thread sort)."""
    g = synth.rng(9)
    b_lon, b_lat = synth.cap(g, 6000, 45.0, 30.0, 0.05)
    a_lon = np.array([45.0, 45.005, 45.01, 45.02, 44.99])
    a_lat = np.array([30.0, 29.995, 30.01, 30.0, 29.98])
    a_col = np.array([170.0, 70.0, 40.0, 12.0, 5.0])
    d = dict(a_lon=a_lon, a_lat=a_lat, b_lon=b_lon, b_lat=b_lat, a_frame=0, b_frame=0,
             region=dict(shape=0, a_col=a_col))
    ref = oracle_ref(d)
    counts = np.bincount(ref["a_row"], minlength=5)
    assert counts[0] > 2048 and 512 < counts[1] <= 2048 and 16 < counts[2] <= 512
    assert 16 < counts[3] <= 512 and counts[4] <= 16
    for a_order in (1, 2):
        _, res = run(xm, d, prec, zone_height=20.0, a_order=a_order)
        check_pairs(res, ref)
        check_best(res, ref, 5)


# ------------------------------------------------------------------ C3

@pytest.mark.parametrize("prec", PRECS)
def test_c3_scaled_all_sky(xm, prec):
    d = synth.c3(scale=0.002, special=2000)
    ref = oracle_ref(d)
    idx, res = run(xm, d, prec, zone_height=8.0)
    check_pairs(res, ref)
    check_best(res, ref, d["a_lon"].size)
    t = d["truth"]
    got = set(zip(_host(res.a_row).tolist(), _host(res.b_row).tolist()))
    found = np.array([(a, b) in got for a, b in zip(t["a_row"].tolist(), t["b_row"].tolist())])
    np.testing.assert_array_equal(found, t["rho_arcsec"] <= 2.0)


# --------------------------------------- further readings of "best pairs"

def _check_pick(res, ref, n_a, n_b, kind):
    exp = oracle.pick(ref, n_a, n_b, kind)
    assert exp["near_tie_b"].size == 0 and exp["near_tie_a"].size == 0
    rows = res.pick(kind)
    np.testing.assert_array_equal(_host(rows.a_row), exp["a_row"])
    np.testing.assert_array_equal(_host(rows.b_row), exp["b_row"])
    if exp["sep"].size:
        assert np.max(np.abs(_host(rows.sep) - exp["sep"])) <= SEP_TOL
    return exp["a_row"].size


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", ["best_b", "mutual"])
def test_pick_c1_c2(xm, c1, c2_small, prec, kind):
    for d, ref in (c1, c2_small):
        for a_order in (1, 2):  # the sorted order keeps a row -> slot map
            _, res = run(xm, d, prec, a_order=a_order)
            assert _check_pick(res, ref, d["a_lon"].size, d["b_lon"].size, kind) > 100


@pytest.mark.parametrize("prec", PRECS)
def test_pick_near_ties_decided_in_float64(xm, prec):
    """B sources between two A sources, closer to one by 1e-6 to 1e-5 arcsec:
    inside the float32 error band, so the choice is made in float64."""
    half = 0.5 / 3600.0
    a_lon, a_lat, b_lon, b_lat = [], [], [], []
    for k, delta in enumerate([1e-6, -1e-6, 3e-6, -5e-6, 1e-5, -2e-5, 4e-5, -8e-5]):
        lon0, lat0 = 20.0 + 0.01 * k, -30.0 + 0.02 * k
        a_lon += [lon0 - half / np.cos(np.radians(lat0)), lon0 + half / np.cos(np.radians(lat0))]
        a_lat += [lat0, lat0]
        b_lon.append(lon0 + delta / 3600.0 / np.cos(np.radians(lat0)))
        b_lat.append(lat0)
    d = dict(a_lon=np.array(a_lon), a_lat=np.array(a_lat), b_lon=np.array(b_lon),
             b_lat=np.array(b_lat), a_frame=0, b_frame=0, region=dict(shape=0, a=1.0))
    ref = oracle_ref(d)
    assert ref["a_row"].size == 16  # every B lies in both regions
    _, res = run(xm, d, prec)
    for kind in ("best_b", "mutual"):
        _check_pick(res, ref, d["a_lon"].size, d["b_lon"].size, kind)


def test_pick_needs_the_selections(xm, c1):
    d, _ = c1
    _, res = run(xm, d, "fp32", selection=xm.SEL_BEST)
    with pytest.raises(xm.XMError, match="EINVAL"):
        res.pick("best_b")
    _, res = run(xm, d, "fp32", selection=xm.SEL_ALL)
    res.pick("best_b")
    with pytest.raises(xm.XMError, match="EINVAL"):
        res.pick("mutual")


def test_deferred_index_check(xm):
    """A build with the check deferred returns at once; invalid B positions
    then fail the match (and the batch) that uses the index."""
    good = _cuda([10.0, 11.0, 12.0])
    lat_bad = _cuda([0.0, np.nan, 0.0])
    idx = xm.Index(good, lat_bad, deferred_check=True)
    with pytest.raises(xm.XMError, match="EINVAL.*B:"):
        xm.Result(idx, good, _cuda([0.0, 0.0, 0.0]), shape=0, a=1.0)
    with pytest.raises(xm.XMError, match="EINVAL"):
        xm.Batch(idx, [dict(lon=good, lat=_cuda([0.0, 0.0, 0.0]), a=1.0)])
    # a clean deferred build matches like a checked one
    d = synth.c1()
    ref = oracle_ref(d)
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]), deferred_check=True)
    res = xm.Result(idx, _cuda(d["a_lon"]), _cuda(d["a_lat"]), **d["region"])
    check_pairs(res, ref)


# ------------------------------------------------- planned index sort

PLAN_CASES = {  # centre lon, lat, half-widths in lon and lat (deg), most passes
    "patch": (150.0, 30.0, 0.3, 0.3, 4),
    "seam": (0.0, -20.0, 0.3, 0.3, 5),
    "two_zones": (77.0, 0.0, 0.5, 1.5e-3, 4),
    "pole": (None, 90.0, None, 0.05, 5),
}


@pytest.mark.parametrize("case", ["identical"] + list(PLAN_CASES))
def test_index_sort_plan(xm, case):
    """The index sort skips digit passes over key bits that no B source
    varies (zone range, RA bits above their spread); the index must be the
    one a full sort gives, so the matches equal the oracle's, and the passes
    counted are whole passes over B."""
    g = synth.rng(900 + len(case))
    n_b = 300_001  # 74 sort tiles, the last one ragged
    if case == "identical":
        b_lon, b_lat = np.full(n_b, 123.456), np.full(n_b, -7.5)
        # on the point, 1.9 arcsec and 2.1 arcsec away (radius 2 arcsec)
        a_lon = np.array([123.456, 123.456, 123.456])
        a_lat = np.array([-7.5, -7.5 + 1.9 / 3600, -7.5 - 2.1 / 3600])
        max_passes = 0
    else:
        c_lon, c_lat, w_lon, w_lat, max_passes = PLAN_CASES[case]
        if c_lon is None:  # a cap around the pole, every RA
            b_lon = g.uniform(0, 360, n_b)
            b_lat = c_lat - g.uniform(0, w_lat, n_b)
        else:
            b_lon = np.mod(c_lon + g.uniform(-w_lon, w_lon, n_b), 360.0)
            b_lat = c_lat + g.uniform(-w_lat, w_lat, n_b)
        a_lon = np.mod(b_lon[::100] + g.normal(0, 3e-4, b_lon[::100].size), 360.0)
        a_lat = b_lat[::100].copy()
    d = dict(a_lon=a_lon, a_lat=a_lat, b_lon=b_lon, b_lat=b_lat, a_frame=0, b_frame=0,
             region=dict(shape=0, a=2.0))
    ref = oracle_ref(d)
    for prec in PRECS:
        xm.reset_stats()
        idx = xm.Index(_cuda(b_lon), _cuda(b_lat), zone_height_arcsec=12.0,
                       build_fp64=prec == "fp64")
        keys = xm.stats()["sort_key_passes"]  # the index sort's alone
        assert keys % n_b == 0 and keys // n_b <= max_passes
        assert xm.stats()["sort_pay_passes"] == keys  # each key carries its offsets
        res = xm.Result(idx, _cuda(a_lon), _cuda(a_lat), precision=_prec(xm, prec), shape=0,
                        a=2.0, selection=xm.SEL_ALL | xm.SEL_BEST)
        check_pairs(res, ref)
        if case == "identical":
            # every B source is a member of the first two; best: lowest B row
            assert list(_host(res.best_b)) == [0, 0, -1]
        else:
            check_best(res, ref, a_lon.size)


def test_large_host_input_equals_device_input(xm):
    """B of 5e6 and A from host memory (A copied and prepared on a side
    stream beside the build): the results equal those from device columns."""
    import torch

    d = synth.c2(scale=1.0)
    out = {}
    for dev in (True, False):
        conv = _cuda if dev else (lambda x: torch.as_tensor(np.ascontiguousarray(x)).pin_memory())
        idx = xm.Index(conv(d["b_lon"]), conv(d["b_lat"]), frame=d["b_frame"], zone_height_arcsec=12.0,
                       deferred_check=True)
        reg = {k: (conv(v) if isinstance(v, np.ndarray) else v) for k, v in d["region"].items()}
        res = xm.Result(idx, conv(d["a_lon"]), conv(d["a_lat"]), frame=d["a_frame"], **reg)
        out[dev] = [_host(t) for t in (res.a_row, res.b_row, res.sep, res.best_b)]
    for x, y in zip(out[True], out[False]):
        np.testing.assert_array_equal(x, y)
    assert out[True][0].size > 1_000_000
