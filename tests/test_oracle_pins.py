"""Pins of the FP64 oracle to facts outside itself (no GPU).

Each test checks the oracle against something it does not compute itself:
brute force, planted truths drawn by the generator, closed forms, published
frame constants, symmetries and set identities of paper §2.2.
"""

import os

import numpy as np
import pytest

import oracle
from paper_1611_08494_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ARCSEC_DEG = 1.0 / 3600.0


def _pairs(r):
    return set(zip(r["a_row"].tolist(), r["b_row"].tolist()))


# ------------------------------------------------------------- pruning --

def _random_mixed(seed, n_a=300, n_b=600):
    """Tiny catalogues crowded around hard places: both poles, the RA 0/360
    seam and an ordinary field, so a few arcsec regions catch members."""
    g = synth.rng(seed)
    parts_a, parts_b = [], []
    for lon0, lat0 in ((0.0, 90.0), (0.0, -90.0), (0.0, 10.0), (200.0, -45.0)):
        parts_a.append(synth.cap(g, n_a // 4, lon0, lat0, 0.01))
        parts_b.append(synth.cap(g, n_b // 4, lon0, lat0, 0.01))
    a_lon = np.concatenate([p[0] for p in parts_a]); a_lat = np.concatenate([p[1] for p in parts_a])
    b_lon = np.concatenate([p[0] for p in parts_b]); b_lat = np.concatenate([p[1] for p in parts_b])
    n = a_lon.size
    cols = dict(a_col=np.exp(g.uniform(np.log(2.0), np.log(40.0), n)),
                pa_col=g.uniform(-200.0, 400.0, n))
    cols["b_col"] = cols["a_col"] * g.uniform(0.2, 1.0, n)
    return a_lon, a_lat, b_lon, b_lat, cols


@pytest.mark.parametrize("shape", [oracle.CIRCLE, oracle.ELLIPSE, oracle.RECT])
@pytest.mark.parametrize("frames", [(0, 0), (1, 1), (1, 0), (0, 1)])
def test_grid_equals_brute_force(shape, frames):
    a_lon, a_lat, b_lon, b_lat, cols = _random_mixed(7 + shape)
    # the catalogues are drawn in one frame; a galactic one is re-expressed so
    # both still cover the same sky
    if frames[0] == oracle.GAL:
        a_lon, a_lat = oracle.from_equatorial(a_lon, a_lat, oracle.GAL)
    if frames[1] == oracle.GAL:
        b_lon, b_lat = oracle.from_equatorial(b_lon, b_lat, oracle.GAL)
    kw = dict(shape=shape, a_frame=frames[0], b_frame=frames[1], pa_zero_deg=12.5, pa_dir=-1,
              size_scale=0.5, **cols)
    g = oracle.match(a_lon, a_lat, b_lon, b_lat, mode="grid", **kw)
    b = oracle.match(a_lon, a_lat, b_lon, b_lat, mode="brute", **kw)
    assert g["a_row"].size > 20  # the case is not vacuous
    np.testing.assert_array_equal(g["a_row"], b["a_row"])
    np.testing.assert_array_equal(g["b_row"], b["b_row"])
    np.testing.assert_array_equal(g["sep"], b["sep"])
    # canonical order
    key = g["a_row"] * (b_lon.size + 1) + g["b_row"]
    assert np.all(np.diff(key) > 0)


def test_grid_finds_rectangle_corners():
    # a rectangle reaches sqrt(a^2 + b^2) from its centre; members sitting
    # just inside the corners must survive the pruning at any orientation
    g = synth.rng(21)
    n = 400
    a_lon, a_lat = synth.uniform_box(g, n, 0.0, 360.0, -89.0, 89.0)
    pa = g.uniform(0.0, 180.0, n)
    a, b = 10.0, 10.0
    corners = np.array([[a, b], [-a, b], [a, -b], [-a, -b]]) * 0.9999
    b_lon, b_lat = [], []
    for i in range(n):
        lo, la = _region_points(a_lon[i], a_lat[i], pa[i], corners)
        b_lon.append(lo); b_lat.append(la)
    b_lon, b_lat = np.concatenate(b_lon), np.concatenate(b_lat)
    kw = dict(shape=oracle.RECT, a=a, b=b, pa_col=pa)
    gr = oracle.match(a_lon, a_lat, b_lon, b_lat, **kw)
    br = oracle.match(a_lon, a_lat, b_lon, b_lat, mode="brute", **kw)
    assert _pairs(gr) == _pairs(br)
    assert {(i, 4 * i + k) for i in range(n) for k in range(4)} <= _pairs(gr)


def test_subset_equals_full():
    a_lon, a_lat, b_lon, b_lat, cols = _random_mixed(3)
    full = oracle.match(a_lon, a_lat, b_lon, b_lat, shape=oracle.ELLIPSE, **cols)
    sub = np.arange(0, a_lon.size, 7)
    part = oracle.match(a_lon, a_lat, b_lon, b_lat, shape=oracle.ELLIPSE, subset=sub, **cols)
    keep = np.isin(full["a_row"], sub)
    np.testing.assert_array_equal(full["a_row"][keep], part["a_row"])
    np.testing.assert_array_equal(full["b_row"][keep], part["b_row"])


# -------------------------------------------------------- planted truth --

def test_planted_truth_c1():
    d = synth.c1()
    r = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], **d["region"])
    t = d["truth"]
    got = _pairs(r)
    found = np.array([(a, b) in got for a, b in zip(t["a_row"].tolist(), t["b_row"].tolist())])
    # every planted pair is a member exactly when its true offset is <= r
    # (no generated offset lies within 1e-6 of the radius)
    assert np.min(np.abs(t["rho_arcsec"] - 1.0)) > 1e-6
    np.testing.assert_array_equal(found, t["rho_arcsec"] <= 1.0)
    # recall of a 2-D Gaussian offset inside r: 1 - exp(-r^2 / 2 sigma^2)
    p = 1.0 - np.exp(-1.0 / (2 * 0.3 ** 2))
    n = found.size
    assert abs(found.sum() - n * p) < 5 * np.sqrt(n * p * (1 - p))
    # separations of planted pairs equal the drawn offsets
    sep = {k: s for k, s in zip(zip(r["a_row"].tolist(), r["b_row"].tolist()), r["sep"].tolist())}
    err = [abs(sep[(a, b)] - rho) for a, b, rho in
           zip(t["a_row"].tolist(), t["b_row"].tolist(), t["rho_arcsec"].tolist()) if (a, b) in sep]
    assert max(err) < 1e-8
    # chance matches: B surface density x circle area, per A (Poisson, 5 sigma)
    area_deg2 = np.degrees(1.0) * (np.sin(np.radians(3.0)) - np.sin(np.radians(2.0)))
    dens_b = d["b_lon"].size / area_deg2
    expect = d["a_lon"].size * dens_b * np.pi * (1.0 * ARCSEC_DEG) ** 2
    extra = r["a_row"].size - found.sum()
    assert abs(extra - expect) < 5 * np.sqrt(expect) + 3
    assert r["border_a"].size == 0


# ----------------------------------------------------------- symmetries --

def test_circle_symmetry():
    d = synth.c1()
    ab = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], a=1.0)
    ba = oracle.match(d["b_lon"], d["b_lat"], d["a_lon"], d["a_lat"], a=1.0)
    assert _pairs(ab) == {(b, a) for a, b in _pairs(ba)}


def _rotate(lon, lat, rot):
    l, b = np.radians(lon), np.radians(lat)
    p = np.stack([np.cos(b) * np.cos(l), np.cos(b) * np.sin(l), np.sin(b)])
    q = rot @ p
    return np.degrees(np.arctan2(q[1], q[0])) % 360.0, np.degrees(np.arctan2(q[2], np.hypot(q[0], q[1])))


def test_rotation_invariance_circles():
    a_lon, a_lat, b_lon, b_lat, _ = _random_mixed(11)
    g = synth.rng(99)
    qm, _ = np.linalg.qr(g.normal(size=(3, 3)))
    if np.linalg.det(qm) < 0:
        qm[:, 0] = -qm[:, 0]
    r0 = oracle.match(a_lon, a_lat, b_lon, b_lat, a=25.0)
    ra_lon, ra_lat = _rotate(a_lon, a_lat, qm)
    rb_lon, rb_lat = _rotate(b_lon, b_lat, qm)
    r1 = oracle.match(ra_lon, ra_lat, rb_lon, rb_lat, a=25.0)
    assert r0["a_row"].size > 50
    assert r0["border_a"].size == 0
    np.testing.assert_array_equal(r0["a_row"], r1["a_row"])
    np.testing.assert_array_equal(r0["b_row"], r1["b_row"])
    np.testing.assert_allclose(r0["sep"], r1["sep"], atol=1e-9)


# ---------------------------------------------------------- closed forms --

def test_golden_equator_meridian():
    rows = np.loadtxt(os.path.join(GOLDEN, "equator_meridian.txt"))
    for a_ra, a_dec, b_ra, b_dec, sep, member in rows:
        assert oracle.separation(a_ra, a_dec, 0, b_ra, b_dec, 0) == pytest.approx(sep, abs=1e-6)
        r = oracle.match([a_ra], [a_dec], [b_ra], [b_dec], a=1.5)
        assert r["a_row"].size == int(member)
        if member:
            assert r["sep"][0] == pytest.approx(sep, abs=1e-6)


def _region_points(lon0, lat0, theta_deg, xy_arcsec):
    """Positions whose azimuthal-equidistant region coordinates about
    (lon0, lat0) are (X, Y): X along the major axis at bearing theta, Y
    towards bearing theta + 90 deg."""
    x, y = xy_arcsec[:, 0], xy_arcsec[:, 1]
    rho = np.hypot(x, y) * synth.ARCSEC
    bearing = np.radians(theta_deg) + np.arctan2(y, x)
    return synth.destination(np.full(x.size, lon0), np.full(x.size, lat0), rho, bearing)


@pytest.mark.parametrize("lat0", [0.0, -48.0, 89.9999])
def test_circle_boundary(lat0):
    r = 7.0
    eps = 1e-8  # the constructed offsets carry ~1e-11 relative error
    bearings = np.linspace(0.0, 360.0, 13)[:-1]
    xy = np.concatenate([np.stack([r * (1 - eps) * np.cos(np.radians(bearings)),
                                   r * (1 - eps) * np.sin(np.radians(bearings))], 1),
                         np.stack([r * (1 + eps) * np.cos(np.radians(bearings)),
                                   r * (1 + eps) * np.sin(np.radians(bearings))], 1)])
    lon, lat = _region_points(45.0, lat0, 0.0, xy)
    res = oracle.match([45.0], [lat0], lon, lat, a=r)
    np.testing.assert_array_equal(res["b_row"], np.arange(12))
    np.testing.assert_allclose(res["sep"], r * (1 - eps), rtol=1e-10)


@pytest.mark.parametrize("lat0", [0.0, 37.0, -89.99, 89.995])
def test_ellipse_axes_and_orientation(lat0):
    a, b, pa = 20.0, 6.0, 30.0
    eps = 1e-8
    xy = np.array([[a * (1 - eps), 0], [a * (1 + eps), 0], [-a * (1 - eps), 0], [-a * (1 + eps), 0],
                   [0, b * (1 - eps)], [0, b * (1 + eps)], [0, -b * (1 - eps)], [0, -b * (1 + eps)],
                   [b * 1.01, a * 0.5], [a * 0.6, b * 0.79], [a * 0.6, b * 0.81]])
    # expected from the construction: inside iff (X/a)^2 + (Y/b)^2 <= 1
    expect = (xy[:, 0] / a) ** 2 + (xy[:, 1] / b) ** 2 <= 1.0
    lon, lat = _region_points(123.0, lat0, pa, xy)
    r = oracle.match([123.0], [lat0], lon, lat, shape=oracle.ELLIPSE, a=a, b=b, pa=pa)
    got = np.zeros(len(xy), bool)
    got[r["b_row"]] = True
    np.testing.assert_array_equal(got, expect)


@pytest.mark.parametrize("lat0", [0.0, -60.0, 89.999])
def test_rectangle_corners(lat0):
    a, b, pa = 15.0, 4.0, 110.0
    eps = 1e-8
    xy = np.array([[a * (1 - eps), b * (1 - eps)], [a * (1 + eps), b * (1 - eps)],
                   [a * (1 - eps), b * (1 + eps)], [-a * (1 - eps), -b * (1 - eps)],
                   [-a * (1 - eps), b * (1 + eps)], [a * 0.99, -b * 0.99], [0.0, b * 1.001]])
    expect = (np.abs(xy[:, 0]) <= a) & (np.abs(xy[:, 1]) <= b)
    lon, lat = _region_points(300.0, lat0, pa, xy)
    r = oracle.match([300.0], [lat0], lon, lat, shape=oracle.RECT, a=a, b=b, pa=pa)
    got = np.zeros(len(xy), bool)
    got[r["b_row"]] = True
    np.testing.assert_array_equal(got, expect)


def test_orientation_identities():
    a_lon, a_lat, b_lon, b_lat, cols = _random_mixed(5)
    base = dict(a_col=cols["a_col"], b_col=cols["b_col"])
    pa = cols["pa_col"]
    for shape in (oracle.ELLIPSE, oracle.RECT):
        ref = _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, shape=shape, pa_col=pa, **base))
        assert len(ref) > 20
        # PA + 180 deg leaves the region unchanged
        assert ref == _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, shape=shape,
                                          pa_col=pa + 180.0, **base))
        # PA + 90 deg with the axes swapped is the same region
        assert ref == _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, shape=shape,
                                          pa_col=pa + 90.0, a_col=base["b_col"],
                                          b_col=base["a_col"]))
        # direction -1 with PA equals direction +1 with -PA
        assert ref == _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, shape=shape, pa_dir=-1,
                                          pa_col=-pa, **base))
        # a zero-point shift is a PA shift
        assert ref == _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, shape=shape, pa_zero_deg=40.0,
                                          pa_col=pa - 40.0, **base))
    # an ellipse with equal axes is the circle
    circ = _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, a_col=cols["a_col"]))
    ell = _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, shape=oracle.ELLIPSE, a_col=cols["a_col"],
                              b_col=cols["a_col"], pa_col=pa))
    assert circ == ell


def test_size_scale_and_unit():
    a_lon, a_lat, b_lon, b_lat, cols = _random_mixed(6)
    ref = _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, a_col=cols["a_col"]))
    # FWHM column with scale 0.5, in arcmin
    alt = _pairs(oracle.match(a_lon, a_lat, b_lon, b_lat, a_col=cols["a_col"] * 2 / 60.0,
                              size_scale=0.5, size_unit_arcsec=60.0))
    assert ref == alt


# --------------------------------------------------------------- frames --

def test_frame_constants_golden():
    with open(os.path.join(GOLDEN, "galactic_frame.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for _, lon, lat, fr, lon2, lat2, fr2, tol in rows:
        lon, lat, lon2, lat2, tol = map(float, (lon, lat, lon2, lat2, tol))
        if fr == "gal":
            ra, dec = oracle.to_equatorial([lon], [lat], oracle.GAL)
        else:
            ra, dec = oracle.from_equatorial([lon], [lat], oracle.GAL)
        assert ra[0] == pytest.approx(lon2, abs=tol)
        assert dec[0] == pytest.approx(lat2, abs=tol)


def test_frame_matrix_orthonormal():
    m = oracle.gal_to_eq_matrix()
    np.testing.assert_allclose(m @ m.T, np.eye(3), atol=1e-15)
    assert np.linalg.det(m) == pytest.approx(1.0, abs=1e-15)


def test_frame_round_trip():
    g = synth.rng(4)
    ra, dec = synth.uniform_box(g, 20000, 0.0, 360.0, -90.0, 90.0)
    ra = np.concatenate([ra, [0.0, 359.9999999, 10.0, 10.0]])
    dec = np.concatenate([dec, [0.0, 0.0, 90.0, -90.0]])
    lon, lat = oracle.from_equatorial(ra, dec, oracle.GAL)
    ra2, dec2 = oracle.to_equatorial(lon, lat, oracle.GAL)
    seps = np.array([oracle.separation(a, b, 0, c, d, 0) for a, b, c, d in zip(ra, dec, ra2, dec2)])
    assert seps.max() * synth.ARCSEC < 1e-12


def test_galactic_position_angle_counts_from_galactic_north():
    # an ellipse given in galactic coordinates with PA 0 has its major axis
    # towards galactic north, wherever it sits
    l0, b0 = 33.0, 20.0
    xy = np.array([[9.99, 0.0], [10.01, 0.0], [0.0, 2.5], [0.0, 1.9]])
    lon, lat = _region_points(l0, b0, 0.0, xy)  # built in the galactic frame
    r = oracle.match([l0], [b0], lon, lat, shape=oracle.ELLIPSE, a=10.0, b=2.0, pa=0.0,
                     a_frame=oracle.GAL, b_frame=oracle.GAL)
    np.testing.assert_array_equal(r["b_row"], [0, 3])
    # B given in equatorial coordinates: same members
    ra, dec = oracle.to_equatorial(lon, lat, oracle.GAL)
    r2 = oracle.match([l0], [b0], ra, dec, shape=oracle.ELLIPSE, a=10.0, b=2.0, pa=0.0,
                      a_frame=oracle.GAL, b_frame=oracle.EQ)
    np.testing.assert_array_equal(r2["b_row"], [0, 3])
    np.testing.assert_allclose(r2["sep"], r["sep"], atol=1e-8)


# ------------------------------------------------------- validity rules --

@pytest.mark.parametrize("bad", [dict(a_lat=[91.0]), dict(a_lat=[np.nan]), dict(a_lon=[np.inf]),
                                 dict(b_lat=[-90.5]), dict(a_col=[-1.0])])
def test_invalid_input_rejected(bad):
    kw = dict(a_lon=[10.0], a_lat=[0.0], b_lon=[10.0], b_lat=[0.0])
    cols = {k: v for k, v in bad.items() if k == "a_col"}
    kw.update({k: v for k, v in bad.items() if k != "a_col"})
    with pytest.raises(oracle.OracleError):
        oracle.match(kw["a_lon"], kw["a_lat"], kw["b_lon"], kw["b_lat"], **cols)


def test_zero_size_matches_nothing():
    r = oracle.match([10.0, 10.0], [0.0, 0.0], [10.0], [0.0], a_col=[0.0, 1.0])
    np.testing.assert_array_equal(r["a_row"], [1])


def test_ra_normalisation():
    r1 = oracle.match([-0.0001], [5.0], [359.9999, 0.0002], [5.0], a=1.5)
    r2 = oracle.match([359.9999], [5.0], [-0.0001, 360.0002], [5.0], a=1.5)
    np.testing.assert_array_equal(r1["b_row"], [0])
    np.testing.assert_array_equal(r2["b_row"], [0])


# ------------------------------------------------- selection and joins --

@pytest.fixture(scope="module")
def c1_result():
    d = synth.c1()
    r = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], a=3.0)  # crowded enough for ties
    return d, r


def test_best_is_argmin_of_all(c1_result):
    d, r = c1_result
    n_a = d["a_lon"].size
    bb = oracle.best(r, n_a)
    sel = oracle.selected_pairs(r, n_a, "best")
    assert _pairs(sel) <= _pairs(r)
    # one pair per A source that has members
    np.testing.assert_array_equal(sel["a_row"], np.unique(r["a_row"]))
    for i in np.unique(r["a_row"])[:2000]:
        m = r["a_row"] == i
        j = np.lexsort((r["b_row"][m], r["sep"][m]))[0]
        assert bb["best_b"][i] == r["b_row"][m][j]
    assert np.all(bb["best_b"][np.setdiff1d(np.arange(n_a), r["a_row"])] == -1)
    assert bb["near_tie"].size == 0


def test_best_tie_goes_to_lowest_b_row():
    # two identical B positions: the lower row wins
    r = oracle.match([10.0], [0.0], [10.0001, 10.0001, 10.0002], [0.0, 0.0, 0.0], a=2.0)
    bb = oracle.best(r, 1)
    assert bb["best_b"][0] == 0


@pytest.mark.parametrize("selection", ["all", "best"])
def test_join_identities(c1_result, selection):
    d, r = c1_result
    n_a, n_b = d["a_lon"].size, d["b_lon"].size
    sel = oracle.selected_pairs(r, n_a, selection)
    J = {t: oracle.join(sel, n_a, n_b, t) for t in oracle.JOINS}
    un_a = np.setdiff1d(np.arange(n_a), sel["a_row"])
    un_b = np.setdiff1d(np.arange(n_b), sel["b_row"])
    assert J["and"]["a_row"].size == sel["a_row"].size
    assert J["or"]["a_row"].size == sel["a_row"].size + un_a.size + un_b.size
    np.testing.assert_array_equal(J["not1_2"]["a_row"], un_a)
    np.testing.assert_array_equal(J["not2_1"]["b_row"], un_b)
    np.testing.assert_array_equal(J["xor"]["a_row"][: un_a.size], un_a)
    np.testing.assert_array_equal(J["xor"]["b_row"][un_a.size:], un_b)
    rows = lambda x: set(zip(x["a_row"].tolist(), x["b_row"].tolist()))  # noqa: E731
    assert rows(J["all1"]) == rows(J["and"]) | rows(J["not1_2"])
    assert rows(J["all2"]) == rows(J["and"]) | rows(J["not2_1"])
    assert rows(J["or"]) == rows(J["and"]) | rows(J["xor"])
    # A-side rows ascending, then B-only rows ascending
    o = J["or"]
    has_a = o["a_row"] >= 0
    k = np.nonzero(~has_a)[0]
    assert np.all(has_a[: k[0]]) and not np.any(has_a[k[0]:])
    key = o["a_row"][has_a] * (n_b + 2) + o["b_row"][has_a] + 1
    assert np.all(np.diff(key) > 0)
    assert np.all(np.diff(o["b_row"][~has_a]) > 0)
    assert np.all(np.isnan(o["sep"][o["b_row"] < 0]))


def test_all_selection_unmatched_are_complements(c1_result):
    d, r = c1_result
    n_a, n_b = d["a_lon"].size, d["b_lon"].size
    j = oracle.join(r, n_a, n_b, "xor")
    in_m_a = np.zeros(n_a, bool); in_m_a[r["a_row"]] = True
    in_m_b = np.zeros(n_b, bool); in_m_b[r["b_row"]] = True
    np.testing.assert_array_equal(j["a_row"][j["a_row"] >= 0], np.nonzero(~in_m_a)[0])
    np.testing.assert_array_equal(j["b_row"][j["a_row"] < 0], np.nonzero(~in_m_b)[0])


# --------------------------------------------------------- fixed seeds --

def test_c2_small_grid_equals_brute_and_no_borderline():
    d = synth.c2(scale=0.002)
    kw = dict(a_frame=d["a_frame"], b_frame=d["b_frame"], **d["region"])
    g = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], **kw)
    b = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], mode="brute", **kw)
    assert g["a_row"].size > 500
    assert _pairs(g) == _pairs(b)
    assert g["border_a"].size == 0


# ------------------------------------------- further readings of "best pairs"

def test_pick_hand_example():
    """Best per B and mutual best on a hand-made pair set (paper §2.2 "best
    pairs" read per B and symmetrically): B0 is held by A0 (1.0) and A1 (0.5);
    B1 by A0 (2.0), A1 (3.0) and A2 (2.0), a tie broken to the lower A row."""
    pairs = {"a_row": np.array([0, 0, 1, 1, 2]), "b_row": np.array([0, 1, 0, 1, 1]),
             "sep": np.array([1.0, 2.0, 0.5, 3.0, 2.0])}
    pb = oracle.best_per_b(pairs, 3)
    np.testing.assert_array_equal(pb["best_a"], [1, 0, -1])
    r = oracle.pick(pairs, 3, 3, "best_b")
    np.testing.assert_array_equal(r["a_row"], [0, 1])
    np.testing.assert_array_equal(r["b_row"], [1, 0])
    np.testing.assert_array_equal(r["sep"], [2.0, 0.5])
    m = oracle.pick(pairs, 3, 3, "mutual")
    np.testing.assert_array_equal(m["a_row"], [1])
    np.testing.assert_array_equal(m["b_row"], [0])


def test_best_per_b_is_best_of_the_swapped_match_for_circles():
    """For circles membership is symmetric, so the best pair of each B source
    in match(A, B) is the best pair of that source in match(B, A)."""
    d = synth.c1()
    ab = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], shape=0, a=1.0)
    ba = oracle.match(d["b_lon"], d["b_lat"], d["a_lon"], d["a_lat"], shape=0, a=1.0)
    pb = oracle.best_per_b(ab, d["b_lon"].size)
    bb = oracle.best(ba, d["b_lon"].size)
    assert pb["near_tie"].size == 0 and bb["near_tie"].size == 0
    np.testing.assert_array_equal(pb["best_a"], bb["best_b"])
    has = pb["best_a"] >= 0
    np.testing.assert_allclose(pb["best_sep"][has], bb["best_sep"][has], rtol=0, atol=1e-9)


def test_mutual_best_is_symmetric_and_inside_both_bests():
    d = synth.c1()
    n_a, n_b = d["a_lon"].size, d["b_lon"].size
    ab = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], shape=0, a=1.0)
    ba = oracle.match(d["b_lon"], d["b_lat"], d["a_lon"], d["a_lat"], shape=0, a=1.0)
    m_ab = oracle.pick(ab, n_a, n_b, "mutual")
    m_ba = oracle.pick(ba, n_b, n_a, "mutual")
    assert m_ab["a_row"].size > 6000  # planted pairs are mostly mutual
    got = set(zip(m_ab["a_row"].tolist(), m_ab["b_row"].tolist()))
    assert got == set(zip(m_ba["b_row"].tolist(), m_ba["a_row"].tolist()))
    best_a = oracle.best(ab, n_a)["best_b"]
    best_b = oracle.best_per_b(ab, n_b)["best_a"]
    assert all(best_a[a] == b and best_b[b] == a for a, b in got)
    # every pair that is best both ways is kept
    both = [(a, b) for a, b in zip(ab["a_row"].tolist(), ab["b_row"].tolist())
            if best_a[a] == b and best_b[b] == a]
    assert set(both) == got


# ------------------------------------------------ Exact Value functional case

def test_match_values_equals_all_pairs_comparison():
    """Brute force over every (i, j) on small integer keys with repeats on
    both sides (paper §2.1, Exact Value case)."""
    g = synth.rng(31)
    a = g.integers(-20, 20, 300)
    b = g.integers(-20, 20, 200)
    r = oracle.match_values(a, b)
    ii, jj = np.nonzero(a[:, None] == b[None, :])
    np.testing.assert_array_equal(r["a_row"], ii)
    np.testing.assert_array_equal(r["b_row"], jj)
    assert np.all(r["sep"] == 0)
    # best (lowest B row per A) is the argmin of the all-pairs list
    bb = oracle.best(r, a.size)
    for i in range(a.size):
        js = np.nonzero(b == a[i])[0]
        assert bb["best_b"][i] == (js[0] if js.size else -1)


def test_match_values_floats_zero_and_nan():
    a = np.array([0.0, -0.0, np.nan, 1.5, 2.0**60, -np.inf])
    b = np.array([-0.0, np.nan, 1.5, 1.5000000000000002, 2.0**60 + 0.0, -np.inf, 0.0])
    r = oracle.match_values(a, b)
    pairs = set(zip(r["a_row"].tolist(), r["b_row"].tolist()))
    assert pairs == {(0, 0), (0, 6), (1, 0), (1, 6), (3, 2), (4, 4), (5, 5)}


def test_match_values_large_int64_keys_compare_exactly():
    big = np.array([2**62 + 1, 2**62 + 2, -(2**63), 2**63 - 1], np.int64)
    r = oracle.match_values(big, big[::-1].copy())
    np.testing.assert_array_equal(r["a_row"], [0, 1, 2, 3])
    np.testing.assert_array_equal(r["b_row"], [3, 2, 1, 0])


# ------------------------------------------- normalised distance (§2.2, §3)

@pytest.mark.parametrize("lat0", [0.0, 37.0, -89.99, 89.995])
def test_normalised_distance_of_scaled_ellipse_points(lat0):
    """A point at t (a cos u, b sin u) in the region frame lies on the
    boundary of the ellipse scaled by t, whatever u: its normalised distance
    is t."""
    a, b, pa = 20.0, 6.0, 30.0
    t = np.array([0.05, 0.3, 0.61, 0.97, 0.9999])
    u = np.radians(np.array([0.0, 17.0, 90.0, 133.0, 200.0, 271.0, 333.0]))
    tt, uu = np.meshgrid(t, u, indexing="ij")
    xy = np.stack([(tt * a * np.cos(uu)).ravel(), (tt * b * np.sin(uu)).ravel()], 1)
    lon, lat = _region_points(123.0, lat0, pa, xy)
    r = oracle.match([123.0], [lat0], lon, lat, shape=oracle.ELLIPSE, a=a, b=b, pa=pa)
    assert r["b_row"].size == xy.shape[0]
    np.testing.assert_allclose(r["dist"], tt.ravel()[r["b_row"]], rtol=1e-9)


@pytest.mark.parametrize("lat0", [0.0, -60.0, 89.999])
def test_normalised_distance_of_rectangle_edges(lat0):
    """Points on the edges of the rectangle scaled by t (t a, w t b) and
    (w t a, t b) with |w| <= 1 have normalised distance t."""
    a, b, pa = 15.0, 4.0, 110.0
    pts, want = [], []
    for t in (0.2, 0.5, 0.93):
        for w in (-1.0, -0.4, 0.0, 0.7, 1.0):
            pts += [[t * a, w * t * b], [-t * a, w * t * b], [w * t * a, t * b], [w * t * a, -t * b]]
            want += [t] * 4
    lon, lat = _region_points(300.0, lat0, pa, np.array(pts))
    r = oracle.match([300.0], [lat0], lon, lat, shape=oracle.RECT, a=a, b=b, pa=pa)
    assert r["b_row"].size == len(pts)
    np.testing.assert_allclose(r["dist"], np.array(want)[r["b_row"]], rtol=1e-9)


def test_normalised_distance_of_circles_is_separation_over_radius():
    a_lon, a_lat, b_lon, b_lat, cols = _random_mixed(11)
    r = oracle.match(a_lon, a_lat, b_lon, b_lat, a_col=cols["a_col"])
    assert r["a_row"].size > 50
    np.testing.assert_allclose(r["dist"], r["sep"] / cols["a_col"][r["a_row"]], rtol=1e-12)
    assert np.all(r["dist"] <= 1.0)


@pytest.mark.parametrize("shape", [1, 2])
def test_normalised_distance_scales_inversely_with_region_size(shape):
    """Scaling every region by s divides each pair's normalised distance by
    s; the members of the smaller regions are the pairs with dist <= 1/s."""
    a_lon, a_lat, b_lon, b_lat, cols = _random_mixed(12)
    kw = dict(shape=shape, a_col=cols["a_col"], b_col=cols["b_col"], pa_col=cols["pa_col"])
    big = oracle.match(a_lon, a_lat, b_lon, b_lat, size_scale=1.5, **kw)
    base = oracle.match(a_lon, a_lat, b_lon, b_lat, **kw)
    key_big = big["a_row"] * 10**6 + big["b_row"]
    key = base["a_row"] * 10**6 + base["b_row"]
    inside = big["dist"] * 1.5 <= 1.0
    np.testing.assert_array_equal(np.sort(key_big[inside]), np.sort(key))
    np.testing.assert_allclose(big["dist"][np.isin(key_big, key)] * 1.5, base["dist"], rtol=1e-12)


def test_best_normalised_hand_example():
    """Ellipse 20 x 2 arcsec, major axis north: B0 10 arcsec along the major
    axis (dist 0.5), B1 1.5 arcsec across it (dist 0.75). By separation the
    best is B1, by normalised distance B0."""
    lon, lat = _region_points(50.0, 10.0, 0.0, np.array([[10.0, 0.0], [0.0, 1.5]]))
    r = oracle.match([50.0], [10.0], lon, lat, shape=oracle.ELLIPSE, a=20.0, b=2.0, pa=0.0)
    np.testing.assert_allclose(r["dist"], [0.5, 0.75], rtol=1e-9)
    assert oracle.best(r, 1)["best_b"][0] == 1
    bn = oracle.best_normalised(r, 1)
    assert bn["best_b"][0] == 0 and bn["best_dist"][0] == pytest.approx(0.5, rel=1e-9)


def test_best_normalised_equals_best_for_fixed_circles(c1_result):
    d, r = c1_result
    n_a = d["a_lon"].size
    np.testing.assert_array_equal(oracle.best_normalised(r, n_a)["best_b"],
                                  oracle.best(r, n_a)["best_b"])


def test_concentric_levels_from_construction():
    """Points at known normalised distances t inside an ellipse: the level is
    the first scale >= t, the counts are cumulative over the scales."""
    a, b, pa = 30.0, 12.0, 75.0
    t = np.array([0.1, 0.29, 0.31, 0.55, 0.65, 0.88, 0.95, 0.999, 0.2])
    u = np.radians(np.arange(t.size) * 41.0)
    xy = np.stack([t * a * np.cos(u), t * b * np.sin(u)], 1)
    lon, lat = _region_points(210.0, -33.0, pa, xy)
    r = oracle.match([210.0], [-33.0], lon, lat, shape=oracle.ELLIPSE, a=a, b=b, pa=pa)
    scales = [0.3, 0.6, 0.9]
    c = oracle.concentric(r, 1, scales)
    np.testing.assert_array_equal(c["level"], np.array([0, 0, 1, 1, 2, 2, 3, 3, 0])[r["b_row"]])
    np.testing.assert_array_equal(c["n_within"][0], [3, 5, 7])
    assert c["border"].size == 0
    # one scale of 1: every member is at level 0
    assert np.all(oracle.concentric(r, 1, [1.0])["level"] == 0)


@pytest.mark.parametrize("bad", [[], [0.5, 0.5], [0.6, 0.3], [0.0, 0.5], [0.5, 1.2], [np.nan]])
def test_concentric_rejects_bad_scales(bad):
    r = oracle.match([1.0], [1.0], [1.0], [1.0], a=1.0)
    with pytest.raises(oracle.OracleError):
        oracle.concentric(r, 1, bad)


# -------------------------------------- borderline and near-tie report --
#
# Parity is exact equality outside the oracle's borderline set (candidates
# whose decision margin is below tau = 1e-9, and best pairs whose two
# smallest separations differ by less than tau times the smallest); these
# pins show the oracle sees that set, with the margin it defines.

TAU = 1e-9


def _on_scaled_boundary(shape, t, a, b, pa, lon0, lat0, n_dir=8):
    """Points whose normalised distance from (lon0, lat0) is t for a region
    of the shape: t times the boundary (ellipse (a cos u, b sin u); the
    rectangle's edges), for n_dir directions."""
    u = np.radians(np.arange(n_dir) * (360.0 / n_dir) + 7.0)
    if shape == oracle.RECT:
        # midpoints and near-corners of the four edges
        xy = np.array([[a, 0.3 * b], [-a, -0.7 * b], [0.4 * a, b], [-0.9 * a, -b],
                       [a, -0.99 * b], [-a, 0.5 * b], [0.0, b], [0.2 * a, -b]])[:n_dir]
    else:
        bb = a if shape == oracle.CIRCLE else b
        xy = np.stack([a * np.cos(u), bb * np.sin(u)], 1)
    return _region_points(lon0, lat0, pa, t * xy)


def _margin_of(shape, t):
    """The decision margin the oracle defines for a point at normalised
    distance t: |rho/r - 1| for circles, |q - 1| = |t^2 - 1| for ellipses,
    |max(|X|/a, |Y|/b) - 1| for rectangles."""
    return abs(t * t - 1.0) if shape == oracle.ELLIPSE else abs(t - 1.0)


@pytest.mark.parametrize("shape", [oracle.CIRCLE, oracle.ELLIPSE, oracle.RECT])
@pytest.mark.parametrize("lat0", [3.0, -71.0, 89.9])
def test_borderline_candidates_are_listed(shape, lat0):
    # large regions (10 arcmin) so the construction's ~1e-10 arcsec position
    # error is ~1e-13 relative, far below every margin used here
    a, b, pa = 600.0, 350.0, 40.0
    listed, unlisted = (1.0 - 1e-11, 1.0 + 1e-11), (1.0 - 1e-7, 1.0 + 1e-7)
    ts = listed + unlisted
    lon, lat = [], []
    for t in ts:
        lo, la = _on_scaled_boundary(shape, t, a, b, pa, 150.0, lat0)
        lon.append(lo); lat.append(la)
    n_dir = lon[0].size
    lon, lat = np.concatenate(lon), np.concatenate(lat)
    r = oracle.match([150.0], [lat0], lon, lat, shape=shape, a=a, b=b, pa=pa)
    t_of = np.repeat(ts, n_dir)
    # members: exactly the points at t <= 1
    np.testing.assert_array_equal(r["b_row"], np.nonzero(t_of <= 1.0)[0])
    # listed: exactly the points within 1e-11 of the boundary, with A's row
    np.testing.assert_array_equal(np.sort(r["border_b"]), np.nonzero(np.abs(t_of - 1.0) < 1e-9)[0])
    assert np.all(r["border_a"] == 0)
    assert np.all(r["border_margin"] < TAU)


@pytest.mark.parametrize("shape", [oracle.CIRCLE, oracle.ELLIPSE, oracle.RECT])
def test_borderline_margin_values(shape):
    """The reported margin is the one defined per shape (not, say, the
    normalised distance's distance from 1 for ellipses)."""
    a, b, pa = 900.0, 500.0, 115.0
    ts = (1.0 - 3e-10, 1.0 + 3e-10, 1.0 - 4.5e-10)
    lon, lat = [], []
    for t in ts:
        lo, la = _on_scaled_boundary(shape, t, a, b, pa, 20.0, 40.0, n_dir=4)
        lon.append(lo); lat.append(la)
    lon, lat = np.concatenate(lon), np.concatenate(lat)
    r = oracle.match([20.0], [40.0], lon, lat, shape=shape, a=a, b=b, pa=pa)
    expect = np.repeat([_margin_of(shape, t) for t in ts], 4)
    assert r["border_b"].size == expect.size
    got = np.empty(expect.size)
    got[r["border_b"]] = r["border_margin"]
    np.testing.assert_allclose(got, expect, rtol=0, atol=2e-11)


def test_borderline_circle_relative_to_radius():
    """The circle's margin is relative to the radius: a point 1e-7 arcsec
    outside a 1e-3 arcsec circle is far from borderline (1e-4), one
    2e-13 arcsec outside it is listed."""
    lon, lat = _region_points(10.0, 0.0, 0.0, np.array([[1e-3 + 1e-7, 0.0], [5e-4, 0.0]]))
    r = oracle.match([10.0], [0.0], lon, lat, a=1e-3)
    assert r["border_b"].size == 0
    np.testing.assert_array_equal(r["b_row"], [1])
    r2 = oracle.match([10.0], [0.0], lon, lat, a=(1e-3 + 1e-7) * (1.0 + 1e-11))
    np.testing.assert_array_equal(r2["border_b"], [0])


def _two_members(s1, s2, s3=None):
    """A at (60, -20) with members at separations s1, s2 (and s3) arcsec
    along different bearings, inside a circle of twice the largest."""
    seps = [s1, s2] + ([s3] if s3 is not None else [])
    xy = np.array([[s * np.cos(np.radians(50 * k + 10)), s * np.sin(np.radians(50 * k + 10))]
                   for k, s in enumerate(seps)])
    lon, lat = _region_points(60.0, -20.0, 0.0, xy)
    return oracle.match([60.0], [-20.0], lon, lat, a=2.0 * max(seps))


@pytest.mark.parametrize("s", [500.0, 2.0])
def test_best_near_tie_listed(s):
    r = _two_members(s, s * (1.0 + 1e-11))
    assert r["a_row"].size == 2
    np.testing.assert_array_equal(oracle.best(r, 1)["near_tie"], [0])
    r = _two_members(s, s * (1.0 + 1e-7))
    assert oracle.best(r, 1)["near_tie"].size == 0


def test_best_near_tie_is_relative_to_the_separation():
    # 500 arcsec apart by 5e-9 arcsec (1e-11 relative): listed; 0.01 arcsec
    # apart by 5e-10 arcsec (5e-8 relative): not listed
    np.testing.assert_array_equal(oracle.best(_two_members(500.0, 500.0 + 5e-9), 1)["near_tie"], [0])
    assert oracle.best(_two_members(0.01, 0.01 * (1 + 5e-8)), 1)["near_tie"].size == 0


def test_best_near_tie_compares_the_two_smallest():
    # first and second differ by 1e-11 (listed) although the third is far;
    # first and second far apart, second and third close: not listed
    r = _two_members(3.0, 3.0 * (1 + 1e-11), 4.0)
    np.testing.assert_array_equal(oracle.best(r, 1)["near_tie"], [0])
    r = _two_members(2.0, 3.0, 3.0 * (1 + 1e-11))
    assert oracle.best(r, 1)["near_tie"].size == 0


def test_near_tie_from_pair_lists():
    """The selection logic alone, on hand-made pair lists: rows 0 and 2 have
    near ties, row 1 an exact duplicate (ties resolve by row, not listed as
    near), row 3 a single member; per B the same through best_per_b."""
    pairs = {"a_row": np.array([0, 0, 1, 1, 2, 2, 2, 3]),
             "b_row": np.array([5, 3, 1, 2, 0, 4, 6, 7]),
             "sep": np.array([7.0, 7.0 * (1 + 3e-10), 2.0, 2.0, 1.5, 9.0, 1.5 * (1 - 4e-10), 1.0])}
    bb = oracle.best(pairs, 4)
    np.testing.assert_array_equal(bb["near_tie"], [0, 2])
    np.testing.assert_array_equal(bb["best_b"], [5, 1, 6, 7])
    # every B source of these pairs is held once: no near tie per B
    np.testing.assert_array_equal(oracle.best_per_b(pairs, 8)["near_tie"], [])
    # B 9 held by A rows 0 and 1 at nearly equal separations
    two = {"a_row": np.array([0, 1]), "b_row": np.array([9, 9]), "sep": np.array([4.0, 4.0 * (1 + 1e-10)])}
    np.testing.assert_array_equal(oracle.best_per_b(two, 10)["near_tie"], [9])
    np.testing.assert_array_equal(oracle.pick(two, 2, 10, "best_b")["near_tie_b"], [9])


def test_concentric_scale_border_listed():
    """Pairs whose normalised distance lies within tau (relative) of a scale
    are listed; the test is relative to the scale (5e-10 away from a scale of
    0.01 is 5e-8 relative: not listed)."""
    sc = [0.01, 0.5, 0.9]
    d = np.array([0.01 * (1 + 1e-11), 0.01 * (1 + 5e-8), 0.5 * (1 - 2e-10), 0.5 * (1 - 1e-7),
                  0.9, 0.3, 0.9 * (1 + 1e-6)])
    pairs = {"a_row": np.zeros(d.size, np.int64), "b_row": np.arange(d.size), "sep": d, "dist": d}
    c = oracle.concentric(pairs, 1, sc)
    np.testing.assert_array_equal(c["border"], [0, 2, 4])
    np.testing.assert_array_equal(c["level"], [1, 1, 1, 1, 2, 1, 3])
