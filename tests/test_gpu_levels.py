"""Normalised distance, best pair by it (paper §2.2) and concentric scaled
regions (paper §3) on the GPU (xm_levels_compute) against the oracle.

Distances agree within 1e-9 (positions are kept as float64 degrees in the
index frame, a few 1e-16 rad apart from the oracle's unit vectors, which is
~1e-11 of a region of a few arcsec); levels, per-copy counts and best pairs
are identical except where the oracle reports a decision within 1e-9 of a
scale or a near tie, which every fixed seed here avoids (asserted)."""

import numpy as np
import pytest

import oracle
from paper_1611_08494_gb300 import synth

pytestmark = pytest.mark.gpu
SCALES = [0.25, 0.5, 0.7071, 0.9]
DIST_TOL = 1e-9


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


def _h(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def _mixed(seed, shape, a_frame=0, b_frame=0):
    """Crowded caps at both poles, the RA seam and two ordinary fields,
    per-source sizes and angles, every region option set."""
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


def _oracle(d):
    return oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], a_frame=d["a_frame"],
                        b_frame=d["b_frame"], **d["region"])


def _gpu(xm, d, prec, a_order=0, build_fp64=True, zone=0.0):
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]), frame=d["b_frame"],
                   zone_height_arcsec=zone, build_fp64=build_fp64)
    reg = {k: (_cuda(v) if isinstance(v, np.ndarray) else v) for k, v in d["region"].items()}
    return xm.Result(idx, _cuda(d["a_lon"]), _cuda(d["a_lat"]), frame=d["a_frame"],
                     precision=xm.PREC_FP32 if prec == "fp32" else xm.PREC_FP64,
                     selection=xm.SEL_ALL | xm.SEL_BEST, a_order=a_order, **reg)


def _check(xm, res, ref, n_a, scales=SCALES):
    np.testing.assert_array_equal(_h(res.a_row), ref["a_row"])
    np.testing.assert_array_equal(_h(res.b_row), ref["b_row"])
    lv = res.levels(scales)
    dist = _h(lv.dist)
    np.testing.assert_allclose(dist, ref["dist"], rtol=0, atol=DIST_TOL)
    bn = oracle.best_normalised(ref, n_a)
    assert bn["near_tie"].size == 0
    np.testing.assert_array_equal(_h(lv.best_b), bn["best_b"])
    bd = _h(lv.best_dist)
    has = bn["best_b"] >= 0
    assert np.all(np.isnan(bd[~has]))
    np.testing.assert_allclose(bd[has], bn["best_dist"][has], rtol=0, atol=DIST_TOL)
    if len(scales):
        c = oracle.concentric(ref, n_a, scales)
        assert c["border"].size == 0
        np.testing.assert_array_equal(_h(lv.level), c["level"])
        np.testing.assert_array_equal(_h(lv.n_within), c["n_within"])
    else:
        assert lv.level.numel() == 0 and lv.n_within.numel() == 0
    return lv


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [0, 1, 2])
@pytest.mark.parametrize("frames", [(0, 0), (1, 0)])
def test_shapes_frames_poles_seam(xm, prec, shape, frames):
    d = _mixed(70 + shape, shape, *frames)
    ref = _oracle(d)
    assert ref["a_row"].size > 30
    for a_order in (1, 2):  # the sorted order keeps a row -> slot map
        _check(xm, _gpu(xm, d, prec, a_order=a_order), ref, d["a_lon"].size)


@pytest.mark.parametrize("build_fp64", [True, False])
def test_c2_small_ellipses(xm, build_fp64):
    d = synth.c2(scale=0.02)
    ref = _oracle(d)
    assert ref["a_row"].size > 5000
    lv = _check(xm, _gpu(xm, d, "fp32", build_fp64=build_fp64), ref, d["a_lon"].size)
    # the outermost copy at scale 1 would hold every member
    within = _h(lv.n_within)
    assert np.all(np.diff(within, axis=1) >= 0)
    assert np.all(within[:, -1] <= np.bincount(ref["a_row"], minlength=d["a_lon"].size))


def test_c1_circles_best_equals_best_by_separation(xm):
    d = synth.c1()
    ref = _oracle(d)
    res = _gpu(xm, d, "fp32")
    lv = _check(xm, res, ref, d["a_lon"].size, scales=[1.0])
    # one fixed radius: deepest inside is nearest
    np.testing.assert_array_equal(_h(lv.best_b), _h(res.best_b))
    assert np.all(_h(lv.level) == 0)


def test_constructed_points_on_scaled_ellipses(xm):
    """B placed at normalised distance t on ellipses of many A sources, the
    level read off the construction."""
    g = synth.rng(81)
    n_a = 400
    a_lon = g.uniform(0, 360, n_a)
    a_lat = np.degrees(np.arcsin(g.uniform(-0.999, 0.999, n_a)))
    a_ax, b_ax, pa = 30.0, 10.0, g.uniform(0, 180, n_a)
    t = np.array([0.1, 0.24, 0.26, 0.49, 0.51, 0.7, 0.72, 0.88, 0.92, 0.99])
    b_lon, b_lat, want_t = [], [], []
    for i in range(n_a):
        u = g.uniform(0, 2 * np.pi, t.size)
        x, y = t * a_ax * np.cos(u), t * b_ax * np.sin(u)
        rho = np.hypot(x, y) * synth.ARCSEC
        bearing = np.radians(pa[i]) + np.arctan2(y, x)
        lo, la = synth.destination(np.full(t.size, a_lon[i]), np.full(t.size, a_lat[i]), rho, bearing)
        b_lon.append(lo); b_lat.append(la); want_t.append(t)
    d = dict(a_lon=a_lon, a_lat=a_lat, b_lon=np.concatenate(b_lon), b_lat=np.concatenate(b_lat),
             a_frame=0, b_frame=0, region=dict(shape=1, a=a_ax, b=b_ax, pa_col=pa))
    ref = _oracle(d)
    assert ref["a_row"].size == n_a * t.size  # regions this far apart do not overlap
    lv = _check(xm, _gpu(xm, d, "fp32"), ref, n_a)
    want = np.concatenate(want_t)[ref["b_row"]]
    np.testing.assert_allclose(_h(lv.dist), want, rtol=1e-9)
    np.testing.assert_array_equal(_h(lv.n_within), np.tile([2, 4, 6, 8], (n_a, 1)))


def test_no_scales_and_no_pairs(xm):
    d = _mixed(75, 1)
    ref = _oracle(d)
    _check(xm, _gpu(xm, d, "fp32"), ref, d["a_lon"].size, scales=[])
    far = dict(d, a_lat=-d["a_lat"] * 0 + 45.0, a_lon=d["a_lon"] * 0 + 100.0)
    res = _gpu(xm, far, "fp32")
    assert res.n_pairs == 0
    lv = res.levels([0.5, 1.0])
    assert np.all(_h(lv.best_b) == -1) and np.all(np.isnan(_h(lv.best_dist)))
    assert np.all(_h(lv.n_within) == 0)


@pytest.mark.parametrize("bad", [[0.5, 0.5], [0.6, 0.3], [0.0, 0.5], [0.5, 1.2], [np.nan],
                                 list(np.linspace(0.01, 1.0, 65))])
def test_bad_scales_rejected(xm, bad):
    d = _mixed(76, 0)
    res = _gpu(xm, d, "fp32")
    with pytest.raises(xm.XMError, match="EINVAL"):
        res.levels(bad)


def test_needs_all_selection_and_positions(xm):
    d = _mixed(77, 0)
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]))
    res = xm.Result(idx, _cuda(d["a_lon"]), _cuda(d["a_lat"]), selection=xm.SEL_BEST, shape=0, a=5.0)
    with pytest.raises(xm.XMError, match="EINVAL"):
        res.levels([0.5])
    vals = xm.ValueResult(_cuda(np.arange(5, dtype=np.int64)), _cuda(np.arange(5, dtype=np.int64)))
    import ctypes

    h = ctypes.c_void_p()
    st = xm.xm_levels_compute(idx.handle, vals.handle, None, 0, None, ctypes.byref(h))
    assert xm.STATUS[st] in ("XM_EUNSUPPORTED", "XM_EINVAL")


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_wide_regions(xm, shape):
    """Regions of a degree and more, around the equator and near a pole:
    pairs beyond the short-series reach (separation or coordinate
    differences above half a degree) take the unit-vector form."""
    g = synth.rng(90 + shape)
    pa_, pb_ = [], []
    for lon0, lat0 in ((30.0, 5.0), (250.0, 87.5)):
        pa_.append(synth.cap(g, 60, lon0, lat0, 2.0))
        pb_.append(synth.cap(g, 1500, lon0, lat0, 3.0))
    n = 120
    a_col = g.uniform(1800.0, 7200.0, n)  # 0.5 to 2 deg
    d = dict(a_lon=np.concatenate([p[0] for p in pa_]), a_lat=np.concatenate([p[1] for p in pa_]),
             b_lon=np.concatenate([p[0] for p in pb_]), b_lat=np.concatenate([p[1] for p in pb_]),
             a_frame=0, b_frame=0,
             region=dict(shape=shape, a_col=a_col, b_col=a_col * g.uniform(0.3, 1.0, n),
                         pa_col=g.uniform(0.0, 180.0, n)))
    ref = _oracle(d)
    assert ref["a_row"].size > 10000
    sep_deg = ref["sep"] / 3600.0
    assert np.sum(sep_deg > 0.6) > 1000 and np.sum(sep_deg < 0.4) > 1000
    for build_fp64 in (True, False):
        _check(xm, _gpu(xm, d, "fp64", build_fp64=build_fp64), ref, n)
