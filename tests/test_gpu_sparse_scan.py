"""The sparse form of the count pass (one lane per source, for fixed regions
small against the zone height) against the FP64 oracle, on a mix built so
that the pass keeps some sources and leaves others to the warp-cooperative
scan: sparse sources, a dense clump (more records in a source's bucket
ranges than one lane takes on), sources on the 0/360 seam whose windows
also cross a zone boundary (more than two items), sources at both poles,
and exact duplicates of B positions (best-pair ties to the lowest B row).
Both kernels must run, and every pair, separation, count and best pair must
equal the oracle's."""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
SEP_TOL = 1e-4  # arcsec
ZONE_H = 12.0  # arcsec: regions up to 4.8 arcsec take the sparse pass


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


def _host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def _mix(seed=31):
    g = np.random.Generator(np.random.Philox(key=seed))
    a_lon, a_lat, b_lon, b_lat = [], [], [], []

    def near(lon, lat, n, sigma_arcsec):
        d = g.normal(0.0, sigma_arcsec / 3600.0, (2, n))
        la = np.clip(lat + d[1], -90.0, 90.0)
        lo = np.mod(lon + d[0] / np.maximum(np.cos(np.radians(la)), 1e-3), 360.0)
        return lo, la

    # sparse field: B uniform in a 2 x 2 deg box, A offset copies of some
    lo, la = g.uniform(40.0, 42.0, 30_000), g.uniform(10.0, 12.0, 30_000)
    b_lon.append(lo); b_lat.append(la)
    pick = g.choice(lo.size, 8_000, replace=False)
    x, y = near(lo[pick], la[pick], pick.size, 1.0)
    a_lon.append(x); a_lat.append(y)
    a_lon.append(g.uniform(40.0, 42.0, 4_000)); a_lat.append(g.uniform(10.0, 12.0, 4_000))
    # dense clump: 3000 B within ~3 arcsec, A inside it
    x, y = near(np.full(3000, 100.0), np.full(3000, -30.0), 3000, 1.5)
    b_lon.append(x); b_lat.append(y)
    x, y = near(np.full(200, 100.0), np.full(200, -30.0), 200, 2.0)
    a_lon.append(x); a_lat.append(y)
    # the seam at zone boundaries: RA within 3 arcsec of 0/360, latitudes
    # at multiples of the zone height (a window meets two zones, two segments)
    lat_b = np.round(g.uniform(-5.0, 5.0, 600) * 3600.0 / ZONE_H) * ZONE_H / 3600.0
    lo = np.mod(g.normal(0.0, 3.0 / 3600.0, 600), 360.0)
    b_lon.append(lo); b_lat.append(lat_b + g.normal(0.0, 1.0 / 3600.0, 600))
    a_lon.append(np.mod(lo + g.normal(0.0, 1.0 / 3600.0, 600), 360.0))
    a_lat.append(lat_b + g.normal(0.0, 1.0 / 3600.0, 600))
    # both poles: random distances from the pole (no source on it, where
    # every longitude is the same point)
    for sign in (1.0, -1.0):
        for lon_s, lat_s, n in ((b_lon, b_lat, 300), (a_lon, a_lat, 200)):
            lon_s.append(g.uniform(0.0, 360.0, n))
            lat_s.append(sign * (90.0 - np.abs(g.normal(0.0, 4.0 / 3600.0, n)) - 1e-7))
    b_lon, b_lat = np.concatenate(b_lon), np.concatenate(b_lat)
    # exact duplicates of some B positions (ties between B rows)
    dup = g.choice(30_000, 500, replace=False)
    b_lon, b_lat = np.concatenate([b_lon, b_lon[dup]]), np.concatenate([b_lat, b_lat[dup]])
    return (np.concatenate(a_lon), np.concatenate(a_lat), b_lon, b_lat)


@pytest.mark.parametrize("region", [dict(shape=0, a=2.0), dict(shape=1, a=3.0, b=1.5, pa=30.0),
                                    dict(shape=2, a=2.5, b=1.0, pa=110.0)])
@pytest.mark.parametrize("selection", ["all+best", "best"])
def test_sparse_count_pass_equals_the_oracle(xm, region, selection):
    a_lon, a_lat, b_lon, b_lat = _mix()
    ref = oracle.match(a_lon, a_lat, b_lon, b_lat, a_frame=0, b_frame=0, **region)
    assert ref["border_a"].size == 0
    bb = oracle.best(ref, a_lon.size)
    assert bb["near_tie"].size == 0
    idx = xm.Index(_cuda(b_lon), _cuda(b_lat), zone_height_arcsec=ZONE_H)
    sel = xm.SEL_ALL | xm.SEL_BEST if selection == "all+best" else xm.SEL_BEST
    xm.reset_stats()
    xm.prof_enable(True)
    try:
        res = xm.Result(idx, _cuda(a_lon), _cuda(a_lat), precision=xm.PREC_FP32,
                        selection=sel, **region)
        n = res.n_pairs
        prof = xm.prof_all()
    finally:
        xm.prof_enable(False)
    # the sparse pass ran, and the warp-cooperative pass over what it left
    assert prof["k_scan_src"][1] == 1 and prof["k_scan_fp32_count"][1] >= 1
    count = np.bincount(ref["a_row"], minlength=a_lon.size)
    np.testing.assert_array_equal(_host(res.count), count)
    assert count.max() > 48  # the clump's sources were left to the warp scan
    np.testing.assert_array_equal(_host(res.best_b), bb["best_b"])
    has = bb["best_b"] >= 0
    got = _host(res.best_sep)
    assert np.all(np.isnan(got[~has]))
    assert np.max(np.abs(got[has] - bb["best_sep"][has])) <= SEP_TOL
    if selection == "all+best":
        assert n == ref["a_row"].size
        np.testing.assert_array_equal(_host(res.a_row), ref["a_row"])
        np.testing.assert_array_equal(_host(res.b_row), ref["b_row"])
        assert np.max(np.abs(_host(res.sep) - ref["sep"])) <= SEP_TOL
    # candidates and members are counted once whichever pass took a source
    st = xm.stats()
    assert st["members"] == ref["a_row"].size


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_sparse_count_pass_rotated_frames(xm, shape):
    """A in galactic coordinates against an equatorial index: every source
    is rotated into the index frame, and for ellipses and rectangles the
    position angle turns with the frame at each position, so the sparse
    pass prepares each such source's region in full (circles keep the
    block's shared terms). Pairs, separations, counts and best pairs equal
    the oracle's."""
    a_lon, a_lat, b_lon, b_lat = _mix(seed=47)
    # A's positions in galactic coordinates (the same points on the sky)
    ga_lon, ga_lat = oracle.from_equatorial(a_lon, a_lat, oracle.GAL)
    region = [dict(shape=0, a=2.0), dict(shape=1, a=3.0, b=1.5, pa=30.0),
              dict(shape=2, a=2.5, b=1.0, pa=110.0)][shape]
    ref = oracle.match(ga_lon, ga_lat, b_lon, b_lat, a_frame=oracle.GAL, b_frame=oracle.EQ,
                       **region)
    assert ref["border_a"].size == 0
    bb = oracle.best(ref, ga_lon.size)
    assert bb["near_tie"].size == 0
    idx = xm.Index(_cuda(b_lon), _cuda(b_lat), zone_height_arcsec=ZONE_H)
    xm.prof_enable(True)
    try:
        res = xm.Result(idx, _cuda(ga_lon), _cuda(ga_lat), frame=xm.GAL, precision=xm.PREC_FP32,
                        selection=xm.SEL_ALL | xm.SEL_BEST, **region)
        n = res.n_pairs
        prof = xm.prof_all()
    finally:
        xm.prof_enable(False)
    assert prof["k_scan_src"][1] == 1
    assert n == ref["a_row"].size
    np.testing.assert_array_equal(_host(res.a_row), ref["a_row"])
    np.testing.assert_array_equal(_host(res.b_row), ref["b_row"])
    assert np.max(np.abs(_host(res.sep) - ref["sep"])) <= SEP_TOL
    np.testing.assert_array_equal(_host(res.best_b), bb["best_b"])
