"""Parity at full size, in the configurations the bench times: the all-sky
circle workload (A = 5e7, B = 2e8) and 4096 batched requests against a
resident B of 1e8, generated on the device.

The oracle cannot take every source at these sizes, so it checks samples it
can compute exactly: all A sources inside a few small caps (both poles, the
0/360 seam, random places) matched against every B source that can reach
them (B inside the cap widened by the largest region), and for the batch a
set of whole requests against the B of their caps. B rows keep their
catalogue order in each cut, so tie-breaks by lowest B row are preserved.
Beyond the sample, the FP32 + recheck and FP64 paths must agree on every
source."""

import math

import numpy as np
import pytest

import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
SEP_TOL = 1e-4


@pytest.fixture(scope="module")
def xm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_08494_gb300 import xm as mod

    return mod


def _h(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def _cut(lon, lat, c_lon, c_lat, rad_deg):
    """Rows (ascending) of the positions within rad_deg of (c_lon, c_lat)."""
    import torch

    cl, cb = math.radians(c_lon), math.radians(c_lat)
    lr, br = torch.deg2rad(lon), torch.deg2rad(lat)
    dot = (torch.cos(br) * torch.cos(lr) * (math.cos(cb) * math.cos(cl)) +
           torch.cos(br) * torch.sin(lr) * (math.cos(cb) * math.sin(cl)) +
           torch.sin(br) * math.sin(cb))
    return torch.nonzero(dot >= math.cos(math.radians(rad_deg))).flatten()


def _oracle_cut(d_a, d_b, a_rows, b_rows, frame, region):
    """Oracle pairs and best of A rows a_rows against B rows b_rows, in
    catalogue rows."""
    a_lon, a_lat = _h(d_a[0][a_rows]), _h(d_a[1][a_rows])
    b_lon, b_lat = _h(d_b[0][b_rows]), _h(d_b[1][b_rows])
    reg = {k: (_h(v[a_rows]) if hasattr(v, "numel") else v) for k, v in region.items()}
    ref = oracle.match(a_lon, a_lat, b_lon, b_lat, a_frame=frame, b_frame=frame, **reg)
    assert ref["border_a"].size == 0
    bb = oracle.best(ref, a_lon.size)
    assert bb["near_tie"].size == 0
    ar, br = _h(a_rows), _h(b_rows)
    best_b = np.where(bb["best_b"] >= 0, br[np.maximum(bb["best_b"], 0)], -1)
    return ref, ar[ref["a_row"]], br[ref["b_row"]], best_b, bb["best_sep"]


# ------------------------------------------------------------------ C3

PATCHES = [(0.0, 90.0), (0.0, -90.0), (0.0, 0.0), (359.95, 30.0), (0.05, -45.0),
           (120.0, 1.0), (250.0, -60.0), (33.0, 12.0)]


@pytest.fixture(scope="module")
def c3_full(xm):
    from paper_1611_08494_gb300 import synth_gpu

    d = synth_gpu.c3()
    idx = {p: xm.Index(d["b_lon"], d["b_lat"], frame=d["b_frame"], ids=d["b_id"],
                       zone_height_arcsec=12.0, build_fp64=(p == "fp64")) for p in ("fp32", "fp64")}
    res = {p: xm.Result(idx[p], d["a_lon"], d["a_lat"], frame=d["a_frame"],
                        precision=xm.PREC_FP32 if p == "fp32" else xm.PREC_FP64,
                        selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"]) for p in ("fp32", "fp64")}
    return d, idx, res


def test_c3_full_size_sampled_caps(xm, c3_full):
    d, _, res = c3_full
    r_cap, r_max = 0.15, 2.0 / 3600.0
    n_checked = 0
    for c_lon, c_lat in PATCHES:
        a_rows = _cut(d["a_lon"], d["a_lat"], c_lon, c_lat, r_cap)
        b_rows = _cut(d["b_lon"], d["b_lat"], c_lon, c_lat, r_cap + 2 * r_max)
        if a_rows.numel() == 0:
            continue
        ref, ea, eb, best_b, best_sep = _oracle_cut((d["a_lon"], d["a_lat"]), (d["b_lon"], d["b_lat"]),
                                                    a_rows, b_rows, d["a_frame"], d["region"])
        ar = _h(a_rows)
        for p in ("fp32", "fp64"):
            r = res[p]
            ga, gb, gs = _h(r.a_row), _h(r.b_row), _h(r.sep)
            keep = np.isin(ga, ar)
            np.testing.assert_array_equal(ga[keep], ea)
            np.testing.assert_array_equal(gb[keep], eb)
            if ea.size:
                assert np.max(np.abs(gs[keep] - ref["sep"])) <= SEP_TOL
            np.testing.assert_array_equal(_h(r.best_b)[ar], best_b)
        n_checked += ar.size
    assert n_checked > 2000


def test_c3_full_size_paths_agree_everywhere(xm, c3_full):
    import torch

    _, _, res = c3_full
    a, b = res["fp32"], res["fp64"]
    assert int(a.n_pairs) == int(b.n_pairs)
    assert torch.equal(a.a_row, b.a_row) and torch.equal(a.b_row, b.b_row)
    assert torch.equal(a.best_b, b.best_b)
    assert float((a.sep - b.sep).abs().max()) <= SEP_TOL


def test_c3_full_size_planted_recall(xm, c3_full):
    """Every planted counterpart within 0.9 r is found (1.8 of 2 arcsec)."""
    import torch

    d, _, res = c3_full
    t = d["truth"]
    near = t["rho_arcsec"] <= 1.8
    want = t["a_row"][near] * (1 << 32) + t["b_row"][near]
    r = res["fp32"]
    got = r.a_row * (1 << 32) + r.b_row
    found = torch.isin(want, got)
    assert bool(found.all())


# ------------------------------------------------------------------ C4

@pytest.fixture(scope="module")
def c4_full(xm):
    from paper_1611_08494_gb300 import synth_gpu

    d = synth_gpu.c4()
    idx = xm.Index(d["b_lon"], d["b_lat"], frame=d["b_frame"], zone_height_arcsec=20.0)
    reqs = [dict(lon=q["lon"], lat=q["lat"], selection=q["selection"], join=q["join"],
                 join_selection=q["join_selection"], **q["region"]) for q in d["requests"]]
    batch = xm.Batch(idx, reqs, use_graph=True)
    return d, idx, batch


def test_c4_full_size_sampled_requests(xm, c4_full):
    d, _, batch = c4_full
    n_b = d["b_lon"].numel()
    h = np.random.Generator(np.random.Philox(key=4242))
    small = [r for r, q in enumerate(d["requests"]) if q["lon"].numel() <= 20_000]
    large = [r for r, q in enumerate(d["requests"]) if q["lon"].numel() > 20_000]
    pick = list(h.choice(small, 16, replace=False)) + list(h.choice(large, 4, replace=False))
    for r in pick:
        q = d["requests"][r]
        c_lon, c_lat, rad = q["cap"]
        n_a = q["lon"].numel()
        # offset copies stay within 8 sigma of the cap (odds ~1e-14 each);
        # a region reaches at most sqrt(2) x its largest size
        reach_a = rad + 8.0 * q["offset_sigma"] / 3600.0
        reach_b = reach_a + 1.5 * q["max_size"] / 3600.0
        import torch

        a_in = _cut(q["lon"], q["lat"], c_lon, c_lat, reach_a)
        assert a_in.numel() == n_a, "an A source lies outside the cut"
        b_rows = _cut(d["b_lon"], d["b_lat"], c_lon, c_lat, reach_b)
        a_rows = torch.arange(n_a, device="cuda")
        ref, ea, eb, best_b, _ = _oracle_cut((q["lon"], q["lat"]), (d["b_lon"], d["b_lat"]),
                                             a_rows, b_rows, 0, q["region"])
        v = batch.view(r)
        np.testing.assert_array_equal(_h(v["a_row"]), ea)
        np.testing.assert_array_equal(_h(v["b_row"]), eb)
        if ea.size:
            assert np.max(np.abs(_h(v["sep"]) - ref["sep"])) <= SEP_TOL
        np.testing.assert_array_equal(_h(v["best_b"]), best_b)
        # the join: rows as the oracle forms them from the selected pairs
        sel = oracle.selected_pairs(ref, n_a, "all" if q["join_selection"] == 1 else "best")
        sel = dict(sel, b_row=_h(b_rows)[sel["b_row"]]) if "b_row" in sel else sel
        exp = oracle.join(sel, n_a, n_b, q["join"])
        full = batch.join(r)
        np.testing.assert_array_equal(_h(full.a_row), exp["a_row"])
        np.testing.assert_array_equal(_h(full.b_row), exp["b_row"])
