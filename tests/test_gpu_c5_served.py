"""Served requests against the oracle, in the serving configuration (C5)
scaled to a tenth: a resident B of 3e7 sources with the all-sky latitude
profile in galactic coordinates, indexed with int64 ids; requests with mixed
shapes (fixed sizes and per-source columns), every selection x join type,
and input in equatorial or galactic coordinates. Equatorial requests are
rotated into the galactic index by the library (paper §2 coordinate
systems); galactic ones take half their A as offset copies of B.

Every request is submitted to a server with several slots, so batches run
concurrently and requests share batches; each served result is compared
with the oracle run on that request alone against the B sources of its cap
(pairs and best pairs exactly, separations within 1e-4 arcsec, the A-side
join rows exactly and the number of unmatched B rows)."""

import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
SEP_TOL = 1e-4  # arcsec
N_B = 30_000_000
JOINS = ("and", "or", "all1", "all2", "not1_2", "not2_1", "xor")


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
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def _cut(lon, lat, c_lon, c_lat, rad_deg):
    """Rows (ascending) of the positions within rad_deg of (c_lon, c_lat)."""
    import torch

    cl, cb = math.radians(c_lon), math.radians(c_lat)
    lr, br = torch.deg2rad(lon), torch.deg2rad(lat)
    dot = (torch.cos(br) * torch.cos(lr) * (math.cos(cb) * math.cos(cl)) +
           torch.cos(br) * torch.sin(lr) * (math.cos(cb) * math.sin(cl)) +
           torch.sin(br) * math.sin(cb))
    return torch.nonzero(dot >= math.cos(math.radians(rad_deg))).flatten()


@pytest.fixture(scope="module")
def c5(xm):
    from paper_1611_08494_gb300 import synth_gpu

    b = synth_gpu.c5_catalogue(n_b=N_B)
    reqs = synth_gpu.c5_requests(b, n_pool=28, a_lo=300, a_hi=30_000)
    # every (selection, join) combination twice
    for r, q in enumerate(reqs):
        q["join"] = JOINS[r % 7]
        q["join_selection"] = 1 if (r // 7) % 2 == 0 else 2
    idx = xm.Index(b["b_lon"], b["b_lat"], frame=b["b_frame"], ids=b["b_id"],
                   zone_height_arcsec=20.0)
    return b, reqs, idx


@pytest.fixture(scope="module")
def expected(c5):
    """The oracle's answer for every request, from A against the B rows of
    its cap (widened by the offsets and the largest region)."""
    b, reqs, _ = c5
    out = []
    for q in reqs:
        c_lon, c_lat, rad = q["cap"]
        if q["frame"] == oracle.EQ:  # the cap centre in B's (galactic) frame
            gl, gb = oracle.from_equatorial([c_lon], [c_lat], oracle.GAL)
            c_lon, c_lat = float(gl[0]), float(gb[0])
        reach_a = rad + 8.0 * q["offset_sigma"] / 3600.0
        reach_b = reach_a + 1.5 * q["max_size"] / 3600.0
        b_rows = _cut(b["b_lon"], b["b_lat"], c_lon, c_lat, reach_b)
        br = _h(b_rows)
        n_a = q["lon"].numel()
        reg = {k: (_h(v) if hasattr(v, "numel") else v) for k, v in q["region"].items()}
        ref = oracle.match(_h(q["lon"]), _h(q["lat"]), _h(b["b_lon"][b_rows]), _h(b["b_lat"][b_rows]),
                           a_frame=q["frame"], b_frame=oracle.GAL, **reg)
        assert ref["border_a"].size == 0
        bb = oracle.best(ref, n_a)
        assert bb["near_tie"].size == 0
        pairs = dict(ref, b_row=br[ref["b_row"]])
        best_b = np.where(bb["best_b"] >= 0, br[np.maximum(bb["best_b"], 0)], -1)
        sel = oracle.selected_pairs(pairs, n_a, "all" if q["join_selection"] == 1 else "best")
        rows = oracle.join(sel, n_a, N_B, q["join"])
        a_side = rows["a_row"] >= 0
        out.append(dict(pairs=pairs, best_b=best_b, best_sep=bb["best_sep"],
                        count=np.bincount(ref["a_row"], minlength=n_a),
                        row_a=rows["a_row"][a_side], row_b=rows["b_row"][a_side],
                        row_sep=rows["sep"][a_side], n_un_b=int((~a_side).sum())))
    return out


def test_c5_workload_covers_the_mix(c5, expected):
    _, reqs, _ = c5
    assert {q["frame"] for q in reqs} == {oracle.EQ, oracle.GAL}
    assert {q["region"]["shape"] for q in reqs} == {oracle.CIRCLE, oracle.ELLIPSE, oracle.RECT}
    assert {("a_col" in q["region"]) for q in reqs} == {True, False}
    # the equatorial requests are not vacuous: they have members too
    eq_pairs = sum(e["pairs"]["a_row"].size for q, e in zip(reqs, expected) if q["frame"] == oracle.EQ)
    gal_pairs = sum(e["pairs"]["a_row"].size for q, e in zip(reqs, expected) if q["frame"] == oracle.GAL)
    assert eq_pairs > 0 and gal_pairs > 1000


@pytest.mark.parametrize("slots,graph", [(3, True), (2, False)])
def test_c5_served_requests_equal_the_oracle(xm, c5, expected, slots, graph):
    _, reqs, idx = c5
    with xm.Server(idx, slots=slots, max_batch_requests=5, use_graph=graph,
                   precision=xm.PREC_FP32) as srv:
        tickets = [srv.submit(q["lon"], q["lat"], frame=q["frame"], selection=q["selection"],
                              join=q["join"], join_selection=q["join_selection"], **q["region"])
                   for q in reqs]
        for t in tickets:
            t.wait(120_000)
        for r, (q, t, e) in enumerate(zip(reqs, tickets, expected)):
            v = t.view()
            msg = f"request {r} (frame {q['frame']}, shape {q['region']['shape']}, join {q['join']})"
            np.testing.assert_array_equal(_h(v["a_row"]), e["pairs"]["a_row"], err_msg=msg)
            np.testing.assert_array_equal(_h(v["b_row"]), e["pairs"]["b_row"], err_msg=msg)
            if e["pairs"]["a_row"].size:
                assert np.max(np.abs(_h(v["sep"]) - e["pairs"]["sep"])) <= SEP_TOL, msg
            np.testing.assert_array_equal(_h(v["count"]), e["count"], err_msg=msg)
            np.testing.assert_array_equal(_h(v["best_b"]), e["best_b"], err_msg=msg)
            gs, es = _h(v["best_sep"]), e["best_sep"]
            np.testing.assert_array_equal(np.isnan(gs), np.isnan(es), err_msg=msg)
            ok = ~np.isnan(es)
            if ok.any():
                assert np.max(np.abs(gs[ok] - es[ok])) <= SEP_TOL, msg
            np.testing.assert_array_equal(_h(v["row_a"]), e["row_a"], err_msg=msg)
            np.testing.assert_array_equal(_h(v["row_b"]), e["row_b"], err_msg=msg)
            rs, ers = _h(v["row_sep"]), e["row_sep"]
            np.testing.assert_array_equal(np.isnan(rs), np.isnan(ers), err_msg=msg)
            ok = ~np.isnan(ers)
            if ok.any():
                assert np.max(np.abs(rs[ok] - ers[ok])) <= SEP_TOL, msg
            assert v["n_unmatched_a"] == int((e["count"] == 0).sum()), msg
            if q["join"] in ("or", "all2", "not2_1", "xor"):
                assert v["n_unmatched_b"] == e["n_un_b"], msg
            t.release()
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["batches"] > 1  # requests were spread over several batches
