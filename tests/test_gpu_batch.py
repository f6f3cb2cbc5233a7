"""Batched cross-match (xm_match_batch): every request's results inside a
batch equal those of the same request matched alone (xm_match / xm_join),
whatever the launch mode (plain, CUDA graph, persistent grid size), input
placement, or arena sizes; and a sample of requests equals the FP64 oracle."""

import numpy as np
import pytest

import oracle
from paper_1611_08494_gb300 import synth

pytestmark = pytest.mark.gpu
SEP_TOL = 1e-4


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


@pytest.fixture(scope="module")
def c4_small(xm):
    d = synth.c4(seed=41, n_b=1_000_000, n_req=24, a_lo=100, a_hi=20_000)
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]), zone_height_arcsec=10.0)
    return d, idx


def _dev_requests(d, on_device=True):
    conv = _cuda if on_device else np.asarray
    out = []
    for q in d["requests"]:
        reg = {k: (conv(v) if isinstance(v, np.ndarray) else v) for k, v in q["region"].items()}
        out.append(dict(lon=conv(q["lon"]), lat=conv(q["lat"]), selection=q["selection"],
                        join=q["join"], join_selection=q["join_selection"], **reg))
    return out


def _same_view(v, w):
    for k in ("a_row", "b_row", "count", "best_b", "row_a", "row_b"):
        np.testing.assert_array_equal(_h(v[k]), _h(w[k]), err_msg=k)
    for k in ("sep", "best_sep", "row_sep"):
        np.testing.assert_array_equal(_h(v[k]), _h(w[k]), err_msg=k)
    assert v["n_unmatched_a"] == w["n_unmatched_a"] and v["n_unmatched_b"] == w["n_unmatched_b"]


def test_batch_equals_single_requests(xm, c4_small):
    d, idx = c4_small
    reqs = _dev_requests(d)
    batch = xm.Batch(idx, reqs)
    info = batch.info()
    assert info["total_a"] == sum(len(q["lon"]) for q in d["requests"])
    sel_code = {1: xm.SEL_ALL, 2: xm.SEL_BEST}
    for r, q in enumerate(reqs):
        q = dict(q)
        lon, lat = q.pop("lon"), q.pop("lat")
        join, jsel = q.pop("join"), q.pop("join_selection")
        q.pop("selection")
        res = xm.Result(idx, lon, lat, selection=xm.SEL_ALL | xm.SEL_BEST, **q)
        v = batch.view(r)
        np.testing.assert_array_equal(_h(v["a_row"]), _h(res.a_row))
        np.testing.assert_array_equal(_h(v["b_row"]), _h(res.b_row))
        np.testing.assert_array_equal(_h(v["sep"]), _h(res.sep))
        np.testing.assert_array_equal(_h(v["count"]), _h(res.count))
        np.testing.assert_array_equal(_h(v["best_b"]), _h(res.best_b))
        np.testing.assert_array_equal(_h(v["best_sep"]), _h(res.best_sep))
        rows = res.join(join, sel_code[jsel])
        ra, rb, rs = _h(rows.a_row), _h(rows.b_row), _h(rows.sep)
        a_side = ra >= 0
        np.testing.assert_array_equal(_h(v["row_a"]), ra[a_side])
        np.testing.assert_array_equal(_h(v["row_b"]), rb[a_side])
        np.testing.assert_array_equal(_h(v["row_sep"]), rs[a_side])
        assert v["n_unmatched_a"] == rows.n_unmatched_a
        if join in ("or", "all2", "not2_1", "xor"):
            assert v["n_unmatched_b"] == rows.n_unmatched_b
        full = batch.join(r)
        np.testing.assert_array_equal(_h(full.a_row), ra)
        np.testing.assert_array_equal(_h(full.b_row), rb)


@pytest.mark.parametrize("mode", ["graph", "blocks1", "blocks8", "host", "short_arenas", "graph_short",
                                  "sorted", "sorted_graph_short"])
def test_batch_modes_agree(xm, c4_small, mode):
    d, idx = c4_small
    base = xm.Batch(idx, _dev_requests(d))
    kw = {}
    reqs = _dev_requests(d)
    if mode == "graph":
        kw = dict(use_graph=True)
    elif mode == "blocks1":
        kw = dict(persistent_blocks=1)
    elif mode == "blocks8":
        kw = dict(persistent_blocks=8)
    elif mode == "host":
        reqs = _dev_requests(d, on_device=False)
    elif mode == "short_arenas":
        kw = dict(pair_capacity=16, row_capacity=16)
    elif mode == "sorted":
        kw = dict(a_order=xm.A_ORDER_SORTED)
    elif mode == "sorted_graph_short":
        kw = dict(a_order=xm.A_ORDER_SORTED, use_graph=True, pair_capacity=64, row_capacity=64)
    else:
        kw = dict(use_graph=True, pair_capacity=64, row_capacity=64)
    other = xm.Batch(idx, reqs, **kw)
    assert other.info()["total_pairs"] == base.info()["total_pairs"]
    for r in range(len(reqs)):
        _same_view(base.view(r), other.view(r))


def test_batch_fp64_equals_fp32(xm, c4_small):
    d, idx = c4_small
    a = xm.Batch(idx, _dev_requests(d), precision=xm.PREC_FP32)
    b = xm.Batch(idx, _dev_requests(d), precision=xm.PREC_FP64)
    for r in range(len(d["requests"])):
        va, vb = a.view(r), b.view(r)
        for k in ("a_row", "b_row", "count", "best_b", "row_a", "row_b"):
            np.testing.assert_array_equal(_h(va[k]), _h(vb[k]), err_msg=k)
        if va["sep"].numel():
            assert np.max(np.abs(_h(va["sep"]) - _h(vb["sep"]))) <= SEP_TOL


def test_batch_oracle_parity(xm, c4_small):
    d, idx = c4_small
    batch = xm.Batch(idx, _dev_requests(d))
    n_b = d["b_lon"].size
    for r in (0, 5, 11, 23):
        q = d["requests"][r]
        ref = oracle.match(q["lon"], q["lat"], d["b_lon"], d["b_lat"], **q["region"])
        assert ref["border_a"].size == 0
        v = batch.view(r)
        np.testing.assert_array_equal(_h(v["a_row"]), ref["a_row"])
        np.testing.assert_array_equal(_h(v["b_row"]), ref["b_row"])
        if ref["sep"].size:
            assert np.max(np.abs(_h(v["sep"]) - ref["sep"])) <= SEP_TOL
        bb = oracle.best(ref, len(q["lon"]))
        np.testing.assert_array_equal(_h(v["best_b"]), bb["best_b"])
        sel = oracle.selected_pairs(ref, len(q["lon"]), "all" if q["join_selection"] == 1 else "best")
        exp = oracle.join(sel, len(q["lon"]), n_b, q["join"])
        full = batch.join(r)
        np.testing.assert_array_equal(_h(full.a_row), exp["a_row"])
        np.testing.assert_array_equal(_h(full.b_row), exp["b_row"])


def test_batch_invalid_request_names_it(xm, c4_small):
    d, idx = c4_small
    reqs = _dev_requests(d)[:5]
    bad = np.array(d["requests"][3]["lat"], copy=True)
    bad[7] = np.nan
    reqs[3] = dict(reqs[3], lat=_cuda(bad))
    with pytest.raises(xm.XMError, match="request 3"):
        xm.Batch(idx, reqs)


def test_batch_empty_and_tiny(xm, c4_small):
    _, idx = c4_small
    import torch

    e = torch.empty(0, dtype=torch.float64, device="cuda")
    b = xm.Batch(idx, [dict(lon=e, lat=e, a=1.0), dict(lon=_cuda([10.0]), lat=_cuda([0.0]), a=1.0)])
    assert b.view(0)["count"].numel() == 0
    assert b.view(1)["count"].numel() == 1
    assert xm.Batch(idx, []).info()["total_a"] == 0
