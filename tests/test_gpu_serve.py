"""Serving loop (xm_serve_*) and autotuner (xm_autotune).

Requests served by continuous batching give exactly the results of the same
request matched alone, whatever batch they land in; admission follows the
memory budget (a request that could never fit is refused with XM_EBUSY, one
that does not fit yet waits); the latency statistics are consistent; the
autotuner returns one of its candidates and caches the answer."""

import numpy as np
import pytest

from paper_1611_08494_gb300 import synth

pytestmark = pytest.mark.gpu


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
def c4(xm):
    d = synth.c4(seed=77, n_b=1_000_000, n_req=32, a_lo=50, a_hi=30_000)
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]), zone_height_arcsec=10.0)
    return d, idx


def _kw(q, conv):
    reg = {k: (conv(v) if isinstance(v, np.ndarray) else v) for k, v in q["region"].items()}
    return dict(selection=q["selection"], join=q["join"], join_selection=q["join_selection"], **reg)


def _same(v, w):
    for k in ("a_row", "b_row", "count", "best_b", "row_a", "row_b", "sep", "best_sep", "row_sep"):
        np.testing.assert_array_equal(_h(v[k]), _h(w[k]), err_msg=k)
    assert v["n_unmatched_a"] == w["n_unmatched_a"] and v["n_unmatched_b"] == w["n_unmatched_b"]


@pytest.mark.parametrize("slots,graph", [(1, False), (3, False), (2, True)])
def test_served_equals_alone(xm, c4, slots, graph):
    d, idx = c4
    with xm.Server(idx, slots=slots, max_batch_requests=7, use_graph=graph) as srv:
        tickets = []
        for r, q in enumerate(d["requests"]):
            conv = _cuda if r % 2 else np.asarray  # host and device inputs alike
            tickets.append(srv.submit(conv(q["lon"]), conv(q["lat"]), **_kw(q, conv)))
        for t in tickets:
            t.wait(60_000)
        for r, (q, t) in enumerate(zip(d["requests"], tickets)):
            alone = xm.Batch(idx, [dict(lon=_cuda(q["lon"]), lat=_cuda(q["lat"]), **_kw(q, _cuda))])
            _same(t.view(), alone.view(0))
            t.release()
        st = srv.stats()
        assert st["submitted"] == st["completed"] == len(d["requests"])
        assert st["failed"] == 0 and st["refused"] == 0
        assert st["a_sources"] == sum(len(q["lon"]) for q in d["requests"])
        assert 1 <= st["batches"] <= len(d["requests"])
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert st["busy_s"] > 0
        assert st["mem_in_use"] == 0


def test_refuses_what_never_fits(xm, c4):
    d, idx = c4
    q = d["requests"][0]
    with xm.Server(idx, mem_budget_bytes=1 << 20) as srv:
        big = np.zeros(20_000)
        with pytest.raises(xm.XMError, match="XM_EBUSY"):
            srv.submit(big, big, a=1.0)
        t = srv.submit(q["lon"][:100], q["lat"][:100], **_kw(q, lambda v: v[:100]))
        t.wait(60_000)
        assert t.view()["count"].numel() == 100
        t.release()
        assert srv.stats()["refused"] == 1


def test_waits_for_budget(xm, c4):
    d, idx = c4
    q = d["requests"][1]
    n = len(q["lon"])
    # room for one request in flight: the second waits until the first is released
    budget = n * 480 + (64 << 10) + 1000
    with xm.Server(idx, slots=2, mem_budget_bytes=budget) as srv:
        t1 = srv.submit(q["lon"], q["lat"], **_kw(q, np.asarray))
        t1.wait(60_000)
        t2 = srv.submit(q["lon"], q["lat"], **_kw(q, np.asarray))
        with pytest.raises(xm.XMError, match="XM_ETIMEOUT"):
            t2.wait(200)
        assert t2.state() == xm.Ticket.QUEUED
        v1 = {k: (x.clone() if hasattr(x, "clone") else x) for k, x in t1.view().items()}
        t1.release()
        t2.wait(60_000)
        _same(v1, t2.view())
        t2.release()
        assert srv.stats()["mem_in_use"] == 0


def test_invalid_request_and_close_with_queue(xm, c4):
    d, idx = c4
    q = d["requests"][2]
    srv = xm.Server(idx, mem_budget_bytes=len(q["lon"]) * 480 + (64 << 10) + 1000)
    bad = np.array(q["lat"], copy=True)
    bad[0] = np.nan
    # NaN positions are found by the batch kernels: the ticket fails, nothing else does
    tb = srv.submit(q["lon"], bad, **_kw(q, np.asarray))
    with pytest.raises(xm.XMError, match="XM_EINVAL"):
        tb.wait(60_000)
    assert tb.state() == xm.Ticket.FAILED
    tb.release()
    t1 = srv.submit(q["lon"], q["lat"], **_kw(q, np.asarray))
    t1.wait(60_000)
    t2 = srv.submit(q["lon"], q["lat"], **_kw(q, np.asarray))  # stays queued behind t1
    assert t2.state() == xm.Ticket.QUEUED
    srv.close()  # fails the queued ticket and frees everything


def test_autotune_picks_a_candidate_and_caches(xm):
    d = synth.c4(seed=5, n_b=500_000, n_req=6, a_lo=1000, a_hi=20_000)
    reqs = []
    for q in d["requests"]:
        reqs.append(dict(lon=_cuda(q["lon"]), lat=_cuda(q["lat"]), **_kw(q, _cuda)))
    b_lon, b_lat = _cuda(d["b_lon"]), _cuda(d["b_lat"])
    a = xm.autotune(b_lon, b_lat, reqs, zone_heights=(8.0, 16.0), blocks_per_sm=(2, 4))
    assert a["trials"] == 4
    assert a["zone_height_arcsec"] in (8.0, 16.0) and a["persistent_blocks"] in (2, 4)
    assert a["best_ms"] > 0
    b = xm.autotune(b_lon, b_lat, reqs, zone_heights=(8.0, 16.0), blocks_per_sm=(2, 4))
    assert b["trials"] == 0
    assert (b["zone_height_arcsec"], b["persistent_blocks"]) == (a["zone_height_arcsec"],
                                                                 a["persistent_blocks"])
