"""The match in two calls (xm_match_async, xm_match_wait) against xm_match.

The two-call form must give exactly xm_match's result: with host A and with
device A, in both A orders. It must stay exact with several matches pending at
once on one host thread, each with its own staging of the count reads and its
own fork to the near-tie resolve, waited for in any order, with index builds
queued between them; and when it is waited for on another thread than the one
that queued it, after that thread has ended. A pending match that is never
waited for must leave nothing behind. An error found on the device (A
coordinates out of range) must surface at the wait and leave nothing either."""

import gc
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_08494_gb300 import synth_gpu, xm

    d = synth_gpu.c3(scale=0.005)
    host = {k: d[k].cpu().numpy() for k in ("a_lon", "a_lat", "b_lon", "b_lat")}
    idx = xm.Index(d["b_lon"], d["b_lat"], frame=d["b_frame"], zone_height_arcsec=12.0)
    return xm, torch, d, host, idx


def _arrays(res):
    return [t.cpu().numpy() for t in (res.a_row, res.b_row, res.sep, res.count, res.best_b,
                                      res.best_sep)]


def _same(got, ref, what):
    for name, a, b in zip(("a_row", "b_row", "sep", "count", "best_b", "best_sep"), got, ref):
        np.testing.assert_array_equal(a, b, err_msg=f"{what}: {name}")


def _live(xm, torch):
    gc.collect()
    torch.cuda.synchronize()
    return xm.mem_info()["live_bytes"]


@pytest.mark.parametrize("a_order", ["input", "sorted"])
@pytest.mark.parametrize("where", ["host", "device"])
def test_async_equals_match(env, a_order, where):
    xm, torch, d, host, idx = env
    order = xm.A_ORDER_INPUT if a_order == "input" else xm.A_ORDER_SORTED
    lon, lat = (host["a_lon"], host["a_lat"]) if where == "host" else (d["a_lon"], d["a_lat"])
    kw = dict(frame=d["a_frame"], selection=xm.SEL_ALL | xm.SEL_BEST, a_order=order, **d["region"])
    ref = _arrays(xm.Result(idx, lon, lat, **kw))
    assert ref[0].size > 100
    p = xm.Pending(idx, lon, lat, **kw)
    _same(_arrays(p.wait()), ref, f"{where} A, {a_order} order")
    with pytest.raises(ValueError):
        p.wait()


def test_several_pending_on_one_thread(env):
    xm, torch, d, host, idx = env
    kw = dict(frame=d["a_frame"], selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
    base = _live(xm, torch)
    ref = _arrays(xm.Result(idx, host["a_lon"], host["a_lat"], **kw))
    # sub-catalogues of A: each pending match reads its own count back
    parts = [slice(0, 40_000), slice(40_000, 130_000), slice(130_000, None)]
    refs = []
    for sl in parts:
        r = xm.Result(idx, host["a_lon"][sl], host["a_lat"][sl], **kw)
        refs.append(_arrays(r))
        del r
    streams = [torch.cuda.Stream() for _ in parts]
    pend = []
    others = []
    for sl, st in zip(parts, streams):
        pend.append(xm.Pending(idx, host["a_lon"][sl], host["a_lat"][sl], stream=st, **kw))
        # an index build queued between them (its B copy after this A copy)
        with torch.cuda.stream(st):
            others.append(xm.Index(host["b_lon"], host["b_lat"], frame=d["b_frame"],
                                   zone_height_arcsec=12.0, deferred_check=True))
    for k in (2, 0, 1):  # waited for out of order
        res = pend[k].wait()
        streams[k].synchronize()
        _same(_arrays(res), refs[k], f"part {k}")
        del res
    torch.cuda.synchronize()
    del pend, others
    assert _live(xm, torch) == base
    assert ref[0].size == sum(r[0].size for r in refs)


def test_unwaited_pending_leaves_nothing(env):
    xm, torch, d, host, idx = env
    base = _live(xm, torch)
    p = xm.Pending(idx, host["a_lon"], host["a_lat"], frame=d["a_frame"],
                   selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
    del p
    assert _live(xm, torch) == base


def test_error_surfaces_at_wait(env):
    xm, torch, d, host, idx = env
    base = _live(xm, torch)
    lat = host["a_lat"].copy()
    lat[1234] = 91.0  # found by the count pass on the device
    p = xm.Pending(idx, host["a_lon"], lat, frame=d["a_frame"],
                   selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
    with pytest.raises(xm.XMError) as ex:
        p.wait()
    assert ex.value.status == "XM_EINVAL"
    del p
    assert _live(xm, torch) == base


def test_waited_on_another_thread(env):
    xm, torch, d, host, idx = env
    kw = dict(frame=d["a_frame"], selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
    ref = _arrays(xm.Result(idx, host["a_lon"], host["a_lat"], **kw))
    st = torch.cuda.Stream()
    held = []

    def queue():
        held.append(xm.Pending(idx, host["a_lon"], host["a_lat"], stream=st, **kw))

    t = threading.Thread(target=queue)
    t.start()
    t.join()  # the queuing thread has ended (its side streams' records with it)
    res = held.pop().wait()
    st.synchronize()
    _same(_arrays(res), ref, "waited on another thread")
