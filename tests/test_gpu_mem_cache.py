"""The device block cache in front of the stream-ordered pool (xm_set_cache_limit,
xm_free_cached, xm_mem_info): blocks freed by one call are reused by later
calls on the same and on other streams without changing any result.

A pipelined run as a throughput-bound caller makes it (index builds two steps
ahead on three low-priority streams, matches and joins on three high-priority
streams that wait for them, results copied out on a further stream, each
step's objects released in their streams' order after a wait on its copy out)
must give every step exactly the rows, separations and best pairs of a serial
run with nothing kept. Kept bytes must shrink while live objects reuse them,
nothing may stay live once every object is gone, a limit of 0 keeps nothing, a
small limit caps what is kept (results unchanged), and xm_free_cached hands
everything back."""

import gc

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_STEPS = 8


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_08494_gb300 import synth_gpu, xm

    d = synth_gpu.c3(scale=0.01)
    host = {k: d[k].cpu().pin_memory() for k in ("a_lon", "a_lat", "b_lon", "b_lat", "b_id")}
    yield xm, torch, d, host
    xm.set_cache_limit(-1)


def _outputs(res, rows):
    return [rows.a_row, rows.b_row, rows.sep, res.best_b, res.best_sep]


def _step(xm, torch, d, host, bs, ms):
    with torch.cuda.stream(bs):
        idx = xm.Index(host["b_lon"], host["b_lat"], frame=d["b_frame"], ids=host["b_id"],
                       zone_height_arcsec=12.0, deferred_check=True)
        built = torch.cuda.Event()
        built.record(bs)
    ms.wait_event(built)
    with torch.cuda.stream(ms):
        res = xm.Result(idx, host["a_lon"], host["a_lat"], frame=d["a_frame"],
                        selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
        rows = res.join("or")
    return idx, res, rows


def _serial(xm, torch, d, host):
    s = torch.cuda.current_stream()
    idx, res, rows = _step(xm, torch, d, host, s, s)
    out = [t.cpu().numpy() for t in _outputs(res, rows)]
    del idx, res, rows
    torch.cuda.synchronize()
    return out


def _pipelined(xm, torch, d, host, n):
    lo, hi = torch.cuda.Stream.priority_range()
    bstreams = [torch.cuda.Stream(priority=lo) for _ in range(3)]
    mstreams = [torch.cuda.Stream(priority=hi) for _ in range(3)]
    out_stream = torch.cuda.Stream(priority=hi)
    keep, got = {}, {}

    def build(k):
        bs = bstreams[k % 3]
        with torch.cuda.stream(bs):
            idx = xm.Index(host["b_lon"], host["b_lat"], frame=d["b_frame"], ids=host["b_id"],
                           zone_height_arcsec=12.0, deferred_check=True)
            built = torch.cuda.Event()
            built.record(bs)
        return idx, built

    def finish(k, ahead):
        idx, built = ahead
        ms = mstreams[k % 3]
        ms.wait_event(built)
        with torch.cuda.stream(ms):
            res = xm.Result(idx, host["a_lon"], host["a_lat"], frame=d["a_frame"],
                            selection=xm.SEL_ALL | xm.SEL_BEST, **d["region"])
            rows = res.join("or")
            done = torch.cuda.Event()
            done.record(ms)
        srcs = _outputs(res, rows)
        out_stream.wait_event(done)
        dst = [torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in srcs]
        with torch.cuda.stream(out_stream):
            for a, b in zip(dst, srcs):
                a.copy_(b, non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(out_stream)
        got[k] = dst
        keep[k] = (idx, res, rows, srcs, copied, (bstreams[k % 3], ms))
        old = keep.pop(k - 2, None)
        if old is not None:  # released in its streams after its copy out
            for st in old[5]:
                st.wait_event(old[4])
            del old

    ahead = {0: build(0), 1: build(1)}
    for k in range(n):
        if k + 2 < n:
            ahead[k + 2] = build(k + 2)
        finish(k, ahead.pop(k))
    for k in sorted(keep):
        for st in keep[k][5]:
            st.wait_event(keep[k][4])
    keep.clear()
    torch.cuda.synchronize()
    return {k: [t.numpy() for t in v] for k, v in got.items()}


def _live_after_gc(xm, torch):
    gc.collect()
    torch.cuda.synchronize()
    return xm.mem_info()


def test_pipelined_reuse_keeps_every_result(env):
    xm, torch, d, host = env
    base = _live_after_gc(xm, torch)["live_bytes"]
    xm.free_cached()
    xm.set_cache_limit(0)
    try:
        ref = _serial(xm, torch, d, host)
        info = _live_after_gc(xm, torch)
        assert info["kept_bytes"] == 0, "a limit of 0 keeps nothing"
        assert info["live_bytes"] == base
    finally:
        xm.set_cache_limit(-1)
    assert ref[0].size > 1000  # the workload has pairs to check

    got = _pipelined(xm, torch, d, host, N_STEPS)
    for k in range(N_STEPS):
        for name, a, b in zip(("a_row", "b_row", "sep", "best_b", "best_sep"), got[k], ref):
            np.testing.assert_array_equal(a, b, err_msg=f"step {k}: {name}")
    info = _live_after_gc(xm, torch)
    assert info["live_bytes"] == base, "every block of the released objects went back"
    assert info["kept_bytes"] > 0


def test_kept_blocks_are_reused_and_handed_back(env):
    xm, torch, d, host = env
    base = _live_after_gc(xm, torch)["live_bytes"]
    ref = _serial(xm, torch, d, host)  # fills the cache with one step's blocks
    kept0 = _live_after_gc(xm, torch)["kept_bytes"]
    assert kept0 > 0
    s = torch.cuda.Stream()  # another stream: its blocks become free on the GPU first
    torch.cuda.synchronize()
    idx, res, rows = _step(xm, torch, d, host, s, s)
    during = xm.mem_info()
    assert during["kept_bytes"] < kept0, "a later call takes kept blocks"
    assert during["live_bytes"] > base
    s.synchronize()
    for a, b in zip([t.cpu().numpy() for t in _outputs(res, rows)], ref):
        np.testing.assert_array_equal(a, b)
    del idx, res, rows
    info = _live_after_gc(xm, torch)
    assert info["live_bytes"] == base
    xm.free_cached()
    torch.cuda.synchronize()
    assert xm.mem_info()["kept_bytes"] == 0


def test_cache_limit_caps_kept_bytes(env):
    xm, torch, d, host = env
    base = _live_after_gc(xm, torch)["live_bytes"]
    ref = _serial(xm, torch, d, host)
    cap = 64 << 20
    xm.free_cached()
    xm.set_cache_limit(cap)
    try:
        for _ in range(3):  # blocks past the cap go back to the pool, oldest first
            got = _serial(xm, torch, d, host)
            info = _live_after_gc(xm, torch)
            assert info["kept_bytes"] <= cap
            assert info["live_bytes"] == base
            for a, b in zip(got, ref):
                np.testing.assert_array_equal(a, b)
    finally:
        xm.set_cache_limit(-1)
