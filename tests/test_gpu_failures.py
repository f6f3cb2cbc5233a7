"""Failure detection on the GPU without a GPU fault.

* A bounded wait that runs out: the radix sort's look-back is given a small
  poll budget and one tile that never publishes (a flag nothing sets); the
  index build must return XM_ETIMEOUT -- the kernels end, they never hang --
  and the next build on the same device must succeed and match correctly.
* A failing allocation: a caller allocator (xm_set_allocator) that fails on
  its k-th request, for every k a match makes; the match must return
  XM_ENOMEM (or, where the failed buffer was optional, the right result),
  give back everything it had allocated, and the next match must succeed."""

import ctypes
import gc
import time

import numpy as np
import pytest

import oracle
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


def test_lookback_that_never_sees_its_predecessor_times_out(xm):
    import torch

    g = synth.rng(11)
    b_lon, b_lat = synth.uniform_box(g, 2_000_000, 0.0, 360.0, -90.0, 90.0)  # ~490 tiles
    lon, lat = _cuda(b_lon), _cuda(b_lat)
    assert xm.xm_debug_lookback(4096, 0) == 0
    try:
        t0 = time.perf_counter()
        with pytest.raises(xm.XMError, match="XM_ETIMEOUT"):
            xm.Index(lon, lat)
        torch.cuda.synchronize()
        assert time.perf_counter() - t0 < 60.0
    finally:
        assert xm.xm_debug_lookback(0, -1) == 0
    # the context is still usable: a build and a match give the oracle's pairs
    d = synth.c1()
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]))
    r = xm.Result(idx, _cuda(d["a_lon"]), _cuda(d["a_lat"]), shape=xm.CIRCLE, a=1.0)
    ref = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], a=1.0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(r.a_row.cpu().numpy(), ref["a_row"])
    np.testing.assert_array_equal(r.b_row.cpu().numpy(), ref["b_row"])


def test_lookback_settings_are_validated(xm):
    assert xm.STATUS[xm.xm_debug_lookback(-1, -1)] == "XM_EINVAL"
    assert xm.STATUS[xm.xm_debug_lookback(0, -2)] == "XM_EINVAL"
    assert xm.xm_debug_lookback(0, -1) == 0


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class _CountingAllocator:
    """Device memory from torch's caching allocator; the k-th request (0-based,
    counted from arm()) fails."""

    def __init__(self):
        import torch

        self.torch = torch
        self.live = {}
        self.calls = 0
        self.fail_at = None
        self.alloc_cb = _ALLOC_FN(self._alloc)
        self.free_cb = _FREE_FN(self._free)

    def arm(self, k):
        self.calls = 0
        self.fail_at = k

    def _alloc(self, nbytes, stream, ctx):
        k = self.calls
        self.calls += 1
        if self.fail_at is not None and k == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, stream, ctx):
        if ptr:
            self.live.pop(ptr)
            self.torch.cuda.caching_allocator_delete(ptr)


def test_failed_allocation_returns_enomem_and_leaks_nothing(xm):
    import torch

    d = synth.c2(scale=0.01)
    cols = {k: _cuda(d[k]) for k in ("a_lon", "a_lat", "b_lon", "b_lat")}
    reg = {k: (_cuda(v) if isinstance(v, np.ndarray) else v) for k, v in d["region"].items()}
    al = _CountingAllocator()
    gc.collect()
    torch.cuda.synchronize()
    assert xm.xm_set_allocator(ctypes.cast(al.alloc_cb, ctypes.c_void_p),
                               ctypes.cast(al.free_cb, ctypes.c_void_p), None) == 0
    try:
        idx = xm.Index(cols["b_lon"], cols["b_lat"], frame=d["b_frame"])
        torch.cuda.synchronize()
        held = dict(al.live)  # the index's arrays

        def match():
            return xm.Result(idx, cols["a_lon"], cols["a_lat"], frame=d["a_frame"],
                             selection=xm.SEL_ALL | xm.SEL_BEST, **reg)

        al.arm(None)
        ok = match()
        n_alloc = al.calls
        ref_a, ref_b = ok.a_row.cpu().numpy(), ok.b_row.cpu().numpy()
        del ok
        torch.cuda.synchronize()
        assert al.live == held
        assert n_alloc >= 3
        refused = 0
        for k in range(n_alloc):
            al.arm(k)
            try:
                r = match()
            except xm.XMError as ex:
                assert ex.status == "XM_ENOMEM", str(ex)
                refused += 1
            else:
                # an optional buffer (the speculative pair list) may fail
                # without failing the call: the result must still be right
                np.testing.assert_array_equal(r.a_row.cpu().numpy(), ref_a)
                np.testing.assert_array_equal(r.b_row.cpu().numpy(), ref_b)
                del r
            torch.cuda.synchronize()
            assert al.live == held, f"allocation {k} failed: {len(al.live) - len(held)} arrays leaked"
        assert refused >= n_alloc // 2
        al.arm(None)
        again = match()  # the next call succeeds
        np.testing.assert_array_equal(again.a_row.cpu().numpy(), ref_a)
        np.testing.assert_array_equal(again.b_row.cpu().numpy(), ref_b)
        del again, idx
        gc.collect()
        torch.cuda.synchronize()
        assert al.live == {}
    finally:
        assert xm.xm_set_allocator(None, None, None) == 0
