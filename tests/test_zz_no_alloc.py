"""The join entry point that allocates nothing (xm_join_noalloc), for callers
that cannot allocate device memory when they need a join (their own
allocator holds the GPU, or a loop must not enter the driver's allocator).

Called through the C ABI and compared with xm_join on the same result, for
both selections and every join type, twice in a row (its scratch array keeps
the previous call's contents, so the second call checks that nothing stale
leaks through). This file is collected last so a run that stops at the first
failure has run every other test first."""

import ctypes
import gc

import numpy as np
import pytest

from paper_1611_08494_gb300 import synth

pytestmark = pytest.mark.gpu
SEP_TOL = 1e-4  # arcsec, as in the parity tests


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


def _noalloc(xm, res, selection, join_type, capacity):
    import torch

    a = torch.full((max(capacity, 1),), -7, dtype=torch.int64, device="cuda")
    b = torch.full((max(capacity, 1),), -7, dtype=torch.int64, device="cuda")
    s = torch.full((max(capacity, 1),), -7.0, dtype=torch.float64, device="cuda")
    n = ctypes.c_int64(-1)
    st = xm.xm_join_noalloc(res.handle, selection, xm.JOINS[join_type], a.data_ptr(),
                            b.data_ptr(), s.data_ptr(), capacity, ctypes.byref(n),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, n.value, a, b, s


def test_join_noalloc_equals_join(xm):
    d = synth.c1()
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]))
    res = xm.Result(idx, _cuda(d["a_lon"]), _cuda(d["a_lat"]), shape=xm.CIRCLE, a=3.0,
                    selection=xm.SEL_ALL | xm.SEL_BEST)
    for _ in range(2):  # twice in a row: the shared scratch must start clean
        for selection in (xm.SEL_ALL, xm.SEL_BEST):
            for jt in xm.JOINS:
                ref = res.join(jt, selection)
                cap = ref.n + 5
                st, n, a, b, s = _noalloc(xm, res, selection, jt, cap)
                assert st == 0, xm.xm_last_error()
                assert n == ref.n
                np.testing.assert_array_equal(a[:n].cpu().numpy(), ref.a_row.cpu().numpy())
                np.testing.assert_array_equal(b[:n].cpu().numpy(), ref.b_row.cpu().numpy())
                got, exp = s[:n].cpu().numpy(), ref.sep.cpu().numpy()
                np.testing.assert_array_equal(np.isnan(got), np.isnan(exp))
                ok = ~np.isnan(exp)
                if ok.any():
                    assert np.max(np.abs(got[ok] - exp[ok])) <= SEP_TOL
                # rows beyond n are untouched
                assert (a[n:].cpu().numpy() == -7).all()


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def test_join_noalloc_allocates_nothing(xm):
    """With a counting allocator installed (one that would fail every
    request), two joins through the entry point succeed and the allocator is
    never called; torch's allocator sees no change either."""
    import torch

    d = synth.c1()
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]))
    res = xm.Result(idx, _cuda(d["a_lon"]), _cuda(d["a_lat"]), shape=xm.CIRCLE, a=3.0,
                    selection=xm.SEL_ALL | xm.SEL_BEST)
    ref = res.join("or")
    n_ref = ref.n
    cap = n_ref + 5
    outs = [torch.full((cap,), -7, dtype=torch.int64, device="cuda") for _ in range(2)] + \
        [torch.full((cap,), -7.0, dtype=torch.float64, device="cuda")]
    torch.cuda.synchronize()
    calls = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, ctx):
        calls["alloc"] += 1
        return None  # a failing allocator: any use would surface as XM_ENOMEM

    def _free(ptr, stream, ctx):
        calls["free"] += 1

    alloc_cb, free_cb = _ALLOC_FN(_alloc), _FREE_FN(_free)
    gc.collect()  # no earlier object is released while the hook is installed
    before = torch.cuda.memory_allocated()
    assert xm.xm_set_allocator(ctypes.cast(alloc_cb, ctypes.c_void_p),
                               ctypes.cast(free_cb, ctypes.c_void_p), None) == 0
    try:
        for _ in range(2):
            n = ctypes.c_int64(-1)
            st = xm.xm_join_noalloc(res.handle, xm.SEL_ALL, xm.JOINS["or"], outs[0].data_ptr(),
                                    outs[1].data_ptr(), outs[2].data_ptr(), cap, ctypes.byref(n),
                                    torch.cuda.current_stream().cuda_stream)
            assert st == 0, xm.xm_last_error()
            assert n.value == n_ref
        torch.cuda.synchronize()
    finally:
        assert xm.xm_set_allocator(None, None, None) == 0
    assert calls == {"alloc": 0, "free": 0}
    assert torch.cuda.memory_allocated() == before
    np.testing.assert_array_equal(outs[0][:n_ref].cpu().numpy(), ref.a_row.cpu().numpy())
    np.testing.assert_array_equal(outs[1][:n_ref].cpu().numpy(), ref.b_row.cpu().numpy())


def test_join_noalloc_refuses_a_result_of_another_device(xm):
    """A result computed on another device is refused with XM_EINVAL before
    any device work (checked with a forged device id on one GPU: the result's
    handle starts with its device number)."""
    import torch

    d = synth.c1()
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]))
    res = xm.Result(idx, _cuda(d["a_lon"]), _cuda(d["a_lat"]), shape=xm.CIRCLE, a=1.0)
    dev = ctypes.c_int.from_address(res.handle)
    assert dev.value == torch.cuda.current_device()
    a = torch.full((8,), -7, dtype=torch.int64, device="cuda")
    n = ctypes.c_int64(-1)
    dev.value = dev.value + 3
    try:
        st = xm.xm_join_noalloc(res.handle, xm.SEL_ALL, xm.JOINS["and"], a.data_ptr(), a.data_ptr(),
                                a.data_ptr(), 8, ctypes.byref(n),
                                torch.cuda.current_stream().cuda_stream)
        msg = xm.xm_last_error()
    finally:
        dev.value = dev.value - 3
    torch.cuda.synchronize()
    assert xm.STATUS[st] == "XM_EINVAL"
    assert b"belongs to device" in msg
    assert (a.cpu().numpy() == -7).all()


def test_join_noalloc_capacity_and_size_limits(xm):
    d = synth.c1()
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]))
    res = xm.Result(idx, _cuda(d["a_lon"]), _cuda(d["a_lat"]), shape=xm.CIRCLE, a=1.0)
    ref = res.join("or")
    st, n, a, _, _ = _noalloc(xm, res, xm.SEL_ALL, "or", ref.n - 1)
    assert xm.STATUS[st] == "XM_EOVERFLOW" and n == ref.n
    assert (a.cpu().numpy() == -7).all()  # nothing written
    # a result larger than the built-in scratch is refused with a clear error
    g = synth.rng(3)
    b_lon, b_lat = synth.uniform_box(g, (1 << 23) + 1, 0.0, 360.0, -90.0, 90.0)
    big = xm.Index(_cuda(b_lon), _cuda(b_lat), zone_height_arcsec=60.0)
    res2 = xm.Result(big, _cuda([10.0]), _cuda([0.0]), shape=xm.CIRCLE, a=1.0)
    st, n, _, _, _ = _noalloc(xm, res2, xm.SEL_ALL, "and", 10)
    assert xm.STATUS[st] == "XM_EOVERFLOW"
    assert b"takes at most" in xm.xm_last_error()
