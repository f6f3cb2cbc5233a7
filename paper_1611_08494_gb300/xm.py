"""Thin ctypes binding of the C ABI in ``include/xm.h`` (same names).

Argument marshalling only: every step of the cross-match runs in the CUDA
library ``_lib/libxm.so``. PyTorch provides device memory and streams; inputs
may be CUDA tensors (used in place), CPU tensors or numpy arrays (copied by
the library). Outputs are zero-copy CUDA tensors that keep their result
handle alive. Importing this module without the built library raises: there
is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libxm.so")

EQ, GAL = 0, 1
CIRCLE, ELLIPSE, RECT = 0, 1, 2
SEL_ALL, SEL_BEST = 1, 2
PREC_FP64, PREC_FP32 = 0, 1
A_ORDER_DEFAULT, A_ORDER_SORTED, A_ORDER_INPUT = 0, 1, 2
JOINS = {"and": 0, "or": 1, "all1": 2, "all2": 3, "not1_2": 4, "not2_1": 5, "xor": 6}
STATUS = {0: "XM_OK", 1: "XM_EINVAL", 2: "XM_ENOMEM", 3: "XM_ECUDA", 4: "XM_ETIMEOUT",
          5: "XM_EOVERFLOW", 6: "XM_EBUSY", 7: "XM_EUNSUPPORTED"}

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; "
                      "g.build()'` (the cross-match has no CPU fallback)")
lib = ctypes.CDLL(_LIB_PATH)

_p = ctypes.c_void_p
_i32, _i64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class Columns(ctypes.Structure):
    _fields_ = [("lon_deg", _p), ("lat_deg", _p), ("id", _p), ("n", _i64), ("frame", _i32),
                ("on_device", _i32)]


class Region(ctypes.Structure):
    _fields_ = [("shape", _i32), ("pa_dir", _i32), ("a", _f64), ("b", _f64), ("pa_deg", _f64),
                ("a_col", _p), ("b_col", _p), ("pa_col", _p), ("size_scale", _f64),
                ("size_unit_arcsec", _f64), ("pa_zero_deg", _f64)]


class IndexOpts(ctypes.Structure):
    _fields_ = [("zone_height_arcsec", _f64), ("build_fp64", _i32), ("deferred_check", _i32)]


class MatchOpts(ctypes.Structure):
    _fields_ = [("selection", _i32), ("precision", _i32), ("block", _i32), ("a_order", _i32)]


class ResultView(ctypes.Structure):
    _fields_ = [("n_pairs", _i64), ("n_a", _i64), ("n_b", _i64), ("a_row", _p), ("b_row", _p),
                ("sep_arcsec", _p), ("count", _p), ("best_b_row", _p), ("best_sep_arcsec", _p)]


class LevelsView(ctypes.Structure):
    _fields_ = [("n_pairs", _i64), ("n_a", _i64), ("n_scales", _i32), ("dist", _p),
                ("best_b_row", _p), ("best_dist", _p), ("level", _p), ("n_within", _p)]


class RowsView(ctypes.Structure):
    _fields_ = [("n", _i64), ("a_row", _p), ("b_row", _p), ("sep_arcsec", _p),
                ("n_unmatched_a", _i64), ("n_unmatched_b", _i64)]


class Stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_uint64), ("rechecked", ctypes.c_uint64),
                ("flipped", ctypes.c_uint64), ("members", ctypes.c_uint64),
                ("tie_resolved", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("sort_key_passes", ctypes.c_uint64), ("sort_pay_passes", ctypes.c_uint64)]


def _sig(name, res, *args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


xm_status_str = _sig("xm_status_str", ctypes.c_char_p, _i32)
xm_last_error = _sig("xm_last_error", ctypes.c_char_p)
xm_version = _sig("xm_version", ctypes.c_char_p)
xm_set_allocator = _sig("xm_set_allocator", _i32, _p, _p, _p)
xm_set_cache_limit = _sig("xm_set_cache_limit", _i32, _i64)
xm_free_cached = _sig("xm_free_cached", _i32, _p)
xm_mem_info = _sig("xm_mem_info", _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64))
xm_get_stats = _sig("xm_get_stats", _i32, ctypes.POINTER(Stats))
xm_reset_stats = _sig("xm_reset_stats", _i32)
xm_prof_enable = _sig("xm_prof_enable", _i32, _i32)
xm_prof_read = _sig("xm_prof_read", _i32, ctypes.c_char_p, ctypes.POINTER(_f64),
                    ctypes.POINTER(_i64))
xm_prof_entry = _sig("xm_prof_entry", _i32, _i32, ctypes.POINTER(ctypes.c_char_p),
                     ctypes.POINTER(_f64), ctypes.POINTER(_i64))
xm_build_index = _sig("xm_build_index", _i32, ctypes.POINTER(Columns), ctypes.POINTER(IndexOpts),
                      _p, ctypes.POINTER(_p))
xm_index_free = _sig("xm_index_free", _i32, _p)
xm_index_info = _sig("xm_index_info", _i32, _p, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                     ctypes.POINTER(_f64), ctypes.POINTER(_i64))
xm_match = _sig("xm_match", _i32, _p, ctypes.POINTER(Columns), ctypes.POINTER(Region),
                ctypes.POINTER(MatchOpts), _p, ctypes.POINTER(_p))
xm_match_async = _sig("xm_match_async", _i32, _p, ctypes.POINTER(Columns), ctypes.POINTER(Region),
                      ctypes.POINTER(MatchOpts), _p, ctypes.POINTER(_p))
xm_match_wait = _sig("xm_match_wait", _i32, _p, ctypes.POINTER(_p))
xm_result_free = _sig("xm_result_free", _i32, _p)
xm_result_get = _sig("xm_result_get", _i32, _p, ctypes.POINTER(ResultView))
xm_join = _sig("xm_join", _i32, _p, _i32, _i32, _p, ctypes.POINTER(_p))
xm_result_mark_b = _sig("xm_result_mark_b", _i32, _p, _i32, _p, _p)
xm_join_shard = _sig("xm_join_shard", _i32, _p, _i32, _i32, _p, _i64, _i32, _p, ctypes.POINTER(_p))
xm_rows_free = _sig("xm_rows_free", _i32, _p)
xm_rows_get = _sig("xm_rows_get", _i32, _p, ctypes.POINTER(RowsView))
xm_copy_to_host = _sig("xm_copy_to_host", _i32, _p, _p, ctypes.c_size_t, _p)
xm_join_noalloc = _sig("xm_join_noalloc", _i32, _p, _i32, _i32, _p, _p, _p, _i64,
                       ctypes.POINTER(_i64), _p)
xm_frame_matrix = _sig("xm_frame_matrix", _i32, ctypes.POINTER(_f64))
xm_debug_lookback = _sig("xm_debug_lookback", _i32, _i32, _i32)
xm_measure_peak = _sig("xm_measure_peak", _i32, _i32, ctypes.POINTER(_f64), _p)
PEAKS = {"fp32_fma_tflops": 0, "fp64_fma_tflops": 1, "hbm_read_gbs": 2}


def measure_peaks(stream=None) -> dict:
    """Measured float32 / float64 FMA rates (TFLOP/s) and read-only HBM
    bandwidth (GB/s) of the current device (xm_measure_peak)."""
    out = {}
    for name, what in PEAKS.items():
        v = _f64()
        check(xm_measure_peak(what, ctypes.byref(v), _stream_handle(stream)), "xm_measure_peak")
        out[name] = v.value
    return out
xm_pick_pairs = _sig("xm_pick_pairs", _i32, _p, _p, _i32, _p, ctypes.POINTER(_p))
xm_match_values = _sig("xm_match_values", _i32, _p, _i64, _p, _i64, _i32, _i32, _i32, _p,
                       ctypes.POINTER(_p))
xm_levels_compute = _sig("xm_levels_compute", _i32, _p, _p, ctypes.POINTER(_f64), _i32, _p,
                         ctypes.POINTER(_p))
xm_levels_free = _sig("xm_levels_free", _i32, _p)
xm_levels_get = _sig("xm_levels_get", _i32, _p, ctypes.POINTER(LevelsView))
KEY_INT64, KEY_FLOAT64 = 0, 1
PICKS = {"best_b": 1, "mutual": 2}


class XMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = STATUS.get(status, str(status))
        msg = xm_last_error().decode(errors="replace")
        super().__init__(f"{where}: {self.status}: {msg}")


def check(status: int, where: str) -> None:
    if status != 0:
        raise XMError(status, where)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def set_cache_limit(nbytes: int) -> None:
    """Most bytes of freed device blocks the library keeps per device for
    reuse (0: none; negative: the default, half the device's memory)."""
    check(xm_set_cache_limit(int(nbytes)), "xm_set_cache_limit")


def free_cached(stream=None) -> None:
    """Returns the kept blocks of the current device to the CUDA pool,
    ordered on ``stream``."""
    check(xm_free_cached(_stream_handle(stream)), "xm_free_cached")


def mem_info() -> dict:
    """Device bytes the library holds in live objects and keeps for reuse."""
    live, kept = _i64(), _i64()
    check(xm_mem_info(ctypes.byref(live), ctypes.byref(kept)), "xm_mem_info")
    return {"live_bytes": live.value, "kept_bytes": kept.value}


def _f64_buffer(x, keep: list, on_device: Optional[bool]):
    """Pointer to a contiguous float64 buffer; returns (ptr, is_device)."""
    if x is None:
        return None, on_device
    if isinstance(x, torch.Tensor):
        t = x.detach()
        if t.dtype != torch.float64:
            t = t.to(torch.float64)
        t = t.contiguous()
        keep.append(t)
        return t.data_ptr(), t.is_cuda
    a = np.ascontiguousarray(x, dtype=np.float64)
    keep.append(a)
    return a.ctypes.data, False


def _i64_buffer(x, keep: list):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        t = x.detach().to(torch.int64).contiguous()
        keep.append(t)
        return t.data_ptr()
    a = np.ascontiguousarray(x, dtype=np.int64)
    keep.append(a)
    return a.ctypes.data


def columns(lon, lat, frame=EQ, ids=None, keep=None):
    keep = [] if keep is None else keep
    lp, dev = _f64_buffer(lon, keep, None)
    bp, dev2 = _f64_buffer(lat, keep, None)
    if dev != dev2:
        raise ValueError("lon and lat must both be on the device or both on the host")
    n = len(lon)
    if len(lat) != n:
        raise ValueError("lon and lat differ in length")
    return Columns(lp, bp, _i64_buffer(ids, keep), n, frame, int(bool(dev))), keep


class _DevArray:
    """__cuda_array_interface__ holder that keeps its owner alive."""

    def __init__(self, ptr, n, typestr, owner):
        self.owner = owner
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3,
                                         "strides": None}


def _tensor(ptr, n, typestr, owner):
    if n == 0 or not ptr:
        dt = {"<i8": torch.int64, "<f8": torch.float64, "<i4": torch.int32}[typestr]
        return torch.empty(0, dtype=dt, device="cuda")
    return torch.as_tensor(_DevArray(ptr, n, typestr, owner), device="cuda")


class Index:
    """Resident B index (paper §2.3). ``xm_build_index``."""

    def __init__(self, lon, lat, frame=EQ, ids=None, zone_height_arcsec=0.0, build_fp64=False,
                 deferred_check=False, stream=None):
        cols, keep = columns(lon, lat, frame, ids)
        opts = IndexOpts(float(zone_height_arcsec), int(bool(build_fp64)), int(bool(deferred_check)))
        h = _p()
        check(xm_build_index(ctypes.byref(cols), ctypes.byref(opts), _stream_handle(stream),
                             ctypes.byref(h)), "xm_build_index")
        self.handle = h.value
        self.n = cols.n
        self.frame = frame
        self._keep = keep  # the build may still be reading them (deferred_check)

    def info(self):
        n, z, hb = _i64(), _i64(), _i64()
        h = _f64()
        check(xm_index_info(self.handle, ctypes.byref(n), ctypes.byref(z), ctypes.byref(h),
                            ctypes.byref(hb)), "xm_index_info")
        return {"n": n.value, "zones": z.value, "zone_height_arcsec": h.value,
                "device_bytes": hb.value}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            xm_index_free(h)
            self.handle = None


def region(shape=CIRCLE, a=1.0, b=None, pa=0.0, a_col=None, b_col=None, pa_col=None,
           size_scale=1.0, size_unit_arcsec=1.0, pa_zero_deg=0.0, pa_dir=1, keep=None):
    keep = [] if keep is None else keep
    ap, _ = _f64_buffer(a_col, keep, None)
    bp, _ = _f64_buffer(b_col, keep, None)
    pp, _ = _f64_buffer(pa_col, keep, None)
    return Region(int(shape), int(pa_dir), float(a), float(a if b is None else b), float(pa),
                  ap, bp, pp, float(size_scale), float(size_unit_arcsec), float(pa_zero_deg)), keep


class Pending:
    """A match queued up to its pair count, ``xm_match_async``: the copy of
    host A comes first on the stream's copy queue, so input copies queued
    after it (an index build's) do not hold it up. ``wait()`` takes the
    match's one synchronisation and returns its Result (``xm_match_wait``).
    The A and region columns and the index stay referenced until then."""

    def __init__(self, index: Index, lon, lat, frame=EQ, selection=SEL_ALL | SEL_BEST,
                 precision=PREC_FP32, block=0, a_order=A_ORDER_DEFAULT, stream=None, **region_kw):
        cols, keep = columns(lon, lat, frame)
        reg, keep = region(keep=keep, **region_kw)
        opts = MatchOpts(int(selection), int(precision), int(block), int(a_order))
        h = _p()
        check(xm_match_async(index.handle, ctypes.byref(cols), ctypes.byref(reg),
                             ctypes.byref(opts), _stream_handle(stream), ctypes.byref(h)),
              "xm_match_async")
        self.handle = h.value
        self.index = index
        self._keep = keep

    def wait(self) -> "Result":
        h, self.handle = self.handle, None
        if not h:
            raise ValueError("this match was already waited for")
        r = _p()
        try:
            check(xm_match_wait(h, ctypes.byref(r)), "xm_match_wait")
        finally:
            self._keep = None
        return Result._from_handle(r.value, self.index)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:  # never waited for: the match completes and its result is dropped
            self.handle = None
            r = _p()
            if xm_match_wait(h, ctypes.byref(r)) == 0 and r.value:
                xm_result_free(r.value)


class Result:
    """Members of every A source. ``xm_match``."""

    def __init__(self, index: Index, lon, lat, frame=EQ, selection=SEL_ALL | SEL_BEST,
                 precision=PREC_FP32, block=0, a_order=A_ORDER_DEFAULT, stream=None, **region_kw):
        cols, keep = columns(lon, lat, frame)
        reg, keep = region(keep=keep, **region_kw)
        opts = MatchOpts(int(selection), int(precision), int(block), int(a_order))
        h = _p()
        check(xm_match(index.handle, ctypes.byref(cols), ctypes.byref(reg), ctypes.byref(opts),
                       _stream_handle(stream), ctypes.byref(h)), "xm_match")
        self._adopt(h.value, index)

    @classmethod
    def _from_handle(cls, handle, index):
        self = cls.__new__(cls)
        self._adopt(handle, index)
        return self

    def _adopt(self, handle, index):
        self.handle = handle
        self.index = index
        v = ResultView()
        check(xm_result_get(self.handle, ctypes.byref(v)), "xm_result_get")
        self.view = v
        self.n_pairs, self.n_a, self.n_b = v.n_pairs, v.n_a, v.n_b

    # zero-copy device tensors
    @property
    def a_row(self):
        return _tensor(self.view.a_row, self.n_pairs, "<i8", self)

    @property
    def b_row(self):
        return _tensor(self.view.b_row, self.n_pairs, "<i8", self)

    @property
    def sep(self):
        return _tensor(self.view.sep_arcsec, self.n_pairs, "<f8", self)

    @property
    def count(self):
        return _tensor(self.view.count, self.n_a, "<i4", self)

    @property
    def best_b(self):
        return _tensor(self.view.best_b_row, self.n_a if self.view.best_b_row else 0, "<i8", self)

    @property
    def best_sep(self):
        return _tensor(self.view.best_sep_arcsec, self.n_a if self.view.best_sep_arcsec else 0,
                       "<f8", self)

    def pick(self, kind: str, stream=None) -> "Rows":
        """Best pair per B source ("best_b") or mutual best pairs ("mutual").
        ``xm_pick_pairs``."""
        h = _p()
        check(xm_pick_pairs(self.index.handle, self.handle, PICKS[kind], _stream_handle(stream),
                            ctypes.byref(h)), "xm_pick_pairs")
        rows = Rows.__new__(Rows)
        rows.handle = h.value
        rows.result = self
        v = RowsView()
        check(xm_rows_get(rows.handle, ctypes.byref(v)), "xm_rows_get")
        rows.view = v
        return rows

    def join(self, join_type: str, selection=SEL_ALL, stream=None) -> "Rows":
        return Rows(self, join_type, selection, stream)

    def mark_b(self, bits, selection=SEL_ALL, stream=None) -> None:
        """ORs the B rows of the selected pairs into ``bits`` (a device int32
        tensor of (n_b + 31) // 32 words). ``xm_result_mark_b``."""
        if not (bits.is_cuda and bits.dtype == torch.int32 and bits.is_contiguous()
                and bits.numel() >= (self.n_b + 31) // 32):
            raise ValueError("bits must be a contiguous device int32 tensor of (n_b + 31) // 32 words")
        check(xm_result_mark_b(self.handle, int(selection), bits.data_ptr(), _stream_handle(stream)),
              "xm_result_mark_b")

    def join_shard(self, join_type: str, b_matched, a_row_offset: int, with_b_rows: bool,
                   selection=SEL_ALL, stream=None) -> "Rows":
        """The join rows of this result as one slice of catalogue 1: unmatched
        B rows decided by ``b_matched`` (the OR of every slice's
        ``mark_b``), A rows shifted by ``a_row_offset``, B-only rows written
        only with ``with_b_rows``. ``xm_join_shard``."""
        if not (b_matched.is_cuda and b_matched.dtype == torch.int32 and b_matched.is_contiguous()
                and b_matched.numel() >= (self.n_b + 31) // 32):
            raise ValueError("b_matched must be a contiguous device int32 tensor of (n_b + 31) // 32 words")
        h = _p()
        check(xm_join_shard(self.handle, int(selection), JOINS[join_type], b_matched.data_ptr(),
                            int(a_row_offset), int(bool(with_b_rows)), _stream_handle(stream),
                            ctypes.byref(h)), "xm_join_shard")
        rows = Rows.__new__(Rows)
        rows.handle = h.value
        rows.result = self
        rows._keep = b_matched
        rows._view = None
        return rows

    def levels(self, scales=(), stream=None) -> "Levels":
        """Normalised distance of every pair, the best pair per A source by
        it, and the levels of concentric copies of the regions scaled by
        ``scales`` (increasing, in (0, 1]). ``xm_levels_compute``."""
        return Levels(self, scales, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            xm_result_free(h)
            self.handle = None


class ValueResult(Result):
    """The Exact Value case: A and B rows whose key columns hold the same value.
    ``xm_match_values``. Same views and joins as ``Result``."""

    def __init__(self, a_keys, b_keys, selection=SEL_ALL | SEL_BEST, stream=None):
        keep = []
        ak, bk = a_keys, b_keys
        if isinstance(ak, np.ndarray) or isinstance(bk, np.ndarray):
            ak, bk = np.ascontiguousarray(ak), np.ascontiguousarray(bk)
            on_dev = 0
            pa, pb = ak.ctypes.data, bk.ctypes.data
            dt = ak.dtype
        else:
            ak, bk = ak.contiguous(), bk.contiguous()
            on_dev = int(ak.is_cuda)
            pa, pb = ak.data_ptr(), bk.data_ptr()
            dt = {torch.int64: np.dtype(np.int64), torch.float64: np.dtype(np.float64)}[ak.dtype]
        keep += [ak, bk]
        kt = KEY_INT64 if dt == np.int64 else KEY_FLOAT64
        h = _p()
        check(xm_match_values(pa, len(ak), pb, len(bk), kt, on_dev, int(selection),
                              _stream_handle(stream), ctypes.byref(h)), "xm_match_values")
        self.handle = h.value
        self.index = None
        v = ResultView()
        check(xm_result_get(self.handle, ctypes.byref(v)), "xm_result_get")
        self.view = v
        self.n_pairs, self.n_a, self.n_b = v.n_pairs, v.n_a, v.n_b
        self._keep = keep


class Levels:
    """Normalised distances and concentric levels of a result (paper §2.2,
    §3). ``xm_levels_compute``; device tensors as views."""

    def __init__(self, result: Result, scales=(), stream=None):
        sc = np.ascontiguousarray(np.asarray(scales, dtype=np.float64).reshape(-1))
        h = _p()
        ptr = sc.ctypes.data_as(ctypes.POINTER(_f64)) if sc.size else None
        check(xm_levels_compute(result.index.handle if result.index else None, result.handle, ptr,
                                int(sc.size), _stream_handle(stream), ctypes.byref(h)),
              "xm_levels_compute")
        self.handle = h.value
        self.result = result
        v = LevelsView()
        check(xm_levels_get(self.handle, ctypes.byref(v)), "xm_levels_get")
        self.view = v
        self.n_pairs, self.n_a, self.n_scales = v.n_pairs, v.n_a, v.n_scales

    @property
    def dist(self):
        return _tensor(self.view.dist, self.n_pairs, "<f8", self)

    @property
    def best_b(self):
        return _tensor(self.view.best_b_row, self.n_a, "<i8", self)

    @property
    def best_dist(self):
        return _tensor(self.view.best_dist, self.n_a, "<f8", self)

    @property
    def level(self):
        return _tensor(self.view.level, self.n_pairs if self.n_scales else 0, "<i4", self)

    @property
    def n_within(self):
        """int32 [n_a, n_scales]: members inside each copy."""
        t = _tensor(self.view.n_within, self.n_a * self.n_scales if self.n_scales else 0, "<i4",
                    self)
        return t.view(self.n_a, self.n_scales) if self.n_scales else t

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            xm_levels_free(h)
            self.handle = None


class Rows:
    """Rows of one join type (paper §2.2). ``xm_join``. The join runs
    without a host synchronisation; the first access to the counts or the
    rows reads them (``xm_rows_get``)."""

    def __init__(self, result: Result, join_type: str, selection=SEL_ALL, stream=None):
        h = _p()
        check(xm_join(result.handle, int(selection), JOINS[join_type], _stream_handle(stream),
                      ctypes.byref(h)), "xm_join")
        self.handle = h.value
        self.result = result
        self._view = None

    @property
    def view(self):
        if self._view is None:
            v = RowsView()
            check(xm_rows_get(self.handle, ctypes.byref(v)), "xm_rows_get")
            self._view = v
        return self._view

    @view.setter
    def view(self, v):
        self._view = v

    @property
    def n(self):
        return self.view.n

    @property
    def n_unmatched_a(self):
        return self.view.n_unmatched_a

    @property
    def n_unmatched_b(self):
        return self.view.n_unmatched_b

    @property
    def a_row(self):
        return _tensor(self.view.a_row, self.n, "<i8", self)

    @property
    def b_row(self):
        return _tensor(self.view.b_row, self.n, "<i8", self)

    @property
    def sep(self):
        return _tensor(self.view.sep_arcsec, self.n, "<f8", self)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            xm_rows_free(h)
            self.handle = None


def stats() -> dict:
    s = Stats()
    check(xm_get_stats(ctypes.byref(s)), "xm_get_stats")
    return {k: getattr(s, k) for k, _ in Stats._fields_}


def reset_stats() -> None:
    check(xm_reset_stats(), "xm_reset_stats")


def prof_enable(on: bool) -> None:
    check(xm_prof_enable(int(bool(on))), "xm_prof_enable")


def prof_read(kernel: str):
    ms, n = _f64(), _i64()
    check(xm_prof_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)), "xm_prof_read")
    return ms.value, n.value


def prof_all() -> dict:
    out, i = {}, 0
    while True:
        name, ms, n = ctypes.c_char_p(), _f64(), _i64()
        if xm_prof_entry(i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(n)) != 0:
            return out
        out[name.value.decode()] = (ms.value, n.value)
        i += 1


def frame_matrix() -> np.ndarray:
    m = (_f64 * 9)()
    check(xm_frame_matrix(m), "xm_frame_matrix")
    return np.array(m[:]).reshape(3, 3)


# ---------------------------------------------------------------- batches

class Request(ctypes.Structure):
    _fields_ = [("A", Columns), ("region", Region), ("selection", _i32), ("join_type", _i32),
                ("join_selection", _i32), ("reserved", _i32)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("precision", _i32), ("use_graph", _i32), ("persistent_blocks", _i32),
                ("a_order", _i32), ("pair_capacity", _i64), ("row_capacity", _i64)]


class BatchView(ctypes.Structure):
    _fields_ = [("n_a", _i64), ("n_pairs", _i64), ("a_row", _p), ("b_row", _p), ("sep_arcsec", _p),
                ("count", _p), ("best_b_row", _p), ("best_sep_arcsec", _p), ("n_rows", _i64),
                ("row_a", _p), ("row_b", _p), ("row_sep", _p), ("n_unmatched_a", _i64),
                ("n_unmatched_b", _i64)]


xm_match_batch = _sig("xm_match_batch", _i32, _p, ctypes.POINTER(Request), _i64,
                      ctypes.POINTER(BatchOpts), _p, ctypes.POINTER(_p))
xm_batch_free = _sig("xm_batch_free", _i32, _p)
xm_batch_get = _sig("xm_batch_get", _i32, _p, _i64, ctypes.POINTER(BatchView))
xm_batch_join = _sig("xm_batch_join", _i32, _p, _i64, _p, ctypes.POINTER(_p))
xm_batch_info = _sig("xm_batch_info", _i32, _p, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                     ctypes.POINTER(_f64))


def request(lon, lat, frame=EQ, selection=SEL_ALL | SEL_BEST, join=None, join_selection=SEL_ALL,
            keep=None, **region_kw):
    """One xm_request (paper §2.1 region, §2.2 selection and join)."""
    keep = [] if keep is None else keep
    cols, keep = columns(lon, lat, frame, keep=keep)
    reg, keep = region(keep=keep, **region_kw)
    jt = -1 if join is None else JOINS[join]
    return Request(cols, reg, int(selection), jt, int(join_selection), 0), keep


class Batch:
    """Many requests against one index in one pass. ``xm_match_batch``."""

    def __init__(self, index: Index, requests, precision=PREC_FP32, use_graph=False,
                 persistent_blocks=0, pair_capacity=0, row_capacity=0, a_order=A_ORDER_DEFAULT,
                 stream=None):
        keep = []
        arr = (Request * max(len(requests), 1))()
        for k, rq in enumerate(requests):
            rq = dict(rq)
            r, keep = request(rq.pop("lon"), rq.pop("lat"), keep=keep, **rq)
            arr[k] = r
        opts = BatchOpts(int(precision), int(bool(use_graph)), int(persistent_blocks),
                         int(a_order), int(pair_capacity), int(row_capacity))
        h = _p()
        check(xm_match_batch(index.handle, arr, len(requests), ctypes.byref(opts),
                             _stream_handle(stream), ctypes.byref(h)), "xm_match_batch")
        self.handle = h.value
        self.index = index
        self.n = len(requests)
        self._keep = keep

    def info(self):
        a, p, ms = _i64(), _i64(), _f64()
        check(xm_batch_info(self.handle, ctypes.byref(a), ctypes.byref(p), ctypes.byref(ms)),
              "xm_batch_info")
        return {"total_a": a.value, "total_pairs": p.value, "device_ms": ms.value}

    def view(self, r: int) -> dict:
        v = BatchView()
        check(xm_batch_get(self.handle, r, ctypes.byref(v)), "xm_batch_get")
        return {
            "a_row": _tensor(v.a_row, v.n_pairs, "<i8", self),
            "b_row": _tensor(v.b_row, v.n_pairs, "<i8", self),
            "sep": _tensor(v.sep_arcsec, v.n_pairs, "<f8", self),
            "count": _tensor(v.count, v.n_a, "<i4", self),
            "best_b": _tensor(v.best_b_row, v.n_a if v.best_b_row else 0, "<i8", self),
            "best_sep": _tensor(v.best_sep_arcsec, v.n_a if v.best_sep_arcsec else 0, "<f8", self),
            "row_a": _tensor(v.row_a, v.n_rows, "<i8", self),
            "row_b": _tensor(v.row_b, v.n_rows, "<i8", self),
            "row_sep": _tensor(v.row_sep, v.n_rows, "<f8", self),
            "n_unmatched_a": v.n_unmatched_a, "n_unmatched_b": v.n_unmatched_b,
        }

    def join(self, r: int, stream=None) -> "Rows":
        h = _p()
        check(xm_batch_join(self.handle, r, _stream_handle(stream), ctypes.byref(h)),
              "xm_batch_join")
        rows = Rows.__new__(Rows)
        rows.handle = h.value
        rows.result = self
        v = RowsView()
        check(xm_rows_get(rows.handle, ctypes.byref(v)), "xm_rows_get")
        rows.view = v
        return rows

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            xm_batch_free(h)
            self.handle = None


# ---------------------------------------------------------------- tuning

class TuneSpace(ctypes.Structure):
    _fields_ = [("zone_heights_arcsec", _f64 * 8), ("n_zone_heights", _i32),
                ("blocks_per_sm", _i32 * 4), ("n_blocks", _i32), ("repeats", _i32),
                ("reserved", _i32)]


class Tuned(ctypes.Structure):
    _fields_ = [("zone_height_arcsec", _f64), ("persistent_blocks", _i32), ("trials", _i32),
                ("best_ms", _f64)]


xm_autotune = _sig("xm_autotune", _i32, ctypes.POINTER(Columns), ctypes.POINTER(Request), _i64,
                   ctypes.POINTER(TuneSpace), _i32, _p, ctypes.POINTER(Tuned))


def autotune(b_lon, b_lat, requests, frame=EQ, zone_heights=(), blocks_per_sm=(), repeats=0,
             precision=PREC_FP32, stream=None) -> dict:
    """Timed choice of the index zone height and the batch grid. ``xm_autotune``."""
    keep = []
    cols, keep = columns(b_lon, b_lat, frame, keep=keep)
    arr = (Request * max(len(requests), 1))()
    for k, rq in enumerate(requests):
        rq = dict(rq)
        r, keep = request(rq.pop("lon"), rq.pop("lat"), keep=keep, **rq)
        arr[k] = r
    sp = TuneSpace()
    for k, z in enumerate(zone_heights):
        sp.zone_heights_arcsec[k] = float(z)
    sp.n_zone_heights = len(zone_heights)
    for k, g in enumerate(blocks_per_sm):
        sp.blocks_per_sm[k] = int(g)
    sp.n_blocks = len(blocks_per_sm)
    sp.repeats = int(repeats)
    out = Tuned()
    check(xm_autotune(ctypes.byref(cols), arr, len(requests), ctypes.byref(sp), int(precision),
                      _stream_handle(stream), ctypes.byref(out)), "xm_autotune")
    return {"zone_height_arcsec": out.zone_height_arcsec,
            "persistent_blocks": out.persistent_blocks, "trials": out.trials,
            "best_ms": out.best_ms}


# ---------------------------------------------------------------- serving

class ServeOpts(ctypes.Structure):
    _fields_ = [("slots", _i32), ("max_batch_requests", _i32), ("max_batch_a", _i64),
                ("mem_budget_bytes", _i64), ("precision", _i32), ("use_graph", _i32),
                ("persistent_blocks", _i32), ("reserved", _i32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", _i64), ("completed", _i64), ("failed", _i64), ("refused", _i64),
                ("a_sources", _i64), ("batches", _i64), ("p50_ms", _f64), ("p99_ms", _f64),
                ("max_ms", _f64), ("busy_s", _f64), ("mem_in_use", _i64), ("mem_budget", _i64)]


xm_serve_open = _sig("xm_serve_open", _i32, _p, ctypes.POINTER(ServeOpts), ctypes.POINTER(_p))
xm_serve_submit = _sig("xm_serve_submit", _i32, _p, ctypes.POINTER(Request),
                       ctypes.POINTER(_i64))
xm_serve_poll = _sig("xm_serve_poll", _i32, _p, _i64, ctypes.POINTER(_i32))
xm_serve_wait = _sig("xm_serve_wait", _i32, _p, _i64, _i32)
xm_serve_result = _sig("xm_serve_result", _i32, _p, _i64, ctypes.POINTER(BatchView))
xm_serve_release = _sig("xm_serve_release", _i32, _p, _i64)
xm_serve_get_stats = _sig("xm_serve_get_stats", _i32, _p, ctypes.POINTER(ServeStats))
xm_serve_close = _sig("xm_serve_close", _i32, _p)
xm_serve_reset_stats = _sig("xm_serve_reset_stats", _i32, _p)


class Ticket:
    """One submitted request. Its result tensors keep it alive; the result is
    released when the ticket and its tensors are gone (or by ``release``)."""

    QUEUED, RUNNING, DONE, FAILED = 0, 1, 2, 3

    def __init__(self, server: "Server", tid: int):
        self.server = server
        self.id = tid
        self._released = False

    def state(self) -> int:
        st = _i32()
        check(xm_serve_poll(self.server.handle, self.id, ctypes.byref(st)), "xm_serve_poll")
        return st.value

    def wait(self, timeout_ms: int = -1) -> "Ticket":
        # the wait blocks in C without the GIL (ctypes releases it)
        check(xm_serve_wait(self.server.handle, self.id, int(timeout_ms)), "xm_serve_wait")
        return self

    def view(self) -> dict:
        v = BatchView()
        check(xm_serve_result(self.server.handle, self.id, ctypes.byref(v)), "xm_serve_result")
        return {
            "a_row": _tensor(v.a_row, v.n_pairs, "<i8", self),
            "b_row": _tensor(v.b_row, v.n_pairs, "<i8", self),
            "sep": _tensor(v.sep_arcsec, v.n_pairs, "<f8", self),
            "count": _tensor(v.count, v.n_a, "<i4", self),
            "best_b": _tensor(v.best_b_row, v.n_a if v.best_b_row else 0, "<i8", self),
            "best_sep": _tensor(v.best_sep_arcsec, v.n_a if v.best_sep_arcsec else 0, "<f8", self),
            "row_a": _tensor(v.row_a, v.n_rows, "<i8", self),
            "row_b": _tensor(v.row_b, v.n_rows, "<i8", self),
            "row_sep": _tensor(v.row_sep, v.n_rows, "<f8", self),
            "n_unmatched_a": v.n_unmatched_a, "n_unmatched_b": v.n_unmatched_b,
        }

    def release(self) -> None:
        if not self._released and self.server.handle:
            check(xm_serve_release(self.server.handle, self.id), "xm_serve_release")
        self._released = True

    def __del__(self):
        try:
            if not self._released and self.server.handle and self.state() >= self.DONE:
                xm_serve_release(self.server.handle, self.id)
                self._released = True
        except Exception:
            pass


class Server:
    """Continuous batching of requests against a resident index. ``xm_serve_*``."""

    def __init__(self, index: Index, slots=0, max_batch_requests=0, max_batch_a=0,
                 mem_budget_bytes=0, precision=PREC_FP32, use_graph=False, persistent_blocks=0):
        opts = ServeOpts(int(slots), int(max_batch_requests), int(max_batch_a),
                         int(mem_budget_bytes), int(precision), int(bool(use_graph)),
                         int(persistent_blocks), 0)
        h = _p()
        check(xm_serve_open(index.handle, ctypes.byref(opts), ctypes.byref(h)), "xm_serve_open")
        self.handle = h.value
        self.index = index

    def submit(self, lon, lat, **kw) -> Ticket:
        keep = []
        r, keep = request(lon, lat, keep=keep, **kw)
        t = _i64()
        check(xm_serve_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "xm_serve_submit")
        return Ticket(self, t.value)

    def stats(self) -> dict:
        s = ServeStats()
        check(xm_serve_get_stats(self.handle, ctypes.byref(s)), "xm_serve_get_stats")
        return {k: getattr(s, k) for k, _ in ServeStats._fields_}

    def reset_stats(self) -> None:
        check(xm_serve_reset_stats(self.handle), "xm_serve_reset_stats")

    def close(self) -> None:
        h = getattr(self, "handle", None)
        if h:
            self.handle = None
            xm_serve_close(h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()
