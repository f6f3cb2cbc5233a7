"""Plain FP64 CPU oracle of the sky cross-match -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The CUDA
library never calls it and shares no code with it.

The membership test itself lives in ``xm_oracle.c`` (paper §2.1, Sky
functional case, written out pair by pair in FP64). This module loads it and
adds the two steps of paper §2.2 in plain numpy:

* match selection: *all* the matches, or only the *best* pair of each source
  of the first catalogue (smallest angular separation; equal separations go to
  the lowest row of the second catalogue);
* the join types i)-v): 1 and 2, 1 or 2, all from 1 / all from 2,
  1 not 2 / 2 not 1, 1 xor 2. A row counts as matched when it appears in the
  selected pairs. Rows come as (a_row, b_row, sep_arcsec) with -1 / NaN for
  the missing side, first every row carrying an A source in ascending
  (a_row, b_row), then the rows of unmatched B sources in ascending b_row.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

EQ, GAL = 0, 1
CIRCLE, ELLIPSE, RECT = 0, 1, 2
JOINS = ("and", "or", "all1", "all2", "not1_2", "not2_1", "xor")

_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (plain C, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
    pd = ctypes.POINTER(ctypes.c_double)
    pi64 = ctypes.POINTER(ctypes.c_int64)
    lib.or_match.restype = ctypes.c_void_p
    lib.or_match.argtypes = [i64, pd, pd, i32, i32, pd, pd, pd, d, d, d, d, d, d, i32, i64, pd, pd,
                             i32, pi64, i64, i32, i32, d, ctypes.POINTER(ctypes.c_int)]
    lib.or_result_npairs.restype = i64
    lib.or_result_npairs.argtypes = [ctypes.c_void_p]
    lib.or_result_nborder.restype = i64
    lib.or_result_nborder.argtypes = [ctypes.c_void_p]
    lib.or_result_copy.argtypes = [ctypes.c_void_p, pi64, pi64, pd]
    lib.or_result_copy_border.argtypes = [ctypes.c_void_p, pi64, pi64, pd]
    lib.or_result_copy_dist.argtypes = [ctypes.c_void_p, pd]
    lib.or_result_free.argtypes = [ctypes.c_void_p]
    lib.or_to_equatorial.restype = i32
    lib.or_to_equatorial.argtypes = [i64, pd, pd, i32, pd, pd]
    lib.or_from_equatorial.restype = i32
    lib.or_from_equatorial.argtypes = [i64, pd, pd, i32, pd, pd]
    lib.or_gal_to_eq_matrix.argtypes = [pd]
    lib.or_separation.restype = d
    lib.or_separation.argtypes = [d, d, i32, d, d, i32]
    _lib = lib
    return lib


class OracleError(ValueError):
    """Invalid input, rejected as the library rejects it (XM_EINVAL)."""


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(x, ctype=ctypes.c_double):
    return None if x is None else x.ctypes.data_as(ctypes.POINTER(ctype))


def gal_to_eq_matrix() -> np.ndarray:
    m = np.zeros(9)
    _load().or_gal_to_eq_matrix(_ptr(m))
    return m.reshape(3, 3)


def to_equatorial(lon, lat, frame):
    lon, lat = _f64(lon), _f64(lat)
    ra, dec = np.empty_like(lon), np.empty_like(lat)
    if _load().or_to_equatorial(lon.size, _ptr(lon), _ptr(lat), frame, _ptr(ra), _ptr(dec)):
        raise OracleError("invalid coordinates")
    return ra, dec


def from_equatorial(ra, dec, frame):
    ra, dec = _f64(ra), _f64(dec)
    lon, lat = np.empty_like(ra), np.empty_like(dec)
    if _load().or_from_equatorial(ra.size, _ptr(ra), _ptr(dec), frame, _ptr(lon), _ptr(lat)):
        raise OracleError("invalid coordinates")
    return lon, lat


def separation(lon1, lat1, frame1, lon2, lat2, frame2) -> float:
    return _load().or_separation(lon1, lat1, frame1, lon2, lat2, frame2)


def match(a_lon, a_lat, b_lon, b_lat, *, shape=CIRCLE, a=1.0, b=None, pa=0.0,
          a_col=None, b_col=None, pa_col=None, size_scale=1.0, size_unit_arcsec=1.0,
          pa_zero_deg=0.0, pa_dir=1, a_frame=EQ, b_frame=EQ, subset=None, mode="grid",
          nthreads=None, tau=1e-9):
    """All members of each A source (paper §2.1). Returns a dict with int64
    ``a_row``, ``b_row``, float64 ``sep`` (arcsec) and ``dist`` (normalised
    distance: the region scale that reaches the pair, at most 1 for members)
    in ascending (a_row, b_row), and the borderline candidates ``border_a``,
    ``border_b``, ``border_margin`` (decision margin below ``tau``)."""
    lib = _load()
    a_lon, a_lat, b_lon, b_lat = _f64(a_lon), _f64(a_lat), _f64(b_lon), _f64(b_lat)
    a_col = None if a_col is None else _f64(a_col)
    b_col = None if b_col is None else _f64(b_col)
    pa_col = None if pa_col is None else _f64(pa_col)
    if b is None:
        b = a
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int64)
    nthreads = nthreads or os.cpu_count() or 1
    st = ctypes.c_int(0)
    res = lib.or_match(a_lon.size, _ptr(a_lon), _ptr(a_lat), a_frame, shape, _ptr(a_col),
                       _ptr(b_col), _ptr(pa_col), float(a), float(b), float(pa),
                       float(size_scale), float(size_unit_arcsec), float(pa_zero_deg),
                       int(pa_dir), b_lon.size, _ptr(b_lon), _ptr(b_lat), b_frame,
                       _ptr(sub, ctypes.c_int64), 0 if sub is None else sub.size,
                       {"brute": 0, "grid": 1}[mode], nthreads, float(tau), ctypes.byref(st))
    if not res:
        if st.value == 1:
            raise OracleError("invalid input")
        raise MemoryError("oracle out of memory")
    try:
        n = lib.or_result_npairs(res)
        nb = lib.or_result_nborder(res)
        out = {"a_row": np.empty(n, np.int64), "b_row": np.empty(n, np.int64),
               "sep": np.empty(n, np.float64), "dist": np.empty(n, np.float64),
               "border_a": np.empty(nb, np.int64),
               "border_b": np.empty(nb, np.int64), "border_margin": np.empty(nb, np.float64)}
        lib.or_result_copy(res, _ptr(out["a_row"], ctypes.c_int64),
                           _ptr(out["b_row"], ctypes.c_int64), _ptr(out["sep"]))
        lib.or_result_copy_dist(res, _ptr(out["dist"]))
        lib.or_result_copy_border(res, _ptr(out["border_a"], ctypes.c_int64),
                                  _ptr(out["border_b"], ctypes.c_int64),
                                  _ptr(out["border_margin"]))
    finally:
        lib.or_result_free(res)
    return out


def best(pairs, n_a, tau=1e-9):
    """Best pair of every A source (paper §2.2 "best"): the member with the
    smallest separation, ties to the lowest B row. Returns ``best_b`` (int64,
    -1 when A has no member), ``best_sep`` (NaN when none) and ``near_tie``, the
    A rows whose two smallest separations differ, but by less than tau times
    the smallest (their order may depend on the last ulp; exactly equal ones
    resolve by row on both sides)."""
    a, b, sep = pairs["a_row"], pairs["b_row"], pairs["sep"]
    best_b = np.full(n_a, -1, np.int64)
    best_sep = np.full(n_a, np.nan)
    near = []
    if a.size:
        order = np.lexsort((b, sep, a))  # by a, then sep, then b
        a_s, b_s, s_s = a[order], b[order], sep[order]
        first = np.ones(a_s.size, bool)
        first[1:] = a_s[1:] != a_s[:-1]
        idx = np.nonzero(first)[0]
        best_b[a_s[idx]] = b_s[idx]
        best_sep[a_s[idx]] = s_s[idx]
        second = idx + 1
        ok = second < a_s.size
        second, idx2 = second[ok], idx[ok]
        same_a = a_s[second] == a_s[idx2]
        second, idx2 = second[same_a], idx2[same_a]
        gap = s_s[second] - s_s[idx2]
        # equal separations are not ambiguous: both programs give them to
        # the lowest B row; unequal ones closer than tau may swap
        near = a_s[idx2[(gap > 0) & (gap < tau * s_s[idx2])]]
    return {"best_b": best_b, "best_sep": best_sep, "near_tie": np.asarray(near, np.int64)}


def best_per_b(pairs, n_b, tau=1e-9):
    """Best pair of every B source, the other reading of paper §2.2's "best
    pairs": among the pairs holding B_j, the one of smallest separation, ties
    to the lowest A row. Returns ``best_a`` (int64, -1 when no pair holds B_j),
    ``best_sep`` and ``near_tie`` (B rows), as ``best`` does for A."""
    swapped = {"a_row": pairs["b_row"], "b_row": pairs["a_row"], "sep": pairs["sep"]}
    r = best(swapped, n_b, tau)
    return {"best_a": r["best_b"], "best_sep": r["best_sep"], "near_tie": r["near_tie"]}


PICKS = ("best_b", "mutual")


def pick(pairs, n_a, n_b, kind, tau=1e-9):
    """The pairs kept by a further reading of "best pairs" (paper §2.2):
    "best_b" keeps each B source's best pair, "mutual" the pairs that are the
    best pair of both their A and their B source. Rows in ascending A row,
    then B row, with the near ties of both selections."""
    if kind not in PICKS:
        raise OracleError(kind)
    a, b, sep = pairs["a_row"], pairs["b_row"], pairs["sep"]
    pb = best_per_b(pairs, n_b, tau)
    keep = pb["best_a"][b] == a if a.size else np.zeros(0, bool)
    near_a = np.empty(0, np.int64)
    if kind == "mutual":
        pa = best(pairs, n_a, tau)
        keep = keep & (pa["best_b"][a] == b) if a.size else keep
        near_a = pa["near_tie"]
    order = np.lexsort((b[keep], a[keep]))
    return {"a_row": a[keep][order], "b_row": b[keep][order], "sep": sep[keep][order],
            "near_tie_b": pb["near_tie"], "near_tie_a": near_a}


def best_normalised(pairs, n_a, tau=1e-9):
    """Best pair of every A source by normalised distance (how deep inside
    the region the B source lies) instead of angular separation, the third
    reading of paper §2.2's "best pairs": the member of smallest ``dist``,
    ties to the lowest B row. Returns ``best_b``, ``best_dist`` (NaN when
    none) and ``near_tie`` as ``best`` does."""
    r = best({"a_row": pairs["a_row"], "b_row": pairs["b_row"], "sep": pairs["dist"]}, n_a, tau)
    return {"best_b": r["best_b"], "best_dist": r["best_sep"], "near_tie": r["near_tie"]}


def concentric(pairs, n_a, scales, tau=1e-9):
    """Concentric regions (paper §3, ClumpPopulator): copies of each A
    source's region about the same centre with the same orientation, sizes
    multiplied by ``scales`` (increasing, in (0, 1]: the matched region is
    the outermost). A member lies inside copy k when its normalised distance
    is at most scales[k]. Returns per pair ``level``, the first copy that
    holds it (len(scales) when only the matched region does), per A and copy
    ``n_within`` (int32 [n_a, K], members inside copy k), and ``border``, the
    pair indices whose distance is within tau (relative) of a scale."""
    sc = np.asarray(scales, np.float64)
    if sc.ndim != 1 or sc.size == 0 or np.any(~np.isfinite(sc)) or np.any(sc <= 0) \
            or np.any(sc > 1) or np.any(np.diff(sc) <= 0):
        raise OracleError("scales must increase within (0, 1]")
    d = pairs["dist"]
    # copies that do not hold the pair: those before the first that does
    level = np.sum(~(d[:, None] <= sc[None, :]), axis=1).astype(np.int32)
    within = np.zeros((n_a, sc.size), np.int32)
    for k in range(sc.size):
        np.add.at(within[:, k], pairs["a_row"][d <= sc[k]], 1)
    near = np.nonzero(np.any(np.abs(d[:, None] / sc[None, :] - 1.0) < tau, axis=1))[0] \
        if d.size else np.empty(0, np.int64)
    return {"level": level, "n_within": within, "border": near.astype(np.int64)}


def match_values(a_keys, b_keys):
    """The Exact Value functional case (paper §2.1): A_i and B_j match when
    their key columns hold the same value. Integer keys compare as integers,
    float64 keys as numbers (-0 equals +0; NaN equals nothing). The plain
    definition: B rows grouped by value, each A key looked up. Returns int64
    ``a_row``, ``b_row`` in ascending (a_row, b_row) and ``sep`` (0: the
    values are equal)."""
    a_list = np.asarray(a_keys).tolist()
    b_list = np.asarray(b_keys).tolist()
    rows_of = {}
    for j, v in enumerate(b_list):
        if v == v:  # NaN equals nothing
            rows_of.setdefault(v, []).append(j)
    a_out, b_out = [], []
    for i, v in enumerate(a_list):
        if v == v:
            for j in rows_of.get(v, ()):
                a_out.append(i)
                b_out.append(j)
    a_row = np.array(a_out, np.int64)
    return {"a_row": a_row, "b_row": np.array(b_out, np.int64), "sep": np.zeros(a_row.size)}


def selected_pairs(pairs, n_a, selection, tau=1e-9):
    """The pair set after match selection ("all" or "best")."""
    if selection == "all":
        return {k: pairs[k] for k in ("a_row", "b_row", "sep")}
    bb = best(pairs, n_a, tau)
    rows = np.nonzero(bb["best_b"] >= 0)[0].astype(np.int64)
    return {"a_row": rows, "b_row": bb["best_b"][rows], "sep": bb["best_sep"][rows]}


def join(sel, n_a, n_b, join_type):
    """Join types of paper §2.2 over a selected pair set. Returns int64
    ``a_row``, ``b_row`` and float64 ``sep`` (-1 / NaN for a missing side)."""
    if join_type not in JOINS:
        raise OracleError(join_type)
    a, b, sep = sel["a_row"], sel["b_row"], sel["sep"]
    matched_a = np.zeros(n_a, bool)
    matched_a[a] = True
    matched_b = np.zeros(n_b, bool)
    matched_b[b] = True
    un_a = np.nonzero(~matched_a)[0].astype(np.int64)
    un_b = np.nonzero(~matched_b)[0].astype(np.int64)
    with_pairs = join_type in ("and", "or", "all1", "all2")
    with_un_a = join_type in ("or", "all1", "not1_2", "xor")
    with_un_b = join_type in ("or", "all2", "not2_1", "xor")
    parts_a, parts_b, parts_s = [], [], []
    if with_pairs:
        parts_a.append(a); parts_b.append(b); parts_s.append(sep)
    if with_un_a:
        parts_a.append(un_a); parts_b.append(np.full(un_a.size, -1, np.int64))
        parts_s.append(np.full(un_a.size, np.nan))
    if parts_a:
        ra, rb, rs = np.concatenate(parts_a), np.concatenate(parts_b), np.concatenate(parts_s)
        order = np.lexsort((rb, ra))
        ra, rb, rs = ra[order], rb[order], rs[order]
    else:
        ra, rb, rs = (np.empty(0, np.int64), np.empty(0, np.int64), np.empty(0))
    if with_un_b:
        ra = np.concatenate([ra, np.full(un_b.size, -1, np.int64)])
        rb = np.concatenate([rb, un_b])
        rs = np.concatenate([rs, np.full(un_b.size, np.nan)])
    return {"a_row": ra, "b_row": rb, "sep": rs}
