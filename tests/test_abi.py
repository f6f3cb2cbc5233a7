"""The C ABI library without a GPU: it loads, exports exactly what
include/xm.h declares, and its host-only logic (status strings, argument
validation that precedes any device work, the galactic frame rotation) is
right."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xm.h")


@pytest.fixture(scope="module")
def xm():
    from paper_1611_08494_gb300 import build

    build.build()
    from paper_1611_08494_gb300 import xm as mod

    return mod


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"XM_API\s+[\w\s\*]+?\b(xm_\w+)\s*\(", src)))


def test_exports_match_header(xm):
    declared = _declared()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", xm._LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T " in ln})
    assert exported == declared
    for name in declared:
        assert hasattr(xm.lib, name)


def test_status_strings(xm):
    assert xm.xm_status_str(0) == b"ok"
    assert xm.xm_status_str(1) == b"invalid argument"
    assert xm.xm_status_str(99) == b"unknown status"
    assert xm.xm_version().startswith(b"xm ")


def test_validation_before_device_work(xm):
    # these fail on argument checks, before any CUDA call
    h = ctypes.c_void_p()
    assert xm.xm_build_index(None, None, None, ctypes.byref(h)) == 1
    assert b"bad catalogue" in xm.xm_last_error()
    cols = xm.Columns(None, None, None, 5, 0, 0)
    assert xm.xm_build_index(ctypes.byref(cols), None, None, ctypes.byref(h)) == 1
    lon = np.zeros(3)
    cols = xm.Columns(lon.ctypes.data, lon.ctypes.data, None, 3, 7, 0)
    assert xm.xm_build_index(ctypes.byref(cols), None, None, ctypes.byref(h)) == 1
    cols = xm.Columns(lon.ctypes.data, lon.ctypes.data, None, 3, 0, 0)
    opts = xm.IndexOpts(0.5, 0, 0)
    assert xm.xm_build_index(ctypes.byref(cols), ctypes.byref(opts), None, ctypes.byref(h)) == 1
    assert b"zone height" in xm.xm_last_error()
    assert xm.xm_join(None, 1, 0, None, ctypes.byref(h)) == 1
    assert xm.xm_match(None, None, None, None, None, ctypes.byref(h)) == 1
    assert xm.xm_set_allocator(ctypes.c_void_p(1), None, None) == 1
    assert xm.xm_set_allocator(None, None, None) == 0


def test_every_entry_point_rejects_null_arguments(xm):
    """Each call checks its handles and output pointers before any device
    work: EINVAL with a message, the output handle cleared; the free
    functions accept NULL."""
    EINVAL = 1
    bad = ctypes.c_void_p(0)

    def rejects(status, word):
        assert status == EINVAL
        assert word.encode() in xm.xm_last_error()

    def cleared():
        h = ctypes.c_void_p(12345)  # overwritten with NULL by the call
        return h

    h = cleared()
    rejects(xm.xm_match(None, None, None, None, None, ctypes.byref(h)), "NULL argument")
    assert h.value is None
    h = cleared()
    rejects(xm.xm_join(None, 1, 0, None, ctypes.byref(h)), "NULL result")
    assert h.value is None
    h = cleared()
    rejects(xm.xm_pick_pairs(None, None, 0, None, ctypes.byref(h)), "NULL argument")
    assert h.value is None
    h = cleared()
    rejects(xm.xm_levels_compute(None, None, None, 0, None, ctypes.byref(h)), "NULL argument")
    assert h.value is None
    h = cleared()
    rejects(xm.xm_match_batch(None, None, 0, None, None, ctypes.byref(h)), "bad arguments")
    assert h.value is None
    h = cleared()
    rejects(xm.xm_batch_join(None, 0, None, ctypes.byref(h)), "bad arguments")
    assert h.value is None
    h = cleared()
    rejects(xm.xm_match_values(None, -1, None, 0, 0, 0, 1, None, ctypes.byref(h)), "")
    assert h.value is None
    rejects(xm.xm_match_values(None, 0, None, 0, 0, 0, 1, None, None), "out is NULL")
    rejects(xm.xm_levels_compute(None, None, None, 0, None, None), "out is NULL")
    rejects(xm.xm_pick_pairs(None, None, 0, None, None), "out is NULL")
    rejects(xm.xm_join(None, 1, 0, None, None), "out is NULL")

    n = xm._i64(7)
    rejects(xm.xm_join_noalloc(None, 1, 0, None, None, None, 0, ctypes.byref(n), None), "NULL result")
    assert n.value == 0
    rejects(xm.xm_join_noalloc(None, 1, 0, None, None, None, 0, None, None), "n_rows")
    rejects(xm.xm_result_get(None, None), "NULL argument")
    rejects(xm.xm_rows_get(None, None), "NULL argument")
    rejects(xm.xm_levels_get(None, None), "NULL argument")
    rejects(xm.xm_index_info(None, None, None, None, None), "NULL index")
    rejects(xm.xm_batch_get(None, 0, None), "bad arguments")
    rejects(xm.xm_batch_info(None, None, None, None), "NULL")
    rejects(xm.xm_autotune(None, None, 0, None, 0, None, None), "bad arguments")
    rejects(xm.xm_serve_open(None, None, ctypes.byref(h)), "bad arguments")
    rejects(xm.xm_serve_submit(None, None, None), "bad arguments")
    rejects(xm.xm_serve_poll(None, 0, None), "bad arguments")
    rejects(xm.xm_serve_wait(None, 0, 0), "NULL server")
    rejects(xm.xm_serve_result(None, 0, None), "bad arguments")
    rejects(xm.xm_serve_release(None, 0), "NULL server")
    rejects(xm.xm_serve_get_stats(None, None), "bad arguments")
    rejects(xm.xm_serve_reset_stats(None), "NULL server")
    rejects(xm.xm_copy_to_host(None, None, 8, None), "NULL pointer")
    assert xm.xm_copy_to_host(None, None, 0, None) == 0  # nothing to copy
    rejects(xm.xm_frame_matrix(None), "NULL")
    rejects(xm.xm_get_stats(None), "NULL")
    rejects(xm.xm_prof_read(None, None, None), "NULL name")
    for free in (xm.xm_index_free, xm.xm_result_free, xm.xm_rows_free, xm.xm_levels_free,
                 xm.xm_batch_free, xm.xm_serve_close):
        assert free(bad) == 0


def test_stats_reset(xm):
    xm.reset_stats()
    s = xm.stats()
    assert all(v == 0 for v in s.values())


def test_frame_matrix_agrees_with_oracle_and_pins(xm):
    m = xm.frame_matrix()
    # an independent construction (three axis rotations) of the same frame
    np.testing.assert_allclose(m, oracle.gal_to_eq_matrix(), atol=2e-15)
    np.testing.assert_allclose(m @ m.T, np.eye(3), atol=1e-15)
    assert np.linalg.det(m) == pytest.approx(1.0, abs=1e-15)
    # north galactic pole and galactic centre (IAU definition, Hipparcos values)
    ngp = m @ np.array([0.0, 0.0, 1.0])
    assert np.degrees(np.arctan2(ngp[1], ngp[0])) % 360 == pytest.approx(192.85948, abs=1e-9)
    assert np.degrees(np.arcsin(ngp[2])) == pytest.approx(27.12825, abs=1e-9)
    gc = m @ np.array([1.0, 0.0, 0.0])
    assert np.degrees(np.arctan2(gc[1], gc[0])) % 360 == pytest.approx(266.40499, abs=1e-4)
    assert np.degrees(np.arcsin(gc[2])) == pytest.approx(-28.93617, abs=1e-4)
