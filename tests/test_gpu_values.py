"""The Exact Value functional case (paper §2.1) on the GPU (xm_match_values)
against the oracle: pairs of equal key values in canonical order, the
lowest-row best pair, and the joins of §2.2 over them."""

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


def _h(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def _check(xm, res, a, b):
    ref = oracle.match_values(a, b)
    np.testing.assert_array_equal(_h(res.a_row), ref["a_row"])
    np.testing.assert_array_equal(_h(res.b_row), ref["b_row"])
    assert np.all(_h(res.sep) == 0)
    bb = oracle.best(ref, a.size)
    np.testing.assert_array_equal(_h(res.best_b), bb["best_b"])
    np.testing.assert_array_equal(_h(res.count), np.bincount(ref["a_row"], minlength=a.size))
    return ref


@pytest.mark.parametrize("device_input", [True, False])
def test_int64_keys_with_repeats(xm, device_input):
    g = synth.rng(5)
    a = g.integers(-5000, 5000, 200_000)
    b = g.integers(-5000, 5000, 150_000)
    conv = _cuda if device_input else np.asarray
    res = xm.ValueResult(conv(a), conv(b))
    ref = _check(xm, res, a, b)
    assert ref["a_row"].size > 1_000_000
    for join in ("and", "or", "not1_2", "xor"):
        for sel, name in ((xm.SEL_ALL, "all"), (xm.SEL_BEST, "best")):
            exp = oracle.join(oracle.selected_pairs(ref, a.size, name), a.size, b.size, join)
            rows = res.join(join, sel)
            np.testing.assert_array_equal(_h(rows.a_row), exp["a_row"])
            np.testing.assert_array_equal(_h(rows.b_row), exp["b_row"])


def test_large_and_extreme_int64_keys(xm):
    g = synth.rng(6)
    ids = synth.unique_ids(300_000, 77)
    b = np.concatenate([ids, ids[:1000], np.array([-(2**63), 2**63 - 1, 0, -1], np.int64)])
    a = np.concatenate([ids[::3], g.integers(0, 2**62, 50_000),
                        np.array([2**63 - 1, -(2**63), -1, 0, 1], np.int64)])
    _check(xm, xm.ValueResult(_cuda(a), _cuda(b)), a, b)


def test_float64_keys_zero_nan_inf(xm):
    g = synth.rng(7)
    base = np.round(g.normal(0, 100, 50_000), 1)
    a = np.concatenate([base, [0.0, -0.0, np.nan, np.inf, -np.inf, 1e-310, -1e-310]])
    b = np.concatenate([base[::2], [-0.0, 0.0, np.nan, np.inf, -np.inf, 1e-310, 5e-324]])
    _check(xm, xm.ValueResult(_cuda(a), _cuda(b)), a, b)


def test_empty_and_single(xm):
    e = np.empty(0, np.int64)
    res = xm.ValueResult(_cuda(e), _cuda(np.array([1, 2], np.int64)))
    assert res.n_pairs == 0 and res.count.numel() == 0
    res = xm.ValueResult(_cuda(np.array([2, 2], np.int64)), _cuda(e))
    assert res.n_pairs == 0 and list(_h(res.best_b)) == [-1, -1]
    one = np.array([42], np.int64)
    _check(xm, xm.ValueResult(_cuda(one), _cuda(one)), one, one)


def test_value_results_have_no_positions(xm):
    a = np.arange(10, dtype=np.int64)
    res = xm.ValueResult(_cuda(a), _cuda(a))
    lon = _cuda(np.linspace(0, 1, 10))
    idx = xm.Index(lon, lon)
    import ctypes

    h = ctypes.c_void_p()
    st = xm.xm_pick_pairs(idx.handle, res.handle, 1, None, ctypes.byref(h))
    assert xm.STATUS[st] in ("XM_EUNSUPPORTED", "XM_EINVAL")


def test_narrow_int64_keys_sort_directly(xm):
    """Keys that differ in at most 32 bits are sorted on their codes (no
    hash): non-negative ids in a 2^20 range, with repeats."""
    g = synth.rng(8)
    b = 1000 + g.integers(0, 1 << 20, 300_000)
    a = np.concatenate([b[::7], 1000 + g.integers(0, 1 << 20, 50_000)])
    _check(xm, xm.ValueResult(_cuda(a), _cuda(b)), a, b)


def _colliding_keys(n_groups, per_group, seed):
    """int64 keys whose 32-bit hash in the library's hashed order collides in
    groups: codes are the inverse of the hash's 64-bit mixer at values that
    share their high 32 bits (the mixer is a bijection)."""
    m64 = (1 << 64) - 1
    c1, c2 = 0xbf58476d1ce4e5b9, 0x94d049bb133111eb
    i1, i2 = pow(c1, -1, 1 << 64), pow(c2, -1, 1 << 64)

    def unxorshift(y, k):
        x = y
        for _ in range(64 // k + 1):
            x = y ^ (x >> k)
        return x & m64

    def unmix(z):
        x = unxorshift(z, 31)
        x = (x * i2) & m64
        x = unxorshift(x, 27)
        x = (x * i1) & m64
        return unxorshift(x, 30)

    g = synth.rng(seed)
    keys = []
    for hi in g.integers(0, 1 << 32, n_groups).tolist():
        for lo in g.integers(0, 1 << 32, per_group).tolist():
            code = unmix((hi << 32) | lo)
            key = code ^ (1 << 63)
            keys.append(key - (1 << 64) if key >= 1 << 63 else key)
    return np.array(keys, np.int64)


def test_hash_collisions_are_told_apart(xm):
    """Groups of distinct keys with one 32-bit hash: each A key matches only
    the B rows of its own value, in ascending B row."""
    col = _colliding_keys(200, 4, 9)
    g = synth.rng(10)
    b = np.concatenate([col, col[::3], g.integers(-(2**62), 2**62, 20_000)])
    b = b[g.permutation(b.size)]
    a = np.concatenate([col[::2], col[1::4], g.integers(-(2**62), 2**62, 5_000)])
    res = xm.ValueResult(_cuda(a), _cuda(b))
    ref = _check(xm, res, a, b)
    assert ref["a_row"].size > 400
