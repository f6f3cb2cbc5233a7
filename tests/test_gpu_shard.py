"""Catalogue 1 split into slices on one GPU (the per-slice kernels of the
multi-process path, run one slice after another): every slice matched
against the same index, their matched-B bitsets OR-ed (xm_result_mark_b),
their join rows written against the union (xm_join_shard) and concatenated
in slice order equal xm_join on the whole catalogue, for every join type and
selection, with the same unmatched counts."""

import numpy as np
import pytest

from paper_1611_08494_gb300 import shard, synth

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


@pytest.mark.parametrize("workload,world", [("c1", 2), ("c1", 3), ("c2", 2)])
def test_slices_in_turn_equal_the_whole(xm, workload, world):
    import torch

    d = synth.c1() if workload == "c1" else synth.c2(scale=0.02)
    reg = {k: (_cuda(v) if isinstance(v, np.ndarray) else v) for k, v in d["region"].items()}
    if workload == "c1":
        reg = dict(shape=0, a=3.0)
    lon, lat = _cuda(d["a_lon"]), _cuda(d["a_lat"])
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]), frame=d["b_frame"])
    kw = dict(frame=d["a_frame"], selection=xm.SEL_ALL | xm.SEL_BEST, **reg)
    whole = xm.Result(idx, lon, lat, **kw)
    parts = [shard.match_shard(idx, lon, lat, r, world, **kw) for r in range(world)]
    assert sum(p.n_a for p, _ in parts) == whole.n_a
    for selection in (xm.SEL_ALL, xm.SEL_BEST):
        bits = torch.zeros((whole.n_b + 31) // 32, dtype=torch.int32, device="cuda")
        for p, _ in parts:
            p.mark_b(bits, selection)
        for jt in xm.JOINS:
            ref = whole.join(jt, selection)
            rows = [p.join_shard(jt, bits, lo, r == world - 1, selection)
                    for r, (p, lo) in enumerate(parts)]
            got_a = np.concatenate([_h(x.a_row) for x in rows])
            got_b = np.concatenate([_h(x.b_row) for x in rows])
            got_s = np.concatenate([_h(x.sep) for x in rows])
            msg = f"{workload} world {world} selection {selection} join {jt}"
            np.testing.assert_array_equal(got_a, _h(ref.a_row), err_msg=msg)
            np.testing.assert_array_equal(got_b, _h(ref.b_row), err_msg=msg)
            np.testing.assert_array_equal(got_s, _h(ref.sep), err_msg=msg)
            assert sum(x.n_unmatched_a for x in rows) == ref.n_unmatched_a, msg
            assert all(x.n_unmatched_b == ref.n_unmatched_b for x in rows), msg


def test_join_shard_validates(xm):
    import torch

    d = synth.c1()
    idx = xm.Index(_cuda(d["b_lon"]), _cuda(d["b_lat"]))
    res = xm.Result(idx, _cuda(d["a_lon"][:100]), _cuda(d["a_lat"][:100]), a=1.0)
    with pytest.raises(ValueError):
        res.mark_b(torch.zeros(3, dtype=torch.int32, device="cuda"))
    bits = torch.zeros((res.n_b + 31) // 32, dtype=torch.int32, device="cuda")
    with pytest.raises(xm.XMError, match="XM_EINVAL"):
        res.join_shard("or", bits, -1, True)
