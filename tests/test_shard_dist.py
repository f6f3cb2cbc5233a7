"""Catalogue 1 split across ranks (paper §2.3), host logic on CPU ranks
(gloo, world size 2): the slices cover the A rows once, the OR-reduction of
the matched-B bitsets gives every rank the union, and the merge rule -- each
rank's A-side rows shifted by its first row, B-only rows from the union
written by the last rank, ranks concatenated in order -- reproduces the
oracle's join of the whole catalogue for every join type and selection.
(The slices' pairs come from the oracle here; the GPU test runs the
library's own per-slice kernels.)"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1611_08494_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_range_covers_each_row_once():
    for n in (0, 1, 7, 10, 1000, 10_001):
        for world in (1, 2, 3, 5, 8):
            seen = []
            for r in range(world):
                lo, hi = shard.shard_range(n, r, world)
                assert 0 <= lo <= hi <= n
                assert hi - lo in (n // world, n // world + 1)
                seen.extend(range(lo, hi))
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def _bits_of(rows, n_b):
    """The matched-B bitset of a set of B rows, as the library lays it out:
    bit j % 32 of int32 word j // 32."""
    words = np.zeros((n_b + 31) // 32, np.uint32)
    for j in np.unique(rows):
        words[j >> 5] |= np.uint32(1) << np.uint32(j & 31)
    return words.view(np.int32)


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = synth.c1()
    n_a, n_b = d["a_lon"].size, d["b_lon"].size
    lo, hi = shard.shard_range(n_a, rank, world)
    # the OR-reduction: two different bitsets become their union on both ranks
    mine = np.zeros(4, np.int32)
    mine[rank] = 1 << (3 + rank)
    t = torch.as_tensor(mine.copy())
    shard.or_reduce_bits(t)
    res = {"or": t.numpy().copy()}
    part = oracle.match(d["a_lon"][lo:hi], d["a_lat"][lo:hi], d["b_lon"], d["b_lat"], a=3.0)
    for selection in ("all", "best"):
        sel = oracle.selected_pairs(part, hi - lo, selection)
        bits = torch.as_tensor(_bits_of(sel["b_row"], n_b))
        shard.or_reduce_bits(bits)
        union = bits.numpy().view(np.uint32)
        matched_b = ((union[np.arange(n_b) >> 5] >> (np.arange(n_b) & 31).astype(np.uint32)) & 1) == 1
        for jt in oracle.JOINS:
            rows = oracle.join(sel, hi - lo, n_b, jt)
            a_side = rows["a_row"] >= 0
            a_rows = rows["a_row"][a_side] + lo
            b_rows, seps = rows["b_row"][a_side], rows["sep"][a_side]
            if rank == world - 1 and jt in ("or", "all2", "not2_1", "xor"):
                un_b = np.nonzero(~matched_b)[0]
                a_rows = np.concatenate([a_rows, np.full(un_b.size, -1)])
                b_rows = np.concatenate([b_rows, un_b])
                seps = np.concatenate([seps, np.full(un_b.size, np.nan)])
            res[(selection, jt)] = (a_rows, b_rows, seps)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_whole_join():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    np.testing.assert_array_equal(res[0]["or"], [8, 16, 0, 0])
    np.testing.assert_array_equal(res[1]["or"], [8, 16, 0, 0])
    d = synth.c1()
    n_a, n_b = d["a_lon"].size, d["b_lon"].size
    full = oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], a=3.0)
    for selection in ("all", "best"):
        sel = oracle.selected_pairs(full, n_a, selection)
        for jt in oracle.JOINS:
            exp = oracle.join(sel, n_a, n_b, jt)
            got = [np.concatenate([res[r][(selection, jt)][k] for r in range(world)]) for k in range(3)]
            np.testing.assert_array_equal(got[0], exp["a_row"], err_msg=f"{selection} {jt}")
            np.testing.assert_array_equal(got[1], exp["b_row"], err_msg=f"{selection} {jt}")
            np.testing.assert_array_equal(np.isnan(got[2]), np.isnan(exp["sep"]))
