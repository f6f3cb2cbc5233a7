"""Catalogue 1 split across processes (paper §2.3), one process per GPU.

The paper's tool gives each process a part of the first catalogue and the
whole second catalogue. Here rank r of a job of `world` ranks matches the
contiguous slice ``shard_range(n_a, r, world)`` of the A rows against its own
copy of the B index; matching needs no exchange. The B-side joins (all from
2, 1 or 2, 2 not 1, 1 xor 2) need the B rows matched by any slice: each rank
marks its own (``Result.mark_b``), one OR-reduction over the ranks gives the
union, and each rank writes its slice's join rows against it
(``Result.join_shard``); the last rank also writes the B-only rows. The rows
of the ranks concatenated in rank order are the rows the whole catalogue's
join would give, in the same order.

Every step on the data runs in the library's kernels; this module only
splits the rows and moves the bitset between ranks (torch.distributed: an
all-reduce with bitwise OR where the backend has it, gloo; otherwise an
all-gather of the ranks' bitsets, OR-ed here).
"""

from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [lo, hi) of rank `rank` when n rows are split into `world`
    contiguous slices of sizes differing by at most one (earlier ranks take
    the larger ones)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad split: n={n}, rank={rank}, world={world}")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def or_reduce_bits(bits, group=None):
    """In place: every rank's ``bits`` (int32 words) becomes the bitwise OR
    of all ranks' bitsets. Without an initialised process group it is left
    as it is (one rank)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return bits
    if dist.get_backend(group) == "gloo":
        dist.all_reduce(bits, op=dist.ReduceOp.BOR, group=group)
        return bits
    world = dist.get_world_size(group)
    gathered = torch.empty((world,) + tuple(bits.shape), dtype=bits.dtype, device=bits.device)
    dist.all_gather_into_tensor(gathered, bits.contiguous(), group=group)
    acc = gathered[0].clone()
    for k in range(1, world):
        acc.bitwise_or_(gathered[k])
    bits.copy_(acc)
    return bits


def match_shard(index, lon, lat, rank: int, world: int, **match_kw):
    """This rank's slice of catalogue A matched against the index: returns
    (result, first row of the slice). Per-source region columns in
    ``match_kw`` (a_col, b_col, pa_col) are sliced with the positions."""
    from . import xm

    lo, hi = shard_range(len(lon), rank, world)
    kw = dict(match_kw)
    for k in ("a_col", "b_col", "pa_col"):
        if kw.get(k) is not None:
            kw[k] = kw[k][lo:hi]
    return xm.Result(index, lon[lo:hi], lat[lo:hi], **kw), lo


def join_shard(result, a_row_offset: int, join_type: str, selection=None, rank=None,
               world=None, group=None):
    """This rank's join rows (see the module text): the union of the matched
    B rows over the ranks, then the rows of this slice; the last rank writes
    the B-only rows."""
    import torch
    import torch.distributed as dist

    from . import xm

    selection = xm.SEL_ALL if selection is None else selection
    if world is None:
        world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    if rank is None:
        rank = dist.get_rank(group) if dist.is_available() and dist.is_initialized() else 0
    bits = torch.zeros((result.n_b + 31) // 32, dtype=torch.int32, device="cuda")
    result.mark_b(bits, selection)
    or_reduce_bits(bits, group)
    return result.join_shard(join_type, bits, a_row_offset, rank == world - 1, selection)
