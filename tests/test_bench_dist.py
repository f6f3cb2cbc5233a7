"""The bench's multi-rank host logic on CPU ranks (gloo, world size 2): the
job time is the slowest rank's, every rank sees it, the whole-job value
counts every rank's units, and the ranks' workloads differ (weak scaling,
no data-path collective)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [12.5, 30.0][rank]
    job = bench.max_over_ranks(local, world, "cpu")
    d = bench.workload(seed_offset=rank, scale=0.0002, device="cpu")
    dist.barrier()
    out[rank] = (job, bench.weak_scaling_value(1000, 10, world, job), float(d["a_lon"][:50].sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 30.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000 * 10 / 0.030)
    assert res[0][2] != res[1][2]  # each rank draws its own catalogue


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(7.0, 1, "cpu") == 7.0
    assert bench.weak_scaling_value(5, 4, 1, 2.0) == pytest.approx(5 * 4 / 0.002)
    assert np.isfinite(bench.weak_scaling_value(1, 1, 8, 1.0))
