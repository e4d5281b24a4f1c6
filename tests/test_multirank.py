"""The multi-GPU path of bench.py on CPU: two gloo ranks (one process each,
as under torchrun) check the per-rank integration assignment, the
max-over-ranks timing and the whole-job aggregate.  The X-engine itself has
no data-path collective: channels and integrations are independent."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.rank_integrations(rank, 10)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        dist.barrier()
        ms = 100.0 + 25.0 * rank  # rank 1 is the slowest
        slowest = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        value = bench.aggregate_tops(world, 7, 10, 1.0e12, slowest)
        results[rank] = (gathered, slowest, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as manager:
        results = manager.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        out = dict(results)
    for rank in range(world):
        gathered, slowest, value = out[rank]
        # Disjoint integrations (seeds) per rank, covering 0..19.
        flat = [i for per in gathered for i in per]
        assert sorted(flat) == list(range(20)) and len(set(flat)) == 20
        # Every rank sees the slowest rank's time and the same whole-job value.
        assert slowest == pytest.approx(125.0)
        assert value == pytest.approx(2 * 7 * 10 * 1.0e12 / 0.125 / 1e12)


def test_single_process_identity():
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.rank_integrations(0, 3) == [0, 1, 2]
    assert bench.aggregate_tops(1, 2, 3, 1e12, 1000.0) == pytest.approx(6.0)
