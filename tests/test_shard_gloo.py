"""Multi-process host logic of the sharded forms, on CPU with the gloo
backend (world size 2): every graph of a batch is owned by exactly one rank,
and the reported time is the maximum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1205_6693_gb300.shard import max_over_ranks, shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, units, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, e = shard_range(units, rank, world)
    owned = torch.zeros(units + 1, dtype=torch.int64)  # last slot: padding
    owned[b:e] = 1
    dist.all_reduce(owned)  # sum of ownership marks over ranks
    t = max_over_ranks(float(rank * 10 + 1))
    marks = owned[:units]
    out[rank] = ((int(marks.min()), int(marks.max())) if units else (1, 1)) + (t,)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("units", [0, 1, 7, 4096])
def test_shards_cover_each_graph_once_and_time_is_max(units):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), units, out), nprocs=world,
                       start_method="spawn")
    for r in range(world):
        lo, hi, t = out[r]
        if units:
            assert lo == 1 and hi == 1
        assert t == 11.0


def test_shard_range_partitions():
    for units in (0, 1, 5, 4096, 4097):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                b, e = shard_range(units, r, world)
                seen.extend(range(b, e))
                assert e - b in (units // world, units // world + 1)
            assert seen == list(range(units))
