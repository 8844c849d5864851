"""Host logic of the multi-rank benchmark on CPU ranks (gloo, world size 2).

Under torchrun every rank advances its own replica of the lattice and the
elapsed time is the maximum over ranks; value = all ranks' node updates / that
time.  No GPU and no data-path collective are involved.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    d = bench.dist_init(world, "gloo")
    elapsed = 1.0 + rank                      # rank 1 is the slowest
    results[rank] = bench.max_over_ranks(elapsed, d, "cpu")
    d.barrier()
    d.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        assert dict(results) == {0: 2.0, 1: 2.0}


def test_single_rank_needs_no_process_group():
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(3.5, None) == 3.5
