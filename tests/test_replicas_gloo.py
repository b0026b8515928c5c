"""The multi-GPU path is replicas only (each rank solves its own problem, no
data-path collective).  Its host logic - per-rank seeds and the max-over-ranks
step time - is checked with two gloo ranks on the CPU."""
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
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(0, rank))
    out[rank] = (t, tuple(seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    manager = mp.get_context("spawn").Manager()  # no fork of this multi-threaded process
    out = manager.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == 2.0 and out[1][0] == 2.0
    assert out[0][1] == (0, 1) and len(set(out[0][1])) == world


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, None) == 3.5
