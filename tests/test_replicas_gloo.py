"""The multi-GPU path is replicas only (one independent lattice per rank, no exchange
step); its host logic -- distinct per-rank seeds and the max-over-ranks timing --
is checked here with two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(2, rank))
    mx = bench.max_over_ranks(10.0 + 5.0 * rank)
    dist.barrier()
    out[rank] = (tuple(seeds), mx)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    seeds0, mx0 = out[0]
    seeds1, mx1 = out[1]
    assert seeds0 == seeds1 and len(set(seeds0)) == world
    assert mx0 == mx1 == 15.0
