"""Host logic of the time decomposition (no GPU): the cut of T into slabs, the extended link slices a
slab loads, the slab's range of a global even/odd field, and the halo exchange and sums of
TorchHaloComm on two and three gloo ranks with CPU tensors (rank r's recv_hi must hold rank r+1's
send_lo, its recv_lo rank r-1's send_hi, periodically)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_0910_0262_gb300 import slab, synth
from oracle.lattice import split_eo


@pytest.mark.parametrize("T,world", [(8, 1), (8, 2), (16, 3), (16, 4), (10, 4), (4, 2)])
def test_slab_bounds_tile_time(T, world):
    covered = []
    for r in range(world):
        t0, tl = slab.slab_bounds(T, world, r)
        assert t0 % 2 == 0 and tl % 2 == 0 and tl >= 2
        covered += list(range(t0, t0 + tl))
    assert covered == list(range(T))
    with pytest.raises(ValueError):
        slab.slab_bounds(T, T, 0)          # slabs thinner than two slices
    with pytest.raises(ValueError):
        slab.slab_bounds(T + 1, world, 0)  # odd T


def test_extended_links_wrap_in_time():
    dims = (2, 2, 2, 6)
    U, _ = synth.make_problem(dims, 0.2, 3)
    E = slab.extended_links(U, 0, 2)
    assert E.shape == (6,) + U.shape[1:]
    for k, t in enumerate([4, 5, 0, 1, 2, 3]):
        assert np.array_equal(E[k], U[t])
    Et = slab.extended_links(torch.from_numpy(U), 4, 2)
    for k, t in enumerate([2, 3, 4, 5, 0, 1]):
        assert torch.equal(Et[k], torch.from_numpy(U[t]))


@pytest.mark.parametrize("t0,tl", [(0, 2), (2, 4), (4, 4), (0, 8)])
def test_slab_rows_are_the_sub_lattice_fields(t0, tl):
    """The rows slab_rows names of a global even (odd) field are the even (odd) field of the sub-lattice
    of time slices t0 .. t0+tl-1, in its own canonical order."""
    dims = (4, 2, 2, 8)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((8, 2, 2, 4, 4, 3)) + 1j * rng.standard_normal((8, 2, 2, 4, 4, 3))
    fe, fo = split_eo(f, dims)
    sub = f[t0:t0 + tl]
    se, so = split_eo(sub, (4, 2, 2, tl))
    a, b = slab.slab_rows(dims, t0, tl)
    assert np.array_equal(fe[a:b], se) and np.array_equal(fo[a:b], so)


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
    comm = slab.TorchHaloComm()
    n = 40
    send_lo = torch.full((n,), 100 * rank + 1, dtype=torch.uint8)
    send_hi = torch.full((n,), 100 * rank + 2, dtype=torch.uint8)
    recv_lo = torch.zeros(n, dtype=torch.uint8)
    recv_hi = torch.zeros(n, dtype=torch.uint8)
    comm.exchange(send_lo, send_hi, recv_lo, recv_hi)
    vals = torch.tensor([1.0 + rank, 0.5 * rank], dtype=torch.float64)
    comm.allreduce(vals)
    out[rank] = (int(recv_lo[0]), int(recv_lo[-1]), int(recv_hi[0]), int(recv_hi[-1]), vals.tolist())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_and_sums_on_gloo(world):
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
    for r in range(world):
        lo0, lo1, hi0, hi1, vals = out[r]
        below, above = (r - 1) % world, (r + 1) % world
        assert lo0 == lo1 == 100 * below + 2      # the lower slab's send_hi
        assert hi0 == hi1 == 100 * above + 1      # the upper slab's send_lo
        assert vals == [sum(1.0 + k for k in range(world)), sum(0.5 * k for k in range(world))]


def test_single_rank_exchange_is_a_self_copy():
    class Solo(slab.TorchHaloComm):
        def __init__(self):
            self.world, self.rank, self.upper, self.lower = 1, 0, 0, 0
    c = Solo()
    a, b = torch.arange(5.0), torch.arange(5.0) + 10
    lo, hi = torch.zeros(5), torch.zeros(5)
    c.exchange(a, b, lo, hi)
    assert torch.equal(hi, a) and torch.equal(lo, b)
