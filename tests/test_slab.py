"""Slab decomposition of one grid over ranks (paper_2305_07390_gb300/slab.py),
checked on the CPU with the oracle as the stepping function.

Every cell's value depends only on the canonical FMA chain over its
neighbours, so a decomposed run must equal one run over the whole grid bit
for bit.  The partition and ghost logic run in one process (LocalExchange)
and over two gloo ranks (DistExchange, torch.distributed send/recv).
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2305_07390_gb300 import slab, synth


def test_partition_covers_the_rows_once():
    for n0, world in [(10, 1), (10, 3), (97, 4), (8, 8)]:
        parts = slab.partition(n0, world)
        assert parts[0][0] == 0 and parts[-1][1] == n0
        assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
        sizes = [b - a for a, b in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab.partition(3, 4)


def test_ghost_depth_and_thin_slabs():
    gs = slab.geometries(100, 2, 3, 4)  # ghost 2*3 + 2 = 8 rows
    assert all(g.ghost == 8 for g in gs)
    assert gs[0].lo == -2 and gs[-1].hi == 102  # clipped at the grid's pad
    assert gs[1].lo == gs[1].a - 8 and gs[1].hi == gs[1].b + 8
    # a neighbour's ghost rows are rows it owns, the same rows on both sides
    for g in gs:
        for nb, sl in g.recvs():
            h = gs[nb]
            rows = range(g.lo + sl.start, g.lo + sl.stop)
            assert h.a <= rows[0] and rows[-1] < h.b
            sent = [s for k, s in h.sends() if k == g.rank][0]
            assert range(h.lo + sent.start, h.lo + sent.stop) == rows
    with pytest.raises(ValueError):
        slab.geometries(30, 2, 5, 4)  # 7-8 rows per slab, ghost 12


def _decomposed_oracle(g, shape, r, c, steps, depth, world, ndim):
    geos = slab.geometries(g.shape[0] - 2 * r, r, depth, world)
    locs = [slab.scatter(g, geo) for geo in geos]

    def step(t):
        for i, loc in enumerate(locs):
            locs[i] = oracle.run(loc, shape, r, c, synth.DIRICHLET, t)

    slab.run_blocks(steps, depth, step, lambda: slab.LocalExchange().exchange(geos, locs))
    out = np.full_like(g, np.nan)
    for geo, loc in zip(geos, locs):
        slab.gather_into(out, loc, geo)
    return out


@pytest.mark.parametrize("ndim,dims,shape,r", [(2, (61, 45), 0, 1), (2, (80, 33), 1, 2), (2, (70, 40), 0, 3),
                                               (3, (40, 9, 11), 1, 1), (3, (36, 10, 8), 0, 2)])
@pytest.mark.parametrize("world,depth,steps", [(2, 3, 7), (3, 2, 9), (4, 1, 5), (1, 4, 6)])
def test_local_exchange_equals_whole_grid(ndim, dims, shape, r, world, depth, steps):
    if (dims[0] // world) < r * depth + r:
        pytest.skip("slabs thinner than the ghost depth")
    g, c = synth.problem(ndim, dims, shape, r, synth.DIRICHLET, seed=61 + world)
    whole = oracle.run(g, shape, r, c, synth.DIRICHLET, steps)
    dec = _decomposed_oracle(g, shape, r, c, steps, depth, world, ndim)
    assert np.array_equal(dec, whole)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, depth, steps, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, shape, dims = 2, 1, (64, 37)
    g, c = synth.problem(2, dims, shape, r, synth.DIRICHLET, seed=71)
    geo = slab.geometries(dims[0], r, depth, world)[rank]
    loc = torch.from_numpy(slab.scatter(g, geo))
    ex = slab.DistExchange(dist)

    def step(t):
        loc.copy_(torch.from_numpy(oracle.run(loc.numpy(), shape, r, c, synth.DIRICHLET, t)))

    slab.run_blocks(steps, depth, step, lambda: ex.exchange(geo, loc))
    res = np.full_like(g, np.nan)
    slab.gather_into(res, loc.numpy(), geo)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_whole_grid():
    import torch.multiprocessing as mp
    world, depth, steps = 2, 3, 10
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, depth, steps, out), nprocs=world, start_method="spawn",
                       join=True)
    r, shape, dims = 2, 1, (64, 37)
    g, c = synth.problem(2, dims, shape, r, synth.DIRICHLET, seed=71)
    whole = oracle.run(g, shape, r, c, synth.DIRICHLET, steps)
    merged = np.where(np.isnan(out[0]), out[1], out[0])
    assert not np.isnan(merged).any()
    assert np.array_equal(merged, whole)
