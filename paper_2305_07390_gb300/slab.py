"""Slab decomposition of one Dirichlet grid over several ranks.

The paper scales a single grid across one GPU by device tiling (Section 4.1:
one tile per thread block, halos exchanged between tiles at every temporal
block; cost model of Section 5.2.2).  The same scheme carries one level up,
across GPUs: the grid's interior is cut along its slowest axis (y in 2D, z
in 3D) into contiguous slabs, one per rank.  Each rank stores its slab
widened by a ghost region of g = r*t + r rows (planes) on each side, clipped
at the grid's own Dirichlet pad, and runs a temporal block of t steps on
that extended array with ebisu_run, its outermost r rows acting as a fixed
pad.  A row's value after t steps depends on rows at most r*t away, so every
row the rank owns comes out exact -- bit for bit what one run over the whole
grid gives, since each cell sees the same canonical FMA chain -- while the
ghost rows go stale.  Before the next block, each rank sends its first and
last g owned rows to the neighbours whose ghosts they are and receives its
own ghosts from them (one exchange of g rows per side per temporal block).

Owned slabs must be at least g rows thick.  Periodic grids are not
decomposed (the local problems are Dirichlet along the cut axis).

Only the partition, the exchange and the block loop live here; the stepping
function is passed in: `device_step` runs ebisu_run (the GPU path), and the
CPU tests pass the oracle.  Transports: `DistExchange` (torch.distributed
send/recv: NCCL between GPUs, gloo between CPU ranks) and `LocalExchange`
(every slab in one process, rows copied directly -- a single-GPU emulation
that exercises the same ghost logic with the real kernels).
"""
from __future__ import annotations

from dataclasses import dataclass


def partition(n0: int, world: int):
    """Contiguous owned ranges [a, b) of the interior rows 0 .. n0-1, sizes
    differing by at most one, in rank order."""
    if world < 1 or n0 < world:
        raise ValueError("need at least one interior row per rank")
    base, extra = divmod(n0, world)
    out, a = [], 0
    for k in range(world):
        b = a + base + (1 if k < extra else 0)
        out.append((a, b))
        a = b
    return out


@dataclass
class SlabGeometry:
    """One rank's slab in interior row coordinates (the pad is row -r and
    n0 + r - 1 at the grid's ends)."""
    rank: int
    world: int
    n0: int          # interior rows of the whole grid
    radius: int
    depth: int       # steps per temporal block between exchanges (t)
    a: int           # first owned interior row
    b: int           # one past the last owned interior row

    @property
    def ghost(self) -> int:
        return self.radius * self.depth + self.radius

    @property
    def lo(self) -> int:
        """First stored row of the local array (interior coordinates)."""
        return max(self.a - self.ghost, -self.radius)

    @property
    def hi(self) -> int:
        """One past the last stored row of the local array."""
        return min(self.b + self.ghost, self.n0 + self.radius)

    @property
    def local_rows(self) -> int:
        return self.hi - self.lo

    @property
    def local_interior(self) -> int:
        """Interior rows of the local problem (its outermost r rows are its pad)."""
        return self.local_rows - 2 * self.radius

    def owned_slice(self):
        """The owned rows inside the local array."""
        return slice(self.a - self.lo, self.b - self.lo)

    def sends(self):
        """(neighbour rank, local row slice) of the owned rows each neighbour
        keeps as ghosts."""
        out = []
        g = self.ghost
        if self.rank > 0:
            out.append((self.rank - 1, slice(self.a - self.lo, self.a - self.lo + g)))
        if self.rank < self.world - 1:
            out.append((self.rank + 1, slice(self.b - self.lo - g, self.b - self.lo)))
        return out

    def recvs(self):
        """(neighbour rank, local row slice) of this rank's ghost rows that a
        neighbour owns."""
        out = []
        if self.rank > 0:
            out.append((self.rank - 1, slice(0, self.a - self.lo)))
        if self.rank < self.world - 1:
            out.append((self.rank + 1, slice(self.b - self.lo, self.hi - self.lo)))
        return out


def geometries(n0: int, radius: int, depth: int, world: int):
    """Every rank's slab; raises if a slab is thinner than its ghost depth
    (a neighbour's ghost would then span more than one rank)."""
    gs = [SlabGeometry(k, world, n0, radius, depth, a, b) for k, (a, b) in enumerate(partition(n0, world))]
    for g in gs:
        if world > 1 and g.b - g.a < g.ghost:
            raise ValueError(f"slab of {g.b - g.a} rows is thinner than the ghost depth {g.ghost}: "
                             "use fewer ranks or a shallower exchange depth")
    return gs


def scatter(grid, geo: SlabGeometry):
    """A copy of one rank's local array, cut from the whole stored grid
    (numpy or torch; the cut is along the first axis)."""
    view = grid[geo.lo + geo.radius:geo.hi + geo.radius]
    return view.clone() if hasattr(view, "clone") else view.copy()


def gather_into(out, local, geo: SlabGeometry):
    """Write a rank's owned rows (and, at the grid's ends, the pad rows it
    holds) into the whole stored grid `out`."""
    r = geo.radius
    a = geo.a if geo.rank > 0 else geo.lo
    b = geo.b if geo.rank < geo.world - 1 else geo.hi
    out[a + r:b + r] = local[a - geo.lo:b - geo.lo]


class LocalExchange:
    """All slabs in one process: ghost rows are copied from the neighbour's
    owned rows directly."""

    def exchange(self, geos, locals_):
        for g, loc in zip(geos, locals_):
            for nb, sl in g.recvs():
                h = geos[nb]
                # the same global rows in the neighbour's array
                a = sl.start + g.lo - h.lo
                loc[sl] = locals_[nb][a:a + (sl.stop - sl.start)]


class DistExchange:
    """One slab per rank over torch.distributed (point-to-point send/recv;
    NCCL between GPUs, gloo between CPU ranks)."""

    def __init__(self, dist):
        self.dist = dist

    def exchange(self, geo: SlabGeometry, local):
        dist = self.dist
        ops = []
        bufs = []
        for nb, sl in geo.sends():
            ops.append(dist.P2POp(dist.isend, local[sl].contiguous(), nb))
        for nb, sl in geo.recvs():
            buf = local[sl].clone()
            bufs.append((sl, buf))
            ops.append(dist.P2POp(dist.irecv, buf, nb))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for sl, buf in bufs:
            local[sl] = buf


def run_blocks(steps: int, depth: int, step_fn, exchange_fn):
    """The block loop: `step_fn(t)` advances every local array by t steps
    (t <= depth), `exchange_fn()` refreshes the ghosts; the last block may be
    shorter and needs no exchange after it."""
    done = 0
    while done < steps:
        t = min(depth, steps - done)
        step_fn(t)
        done += t
        if done < steps:
            exchange_fn()


def device_step(plan, x, y, ws, t, stream=None):
    """One temporal block on the GPU path: t steps of `plan` (the local
    problem: local_interior x the other extents) from x into y."""
    plan.run(x, y, t, ws, stream=stream)
    return y
