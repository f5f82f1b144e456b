"""Slab decomposition with the GPU kernels: several slabs of one grid on one
GPU, ghost rows refreshed between temporal blocks (LocalExchange), each
slab stepped by ebisu_run on its own plan.  The gathered result must equal
one ebisu_run over the whole grid bit for bit.  (Stochastic rounding draws
its bits from the cell's index in the stored array and the step within the
run, which differ between a slab and the whole grid, so it is not part of
this equality.)"""
import pytest

from paper_2305_07390_gb300 import slab, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _eb():
    from paper_2305_07390_gb300 import ebisu
    return ebisu


@pytest.mark.parametrize("ndim,dims,shape,r,dtype", [(2, (600, 700), 1, 2, 0), (2, (512, 900), 0, 1, 1),
                                                     (2, (400, 300), 1, 1, 2), (3, (90, 40, 100), 0, 1, 0),
                                                     (3, (72, 30, 80), 1, 1, 1)])
@pytest.mark.parametrize("world,depth,steps", [(3, 4, 21), (2, 7, 14)])
def test_slabs_equal_whole_grid(ndim, dims, shape, r, dtype, world, depth, steps):
    eb = _eb()
    g, c = synth.problem(ndim, dims, shape, r, synth.DIRICHLET, seed=81)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    whole_plan = eb.Plan(ndim, dims, shape, r, c, dtype, eb.DIRICHLET)
    ws = whole_plan.workspace()
    ref = torch.empty_like(x)
    whole_plan.run(x, ref, steps, ws)
    assert whole_plan.sync(ws) == 0

    geos = slab.geometries(dims[0], r, depth, world)
    locs, outs, plans, wss = [], [], [], []
    for geo in geos:
        ld = (geo.local_interior,) + tuple(dims[1:])
        p = eb.Plan(ndim, ld, shape, r, c, dtype, eb.DIRICHLET)
        locs.append(slab.scatter(x, geo))
        outs.append(torch.empty_like(locs[-1]))
        plans.append(p)
        wss.append(p.workspace())

    def step(t):
        for i in range(world):
            slab.device_step(plans[i], locs[i], outs[i], wss[i], t)
            locs[i], outs[i] = outs[i], locs[i]

    slab.run_blocks(steps, depth, step, lambda: slab.LocalExchange().exchange(geos, locs))
    for p, w in zip(plans, wss):
        assert p.sync(w) == 0
    got = torch.full_like(x, float("nan"))
    for geo, loc in zip(geos, locs):
        slab.gather_into(got, loc, geo)
    assert torch.equal(got, ref)
