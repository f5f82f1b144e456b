"""Degenerate stencils and degenerate grids on the GPU path.

* The identity stencil (weight 1 on the centre, 0 on every other point of
  the star or box) leaves a grid unchanged, and a stencil whose only weight
  is 1 on the +x neighbour shifts a periodic grid by one cell per step:
  after T steps the grid is rolled by T cells along x.  Both results are
  exact in every storage type (the FMA chain multiplies by 1 and 0 and adds
  zeros), so every kernel -- one-step, shared-memory queues, register
  streaming -- must reproduce them bit for bit, including the last,
  partial temporal block.
* Grids smaller than a tile, than the radius or than the temporal halo (a
  1 x 1 interior, a single row, a periodic grid of 2r + 1 cells per axis)
  run through the plan's default kernel and the one-step kernel, which
  must agree bit for bit and match the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2305_07390_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 2e-2}


def _eb():
    from paper_2305_07390_gb300 import ebisu
    return ebisu


def one_hot(ndim, shape, r, offset):
    """Weights 1 on `offset` (dz, dy, dx) and 0 elsewhere, in the canonical
    order of the stencil's offsets."""
    offs = [tuple(int(v) for v in o) for o in oracle.offsets(ndim, shape, r)]
    c = np.zeros(len(offs))
    c[offs.index(offset)] = 1.0
    return c


def variants(plan, ndim):
    """(name, run kwargs, params) of the kernels a plan of this kind can
    run: the one-step kernel, the shared-memory build (several tiles, a
    partial last block), and the register-streaming build at each of its
    depths (one segment per strip)."""
    tb = (dict(variant=0, tile_x=64, tile_s=32, depth=3, ctas_per_sm=2) if ndim == 2 else
          dict(variant=0, tile_x=32, tile_y=8, tile_s=16, depth=2, ctas_per_sm=2))
    out = [("naive", {"naive": True}, None), ("shared", {}, tb)]
    lo, hi = plan.rs_depths()
    for d in sorted({lo, hi} - {0}):
        out.append((f"rs{d}", {}, dict(variant=2, depth=d, tile_s=0, ctas_per_sm=4)))
    return out


def run_kernel(eb, plan, x, steps, kw, params):
    if params is not None:
        plan.set_params(**params)
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.run(x, y, steps, ws, **kw)
    assert plan.sync(ws) == 0
    return y


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("ndim,dims,shape,r", [(2, (70, 140), 0, 1), (2, (70, 140), 0, 2),
                                               (2, (70, 140), 1, 1), (3, (20, 24, 80), 0, 1),
                                               (3, (20, 24, 80), 1, 1)])
@pytest.mark.parametrize("boundary", [0, 1])
def test_identity_stencil_keeps_the_grid(dtype, ndim, dims, shape, r, boundary):
    eb = _eb()
    g, _ = synth.problem(ndim, dims, shape, r, boundary, seed=500 + 7 * r + shape)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    c = one_hot(ndim, shape, r, (0, 0, 0))
    plan = eb.Plan(ndim, dims, shape, r, c, dtype, boundary)
    for name, kw, params in variants(plan, ndim):
        y = run_kernel(eb, plan, x, 13, kw, params)
        assert torch.equal(y, x), f"{name}: the identity stencil changed the grid"


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("ndim,dims,shape,r", [(2, (70, 140), 0, 1), (2, (66, 150), 0, 3),
                                               (2, (70, 140), 1, 2), (3, (20, 24, 80), 0, 1),
                                               (3, (18, 20, 76), 1, 1)])
def test_shift_stencil_rolls_a_periodic_grid(dtype, ndim, dims, shape, r):
    eb = _eb()
    g, _ = synth.problem(ndim, dims, shape, r, synth.PERIODIC, seed=520 + 7 * r + shape)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    c = one_hot(ndim, shape, r, (0, 0, 1))  # u_new(x) = u(x + 1)
    plan = eb.Plan(ndim, dims, shape, r, c, dtype, synth.PERIODIC)
    steps = 13
    want = torch.roll(x, shifts=-steps, dims=ndim - 1)
    for name, kw, params in variants(plan, ndim):
        y = run_kernel(eb, plan, x, steps, kw, params)
        assert torch.equal(y, want), f"{name}: not the grid rolled by {steps} cells"


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("ndim,dims,shape,r,boundary", [
    (2, (1, 1), 0, 1, 0), (2, (1, 7), 0, 3, 0), (2, (3, 2), 1, 2, 0), (2, (1, 300), 1, 1, 0),
    (2, (3, 3), 0, 1, 1), (2, (7, 7), 0, 3, 1), (2, (5, 9), 1, 2, 1),
    (3, (1, 1, 1), 0, 1, 0), (3, (2, 3, 1), 1, 1, 0), (3, (3, 3, 3), 0, 1, 1), (3, (5, 5, 5), 0, 2, 1)])
def test_tiny_grids(dtype, ndim, dims, shape, r, boundary):
    eb = _eb()
    g, c = synth.problem(ndim, dims, shape, r, boundary, seed=540 + r + 3 * shape + 11 * boundary)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    held = x.double().cpu().numpy()
    ch = c if dtype == 0 else c.astype(np.float32).astype(np.float64)
    plan = eb.Plan(ndim, dims, shape, r, c, dtype, boundary)
    steps = 11
    y = run_kernel(eb, plan, x, steps, {}, None)
    yn = run_kernel(eb, plan, x, steps, {"naive": True}, None)
    assert torch.equal(y, yn), "default kernel and one-step kernel differ"
    ref = oracle.run(held, shape, r, ch, boundary, steps)
    pad = r if boundary == 0 else 0
    assert oracle.rel_linf(y.double().cpu().numpy(), ref, pad) <= TOL[dtype]
