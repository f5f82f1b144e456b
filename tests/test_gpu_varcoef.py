"""Variable coefficients (per-cell weights, ebisu_plan_set_coefficient_field)
on the GPU against the oracle's plain loops (oracle.run_varcoef)."""
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


def _field(eb, npts, stored, dtype, seed):
    rng = np.random.default_rng(seed)
    w = rng.random((npts,) + stored)
    w /= w.sum(axis=0, keepdims=True)  # each cell's weights sum to one
    td = torch.float64 if dtype == eb.F64 else torch.float32
    f = torch.from_numpy(w).to(td).cuda()
    return f, f.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("ndim,dims,shape,r", [(2, (150, 260), 0, 2), (2, (97, 133), 1, 1), (3, (20, 24, 30), 0, 1),
                                               (3, (18, 20, 22), 2, 1)])
@pytest.mark.parametrize("boundary", [0, 1])
def test_varcoef_matches_oracle(ndim, dims, shape, r, dtype, boundary):
    eb = _eb()
    g, c = synth.problem(ndim, dims, shape, r, boundary, seed=91)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    held = x.double().cpu().numpy()
    plan = eb.Plan(ndim, dims, shape, r, c, dtype, boundary)
    f, f_held = _field(eb, len(c), plan.stored_shape, dtype, seed=92)
    plan.set_coefficient_field(f)
    ws = plan.workspace()
    steps = 6
    y = torch.empty_like(x)
    plan.run(x, y, steps, ws)
    assert plan.sync(ws) == 0
    ref = oracle.run_varcoef(held, shape, r, f_held, boundary, steps)
    pad = r if boundary == 0 else 0
    assert oracle.rel_linf(y.double().cpu().numpy(), ref, pad) <= TOL[dtype]
    # in place, and the naive entry point, give the same bits
    y2 = x.clone()
    plan.run(y2, y2, steps, ws)
    yn = torch.empty_like(x)
    plan.run(x, yn, steps, ws, naive=True)
    assert plan.sync(ws) == 0
    assert torch.equal(y2, y) and torch.equal(yn, y)


def test_uniform_field_equals_fixed_weights_and_refusals():
    eb = _eb()
    dims = (120, 200)
    g, c = synth.problem(2, dims, 1, 1, 0, seed=93)
    x = torch.from_numpy(g).cuda()
    plan = eb.Plan(2, dims, 1, 1, c, eb.F64, 0)
    ws = plan.workspace()
    ref = torch.empty_like(x)
    plan.run(x, ref, 9, ws, naive=True)
    f = torch.from_numpy(np.broadcast_to(c[:, None, None], (9,) + plan.stored_shape).copy()).cuda()
    plan.set_coefficient_field(f)
    y = torch.empty_like(x)
    plan.run(x, y, 9, ws)
    assert plan.sync(ws) == 0
    assert torch.equal(y, ref)  # the same FMA chain with the same weights
    with pytest.raises(eb.EbisuError):
        plan.tune(x, torch.empty_like(x), 4, ws)
    wsb = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(eb.EbisuError):
        eb.batch_run([plan], [x], [torch.empty_like(x)], [3], wsb)
    plan.set_coefficient_field(None)
    plan.run(x, y, 9, ws)
    assert plan.sync(ws) == 0
    assert torch.equal(y, ref)
