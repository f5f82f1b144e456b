"""GPU parity of the register-streaming temporally blocked kernel (variant 2).

Every 2D stencil, storage type, boundary and both built temporal depths,
against the FP64 oracle (relative L-infinity: FP64 1e-12, FP32 1e-5,
BF16 2e-2) and bit-exact against the naive one-step kernel (same per-cell
FMA order).  The grids span several 128-column strips and several segments,
with ragged last strips and segments, and step counts that leave a partial
last temporal block.
"""
import numpy as np
import pytest

import oracle
from paper_2305_07390_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 2e-2}
STENCILS_2D = [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)]


def _eb():
    from paper_2305_07390_gb300 import ebisu
    return ebisu


def device_problem(eb, dims, shape, r, dtype, boundary, seed):
    g, c = synth.problem(2, dims, shape, r, boundary, seed=seed)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    held = x.double().cpu().numpy()
    c_held = c if dtype == eb.F64 else c.astype(np.float32).astype(np.float64)
    return x, held, c, c_held


def rs_plan(eb, dims, shape, r, c, dtype, boundary, which, tile_s):
    plan = eb.Plan(2, dims, shape, r, c, dtype, boundary)
    d = plan.rs_depths()[which]
    plan.set_params(variant=2, depth=d, tile_s=tile_s, ctas_per_sm=8)
    return plan, d


def run(plan, x, steps, naive=False):
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.run(x, y, steps, ws, naive=naive)
    assert plan.sync(ws) == 0
    return y


def check_pad(y, held, pad):
    m = np.ones(held.shape, bool)
    m[pad:-pad, pad:-pad] = False
    assert np.array_equal(y.double().cpu().numpy()[m], held[m])


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("shape,r", STENCILS_2D)
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("which", [0, 1])
def test_rs_parity(shape, r, dtype, boundary, which):
    eb = _eb()
    dims = (203, 517)
    x, held, c, c_held = device_problem(eb, dims, shape, r, dtype, boundary, seed=300 + 7 * r + shape)
    plan, d = rs_plan(eb, dims, shape, r, c, dtype, boundary, which, tile_s=37)
    p = plan.params()
    assert p.variant == 2 and p.tile_x == 128 - 2 * d * r and p.tile_s == 37
    steps = 2 * d + 1  # a partial last block
    y = run(plan, x, steps)
    yn = run(plan, x, steps, naive=True)
    assert torch.equal(y, yn), "register-streaming and naive kernels differ"
    ref = oracle.run(held, shape, r, c_held, boundary, steps)
    pad = r if boundary == 0 else 0
    assert oracle.rel_linf(y.double().cpu().numpy(), ref, pad) <= TOL[dtype]
    if boundary == 0:
        check_pad(y, held, pad)


@pytest.mark.parametrize("steps", [1, 2, 3, 7, 8, 9, 17])
@pytest.mark.parametrize("dtype", [0, 1])
def test_rs_step_counts(steps, dtype):
    eb = _eb()
    dims = (150, 260)
    x, held, c, c_held = device_problem(eb, dims, 0, 1, dtype, 0, seed=11)
    plan, d = rs_plan(eb, dims, 0, 1, c, dtype, 0, 1, tile_s=40)
    y = run(plan, x, steps)
    assert torch.equal(y, run(plan, x, steps, naive=True))
    ref = oracle.run(held, 0, 1, c_held, 0, steps)
    assert oracle.rel_linf(y.double().cpu().numpy(), ref, 1) <= TOL[dtype]


@pytest.mark.parametrize("dims,tile_s", [((9, 50), 0), ((64, 120), 8), ((300, 140), 300), ((70, 1000), 9)])
@pytest.mark.parametrize("shape,r", [(0, 1), (1, 2)])
def test_rs_shapes(dims, tile_s, shape, r):
    """A strip wider than the grid, segments exactly depth*radius rows, one
    segment over the whole height, many narrow segments."""
    eb = _eb()
    x, held, c, c_held = device_problem(eb, dims, shape, r, eb.F32, 0, seed=12)
    plan = eb.Plan(2, dims, shape, r, c, eb.F32, 0)
    d = plan.rs_depths()[0]
    ts = tile_s if tile_s else 0
    if ts and ts < d * r and ts < dims[0]:
        ts = d * r
    plan.set_params(variant=2, depth=d, tile_s=ts, ctas_per_sm=4)
    steps = d + 2
    y = run(plan, x, steps)
    assert torch.equal(y, run(plan, x, steps, naive=True))
    ref = oracle.run(held, shape, r, c_held, 0, steps)
    assert oracle.rel_linf(y.double().cpu().numpy(), ref, r) <= TOL[1]


@pytest.mark.parametrize("steps", [1, 4, 5, 8, 9])
def test_rs_in_place(steps):
    eb = _eb()
    dims = (96, 300)
    x, held, c, c_held = device_problem(eb, dims, 0, 1, eb.F32, 0, seed=13)
    plan, d = rs_plan(eb, dims, 0, 1, c, eb.F32, 0, 0, tile_s=24)
    ws = plan.workspace()
    y = x.clone()
    plan.run(y, y, steps, ws)
    assert plan.sync(ws) == 0
    ref = oracle.run(held, 0, 1, c_held, 0, steps)
    assert oracle.rel_linf(y.double().cpu().numpy(), ref, 1) <= TOL[1]


def test_rs_wait_timeout_reports_status(monkeypatch):
    eb = _eb()
    monkeypatch.setenv("EBISU_WAIT_TIMEOUT_MS", "200")
    dims = (64, 200)
    x, held, c, _ = device_problem(eb, dims, 0, 1, eb.F64, 0, seed=14)
    plan, d = rs_plan(eb, dims, 0, 1, c, eb.F64, 0, 0, tile_s=32)
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.run_stalled(x, y, 3, ws)
    assert plan.sync(ws) == eb.ERR_TIMEOUT
    # the context stays usable: a normal run afterwards succeeds
    plan.run(x, y, 3, ws)
    assert plan.sync(ws) == 0


def test_rs_tuner_may_pick_it():
    """The tuner times the register-streaming build beside the others; the
    plan then runs whichever won, and the result matches the naive kernel."""
    eb = _eb()
    dims = (1024, 1024)
    x, held, c, _ = device_problem(eb, dims, 0, 1, eb.F32, 0, seed=15)
    plan = eb.Plan(2, dims, 0, 1, c, eb.F32, 0)
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.tune(x, y, 16, ws, max_candidates=4)
    assert plan.params().variant in (0, 1, 2)
    y = run(plan, x, 21)
    assert torch.equal(y, run(plan, x, 21, naive=True))


# ---- 3D register streaming (FP64, depth 1: the 7-point star, the 27-point box)

@pytest.mark.parametrize("shape,r", [(0, 1), (1, 1), (0, 2), (2, 1), (3, 1)])
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("tile_s", [0, 7, 16])
def test_rs3_parity(shape, r, boundary, tile_s):
    eb = _eb()
    # several strips (64 - 2r columns), bands and z segments, ragged tails (a
    # periodic grid's last band must still cover the radius)
    dims = (37, 45, 150) if boundary == 0 else (37, 46, 150)
    g, c = synth.problem(3, dims, shape, r, boundary, seed=400 + shape + 2 * boundary + 5 * r)
    x = torch.from_numpy(g).cuda()
    plan = eb.Plan(3, dims, shape, r, c, eb.F64, boundary)
    assert plan.rs_depths() == (1, 1)
    plan.set_params(variant=2, depth=1, tile_s=tile_s, ctas_per_sm=4)
    p = plan.params()
    assert (p.variant, p.tile_x, p.tile_y) == (2, 64 - 2 * r, 2)
    steps = 5
    y = run(plan, x, steps)
    assert torch.equal(y, run(plan, x, steps, naive=True)), "3D register-streaming and naive kernels differ"
    ref = oracle.run(g, shape, r, c, boundary, steps)
    pad = r if boundary == 0 else 0
    assert oracle.rel_linf(y.cpu().numpy(), ref, pad) <= TOL[0]
    if boundary == 0:
        m = np.ones(g.shape, bool)
        m[r:-r, r:-r, r:-r] = False
        assert np.array_equal(y.cpu().numpy()[m], g[m])


@pytest.mark.parametrize("steps", [1, 2, 6])
def test_rs3_in_place_and_unsupported(steps):
    eb = _eb()
    dims = (20, 24, 80)
    g, c = synth.problem(3, dims, 0, 1, 0, seed=410)
    plan = eb.Plan(3, dims, 0, 1, c, eb.F64, 0)
    plan.set_params(variant=2, depth=1, tile_s=8, ctas_per_sm=4)
    ws = plan.workspace()
    y = torch.from_numpy(g).cuda()
    plan.run(y, y, steps, ws)
    assert plan.sync(ws) == 0
    ref = oracle.run(g, 0, 1, c, 0, steps)
    assert oracle.rel_linf(y.cpu().numpy(), ref, 1) <= TOL[0]
    # no 3D build for the 125-point box, nor for the BF16 13-point star
    p2 = eb.Plan(3, dims, 1, 2, [0.01] * 125, eb.F64, 0)
    assert p2.rs_depths() == (0, 0)
    assert eb.Plan(3, dims, 0, 2, [0.07] * 13, eb.BF16, 0).rs_depths() == (0, 0)
    with pytest.raises(eb.EbisuError):
        p2.set_params(variant=2, depth=1)


def test_rs3_wait_timeout_reports_status(monkeypatch):
    eb = _eb()
    monkeypatch.setenv("EBISU_WAIT_TIMEOUT_MS", "200")
    dims = (16, 16, 70)
    g, c = synth.problem(3, dims, 1, 1, 0, seed=411)
    plan = eb.Plan(3, dims, 1, 1, c, eb.F64, 0)
    plan.set_params(variant=2, depth=1, tile_s=8, ctas_per_sm=4)
    x = torch.from_numpy(g).cuda()
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.run_stalled(x, y, 3, ws)
    assert plan.sync(ws) == eb.ERR_TIMEOUT
    plan.run(x, y, 3, ws)
    assert plan.sync(ws) == 0


# ---- 3D register streaming with temporal blocking (FP32 and BF16 storage:
# the 7-point star at depth 2, 3; the 27-point box at depth 2)

@pytest.mark.parametrize("dtype", [1, 2])
@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("steps", [1, 5, 7])
def test_rs3t_parity(dtype, shape, boundary, which, steps):
    eb = _eb()
    # ragged z segments and strips; a periodic grid's last segment, band and
    # strip must still cover depth * radius cells
    dims = (29, 45, 150) if boundary == 0 else (30, 44, 150)
    g, c = synth.problem(3, dims, shape, 1, boundary, seed=420 + boundary + 3 * which + 7 * shape + 17 * dtype)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    held = x.double().cpu().numpy()
    c_held = c.astype(np.float32).astype(np.float64)
    plan = eb.Plan(3, dims, shape, 1, c, dtype, boundary)
    lo, hi = plan.rs_depths()
    assert (lo, hi) == ((2, 3) if shape == 0 else (2, 2))
    d = (lo, hi)[which]
    plan.set_params(variant=2, depth=d, tile_s=9 if boundary == 0 else 10, ctas_per_sm=4)
    p = plan.params()
    assert (p.variant, p.tile_x, p.tile_y, p.depth) == (2, 64 - 2 * d - (2 if d % 2 == 0 else 0), 4, d)
    y = run(plan, x, steps)
    assert torch.equal(y, run(plan, x, steps, naive=True)), "3D register-streaming and naive kernels differ"
    ref = oracle.run(held, shape, 1, c_held, boundary, steps)
    pad = 1 if boundary == 0 else 0
    assert oracle.rel_linf(y.double().cpu().numpy(), ref, pad) <= TOL[dtype]
    if boundary == 0:
        m = np.ones(held.shape, bool)
        m[1:-1, 1:-1, 1:-1] = False
        assert np.array_equal(y.double().cpu().numpy()[m], held[m])


def test_rs3t_in_place_and_timeout(monkeypatch):
    eb = _eb()
    dims = (20, 24, 90)
    g, c = synth.problem(3, dims, 0, 1, 0, seed=430)
    x = torch.from_numpy(g).to(torch.float32).cuda()
    held = x.double().cpu().numpy()
    plan = eb.Plan(3, dims, 0, 1, c, eb.F32, 0)
    plan.set_params(variant=2, depth=3, tile_s=6, ctas_per_sm=4)
    ws = plan.workspace()
    y = x.clone()
    plan.run(y, y, 4, ws)
    assert plan.sync(ws) == 0
    ref = oracle.run(held, 0, 1, c.astype(np.float32).astype(np.float64), 0, 4)
    assert oracle.rel_linf(y.double().cpu().numpy(), ref, 1) <= TOL[1]
    monkeypatch.setenv("EBISU_WAIT_TIMEOUT_MS", "200")
    plan.run_stalled(x, y, 4, ws)
    assert plan.sync(ws) == eb.ERR_TIMEOUT
    plan.run(x, y, 4, ws)
    assert plan.sync(ws) == 0


@pytest.mark.parametrize("dims,dtype", [((256, 611), 1), ((261, 401), 2), ((64, 96), 0)])
def test_tune_asks_for_more_candidates_than_ranked(dims, dtype):
    """Small grids give the cost model few shared-memory candidates; asking
    the tuner for more must time only real ones and leave a runnable plan."""
    eb = _eb()
    g, c = synth.problem(2, dims, 1, 1, synth.DIRICHLET, seed=17)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    plan = eb.Plan(2, dims, 1, 1, c, dtype, eb.DIRICHLET)
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.tune(x, y, 16, ws, max_candidates=64)
    plan.run(x, y, 9, ws)
    yn = torch.empty_like(x)
    plan.run(x, yn, 9, ws, naive=True)
    assert plan.sync(ws) == 0
    assert torch.equal(y, yn)
