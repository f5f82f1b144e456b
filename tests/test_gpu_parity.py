"""GPU parity: the CUDA path against the CPU oracle, and blocked against naive.

Sizes are small enough for the oracle to finish in seconds but span several
tiles (parameters are forced to small tiles) and ragged tails in every axis.
Tolerances (relative L-infinity over the interior, against the FP64 oracle):
FP64 1e-12, FP32 1e-5, BF16 2e-2.  Blocked vs naive: bit-exact.
For FP32/BF16 the oracle is given the values the device holds: the grid
rounded to the storage type and the coefficients rounded to FP32.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2305_07390_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 2e-2}
STENCILS_2D = [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)]
STENCILS_3D = [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (2, 1), (3, 1)]  # + poisson, j3d17pt


def _eb():
    from paper_2305_07390_gb300 import ebisu
    return ebisu


def device_problem(eb, ndim, dims, shape, r, dtype, boundary, seed):
    g, c = synth.problem(ndim, dims, shape, r, boundary, seed=seed)
    td = eb.torch_dtype(dtype)
    x = torch.from_numpy(g).to(td).cuda()
    held = x.double().cpu().numpy()          # what the device holds
    c_held = c if dtype == eb.F64 else c.astype(np.float32).astype(np.float64)
    return x, held, c, c_held


def run_both(eb, plan, x, steps):
    ws = plan.workspace()
    yb = torch.empty_like(x)
    yn = torch.empty_like(x)
    plan.run(x, yb, steps, ws)
    assert plan.sync(ws) == 0
    plan.run(x, yn, steps, ws, naive=True)
    assert plan.sync(ws) == 0
    return yb, yn


def rel_err(dev, ref, pad):
    return oracle.rel_linf(dev.double().cpu().numpy(), ref, pad)


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("shape,r", STENCILS_2D)
@pytest.mark.parametrize("boundary", [0, 1])
def test_parity_2d(shape, r, dtype, boundary):
    eb = _eb()
    dims = (203, 517)
    x, held, c, c_held = device_problem(eb, 2, dims, shape, r, dtype, boundary, seed=100 + r)
    plan = eb.Plan(2, dims, shape, r, c, dtype, boundary)
    plan.set_params(tile_x=128, tile_s=57, depth=3)
    steps = 7
    yb, yn = run_both(eb, plan, x, steps)
    assert torch.equal(yb, yn), "blocked and naive kernels differ"
    ref = oracle.run(held, shape, r, c_held, boundary, steps)
    pad = r if boundary == 0 else 0
    assert rel_err(yb, ref, pad) <= TOL[dtype]
    if boundary == 0:  # Dirichlet pad untouched
        m = np.ones(held.shape, bool)
        m[pad:-pad, pad:-pad] = False
        assert np.array_equal(yb.double().cpu().numpy()[m], held[m])


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("shape,r", STENCILS_3D)
@pytest.mark.parametrize("boundary", [0, 1])
def test_parity_3d(shape, r, dtype, boundary):
    eb = _eb()
    dims = (23, 37, 45)
    x, held, c, c_held = device_problem(eb, 3, dims, shape, r, dtype, boundary, seed=200 + r)
    plan = eb.Plan(3, dims, shape, r, c, dtype, boundary)
    plan.set_params(tile_x=16, tile_y=12, tile_s=9, depth=2)
    steps = 5
    yb, yn = run_both(eb, plan, x, steps)
    assert torch.equal(yb, yn), "blocked and naive kernels differ"
    ref = oracle.run(held, shape, r, c_held, boundary, steps)
    pad = r if boundary == 0 else 0
    assert rel_err(yb, ref, pad) <= TOL[dtype]


@pytest.mark.parametrize("depth,steps", [(1, 1), (4, 3), (3, 10), (5, 5), (16, 17), (2, 2)])
def test_depth_and_step_counts(depth, steps):
    eb = _eb()
    dims = (150, 260)
    x, held, c, _ = device_problem(eb, 2, dims, 1, 2, eb.F64, 0, seed=7)
    plan = eb.Plan(2, dims, 1, 2, c, eb.F64, 0)
    plan.set_params(tile_x=100, tile_s=40, depth=depth)
    yb, yn = run_both(eb, plan, x, steps)
    assert torch.equal(yb, yn)
    ref = oracle.run(held, 1, 2, c, 0, steps)
    assert rel_err(yb, ref, 2) <= 1e-12


@pytest.mark.parametrize("steps", [1, 2, 3, 4])
@pytest.mark.parametrize("naive", [False, True])
def test_in_place(steps, naive):
    eb = _eb()
    dims = (64, 96)
    x, held, c, _ = device_problem(eb, 2, dims, 0, 1, eb.F64, 0, seed=8)
    plan = eb.Plan(2, dims, 0, 1, c, eb.F64, 0)
    plan.set_params(tile_x=40, tile_s=20, depth=2)
    ws = plan.workspace()
    y = x.clone()
    plan.run(y, y, steps, ws, naive=naive)
    assert plan.sync(ws) == 0
    ref = oracle.run(held, 0, 1, c, 0, steps)
    assert rel_err(y, ref, 1) <= 1e-12


def test_zero_steps_copies():
    eb = _eb()
    x, held, c, _ = device_problem(eb, 2, (30, 40), 0, 1, eb.F64, 0, seed=9)
    plan = eb.Plan(2, (30, 40), 0, 1, c, eb.F64, 0)
    ws = plan.workspace()
    y = torch.zeros_like(x)
    plan.run(x, y, 0, ws)
    assert plan.sync(ws) == 0
    assert torch.equal(x, y)


def test_run_composes():
    # run(a + b) == run(b) after run(a), bit for bit (resume from a state)
    eb = _eb()
    dims = (120, 333)
    x, _, c, _ = device_problem(eb, 2, dims, 1, 1, eb.F64, 0, seed=10)
    plan = eb.Plan(2, dims, 1, 1, c, eb.F64, 0)
    plan.set_params(tile_x=64, tile_s=30, depth=4)
    ws = plan.workspace()
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    plan.run(x, y1, 11, ws)
    plan.run(x, y2, 5, ws)
    y3 = torch.empty_like(x)
    plan.run(y2, y3, 6, ws)
    assert plan.sync(ws) == 0
    assert torch.equal(y1, y3)


def test_reductions_match_oracle():
    eb = _eb()
    dims = (301, 257)
    x, held, c, _ = device_problem(eb, 2, dims, 1, 2, eb.F64, 0, seed=11)
    plan = eb.Plan(2, dims, 1, 2, c, eb.F64, 0)
    ws = plan.workspace()
    s, l2, mx = plan.reduce(x, ws)
    rs, rl2, rmx = oracle.reduce(held, 2)
    assert abs(s - rs) <= 1e-12 * abs(rs)
    assert abs(l2 - rl2) <= 1e-12 * rl2
    assert mx == rmx
    y = torch.empty_like(x)
    plan.run(x, y, 3, ws)
    assert plan.sync(ws) == 0
    _, _, dmx = plan.reduce(y, ws, x)
    _, _, rdmx = oracle.reduce(y.cpu().numpy(), 2, held)
    assert dmx == rdmx


def test_periodic_fourier_mode_decay_gpu():
    # closed form on the device path too: lambda(k)^T decay of a cosine mode
    eb = _eb()
    dims = (16, 20, 24)
    k = (2, 1, 3)
    c = synth.coefficients(3, 0, 1, dims, 1, seed=12)
    u0 = synth.cosine_mode(dims, k)
    x = torch.from_numpy(u0).cuda()
    plan = eb.Plan(3, dims, 0, 1, c, eb.F64, eb.PERIODIC)
    plan.set_params(tile_x=8, tile_y=8, tile_s=5, depth=3)
    ws = plan.workspace()
    y = torch.empty_like(x)
    T = 9
    plan.run(x, y, T, ws)
    assert plan.sync(ws) == 0
    offs = oracle.offsets(3, 0, 1)
    lam = sum(ck * np.exp(2j * np.pi * sum(kd * od / nd for kd, od, nd in zip(k, o, dims)))
              for o, ck in zip(offs, c))
    mesh = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims], indexing="ij")
    phase = sum(2 * np.pi * kd * xd / nd for kd, xd, nd in zip(k, mesh, dims))
    ref = np.real(lam ** T * np.exp(1j * phase))
    assert np.max(np.abs(y.cpu().numpy() - ref)) < 1e-12


def test_wait_timeout_reports_status(monkeypatch):
    # A dependency wait that nothing satisfies must give up within its bound
    # and report EBISU_ERR_TIMEOUT; the context stays usable afterwards.
    eb = _eb()
    monkeypatch.setenv("EBISU_WAIT_TIMEOUT_MS", "300")
    dims = (64, 64)
    x, held, c, _ = device_problem(eb, 2, dims, 0, 1, eb.F64, 0, seed=13)
    plan = eb.Plan(2, dims, 0, 1, c, eb.F64, 0)
    plan.set_params(tile_x=32, tile_s=32, depth=1)
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.run_stalled(x, y, 4, ws)
    assert plan.sync(ws) == eb.ERR_TIMEOUT
    plan.run(x, y, 4, ws)
    assert plan.sync(ws) == 0
    ref = oracle.run(held, 0, 1, c, 0, 4)
    assert rel_err(y, ref, 1) <= 1e-12


def test_config1_small_exact_case():
    # 2D 5-point star, c_centre = 0.5, c_NSEW = 0.125, 512^2 + Dirichlet pad, 8 steps
    eb = _eb()
    dims = (512, 512)
    g = synth.grid(dims, 1, 0)
    c = synth.config1_coefficients()
    x = torch.from_numpy(g).cuda()
    plan = eb.Plan(2, dims, 0, 1, c, eb.F64, 0)
    yb, yn = run_both(eb, plan, x, 8)
    assert torch.equal(yb, yn)
    ref = oracle.run(g, 0, 1, c, 0, 8)
    assert rel_err(yb, ref, 1) <= 1e-12


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("boundary", [0, 1])
def test_offset_list_plans(ndim, dtype, boundary):
    """Plans from explicit offset lists: an asymmetric subset of the
    radius-2 box runs on the box kernels with zero weights elsewhere; the
    oracle steps the list itself."""
    eb = _eb()
    import itertools
    rng = np.random.default_rng(50 + ndim)
    rr = range(-2, 3)
    full = [(0, a, b) for a, b in itertools.product(rr, rr)] if ndim == 2 else list(itertools.product(rr, rr, rr))
    pick = [full[i] for i in sorted(rng.choice(len(full), 11, replace=False))]
    pick = sorted(set(pick) | {(0, 0, 2)})  # radius 2 reached along x
    c = rng.random(len(pick))
    c /= c.sum()
    dims = (90, 150) if ndim == 2 else (24, 30, 40)
    g = synth.grid(dims, 2, boundary, seed=51)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    held = x.double().cpu().numpy()
    c_held = c if dtype == 0 else c.astype(np.float32).astype(np.float64)
    order = rng.permutation(len(pick))  # the list's order does not matter
    plan = eb.Plan.from_offsets(ndim, dims, [pick[i] for i in order], c[order], dtype, boundary)
    yb, yn = run_both(eb, plan, x, 6)
    assert torch.equal(yb, yn)
    ref = oracle.run_offsets(held, pick, 2, c_held, boundary, 6)
    assert rel_err(yb, ref, 2 if boundary == 0 else 0) <= TOL[dtype]


def test_offset_list_matching_a_named_shape_gets_its_kernels():
    eb = _eb()
    offs = [tuple(o) for o in oracle.offsets(3, 2, 1)]  # poisson
    c = np.full(len(offs), 1.0 / len(offs))
    plan = eb.Plan.from_offsets(3, (20, 22, 70), offs, c)
    assert plan.rs_depths() == (1, 1)  # the FP64 3D register-streaming build exists for it
    n = ctypes_npoints(eb, plan)
    assert n == 19


def ctypes_npoints(eb, plan):
    import ctypes
    v = ctypes.c_int()
    assert eb.lib().ebisu_plan_npoints(plan.h, ctypes.byref(v)) == 0
    return v.value


@pytest.mark.parametrize("mask", [15, 7, 6, 4, 0])
@pytest.mark.parametrize("ndim,dtype", [(2, 1), (2, 0), (3, 1), (3, 0)])
def test_ablation_builds_equal_naive(ndim, dtype, mask):
    """The breakdown builds (queues shifted instead of circular, no prefetch,
    a barrier per level, no register reuse) change the schedule, never the
    arithmetic: every one equals the one-step kernel bit for bit."""
    eb = _eb()
    dims = (203, 517) if ndim == 2 else (23, 37, 45)
    x, held, c, c_held = device_problem(eb, ndim, dims, 0, 1, dtype, 0, seed=60 + mask)
    plan = eb.Plan(ndim, dims, 0, 1, c, dtype, 0)
    if ndim == 2:
        plan.set_params(tile_x=128, tile_s=57, depth=1 if mask == 15 else 4)
    else:
        plan.set_params(tile_x=16, tile_y=12, tile_s=9, depth=1 if mask == 15 else 3)
    plan.set_ablation(mask)
    yb, yn = run_both(eb, plan, x, 9)
    assert torch.equal(yb, yn), f"ablation mask {mask} differs"
    ref = oracle.run(held, 0, 1, c_held, 0, 9)
    assert rel_err(yb, ref, 1) <= TOL[dtype]
