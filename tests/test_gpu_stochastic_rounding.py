"""Stochastic rounding of BF16 storage (ebisu_plan_set_rounding).

The rounding itself is pinned by what defines it rather than by another
implementation: every result is one of the two BF16 neighbours of the FP32
value, it rounds up with probability equal to the discarded fraction of an
ulp (so the mean over many cells is the FP32 value), the random bits depend
on the seed, and they are a function of (seed, step, cell) only -- so a run
is reproducible and the blocked, naive and batched kernels agree bit for bit
(covered at scale in test_gpu_precision.py).
"""
import numpy as np
import pytest

from paper_2305_07390_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _eb():
    from paper_2305_07390_gb300 import ebisu
    return ebisu


def _bf16_neighbours(v):
    """The BF16 values just below and above the FP32 value v (> 0)."""
    b = np.array([v], dtype=np.float32).view(np.uint32)[0]
    lo = np.array([b & 0xFFFF0000], dtype=np.uint32).view(np.float32)[0]
    hi = np.array([(b & 0xFFFF0000) + 0x10000], dtype=np.uint32).view(np.float32)[0]
    return float(lo), float(hi)


@pytest.mark.parametrize("naive", [False, True])
def test_one_step_rounds_up_with_the_discarded_fraction(naive):
    eb = _eb()
    dims = (512, 1024)
    # every cell 1.0; a 5-point star whose weights sum to w (FP32), so the
    # FP32 result of one step is the same value x = w in every cell
    c = np.array([0.1, 0.2, 0.3001, 0.15, 0.2], dtype=np.float64)
    x32 = np.float32(0.0)
    for k, ck in enumerate(c.astype(np.float32)):  # the kernel's FMA chain on ones
        x32 = np.float32(ck) if k == 0 else np.float32(np.float64(ck) + np.float64(x32))
    lo, hi = _bf16_neighbours(float(x32))
    assert lo < float(x32) < hi
    frac = (float(x32) - lo) / (hi - lo)
    plan = eb.Plan(2, dims, eb.STAR, 1, c, eb.BF16, eb.DIRICHLET)
    plan.set_rounding(eb.ROUND_STOCHASTIC, seed=7)
    x = torch.ones((dims[0] + 2, dims[1] + 2), dtype=torch.bfloat16, device="cuda")
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.run(x, y, 1, ws, naive=naive)
    assert plan.sync(ws) == 0
    v = y[1:-1, 1:-1].float().cpu().numpy().ravel()
    assert set(np.unique(v)) <= {lo, hi}
    up = float(np.mean(v == hi))
    n = v.size
    assert abs(up - frac) < 5 * np.sqrt(frac * (1 - frac) / n) + 1e-9, (up, frac)
    # round to nearest gives one value everywhere
    plan.set_rounding(eb.ROUND_NEAREST)
    yr = torch.empty_like(x)
    plan.run(x, yr, 1, ws, naive=naive)
    assert plan.sync(ws) == 0
    assert torch.unique(yr[1:-1, 1:-1]).numel() == 1


def test_seed_and_reproducibility():
    eb = _eb()
    dims = (300, 700)
    g, c = synth.problem(2, dims, synth.STAR, 1, synth.DIRICHLET, seed=5)
    x = torch.from_numpy(g).to(torch.bfloat16).cuda()
    outs = []
    for seed in (1, 1, 2):
        plan = eb.Plan(2, dims, eb.STAR, 1, c, eb.BF16, eb.DIRICHLET)
        plan.set_rounding(eb.ROUND_STOCHASTIC, seed=seed)
        assert plan.rounding() == (eb.ROUND_STOCHASTIC, seed)
        ws = plan.workspace()
        y = torch.empty_like(x)
        plan.run(x, y, 20, ws)
        assert plan.sync(ws) == 0
        outs.append(y)
    assert torch.equal(outs[0], outs[1])
    assert not torch.equal(outs[0], outs[2])


@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("shape,r", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)])
def test_2d_blocked_equals_naive(shape, r, boundary):
    eb = _eb()
    dims = (203, 517) if boundary == 0 else (200, 520)
    g, c = synth.problem(2, dims, shape, r, boundary, seed=100 + r)
    x = torch.from_numpy(g).to(torch.bfloat16).cuda()
    plan = eb.Plan(2, dims, shape, r, c, eb.BF16, boundary)
    plan.set_rounding(eb.ROUND_STOCHASTIC, seed=3)
    ws = plan.workspace()
    yn = torch.empty_like(x)
    plan.run(x, yn, 13, ws, naive=True)
    assert plan.sync(ws) == 0
    for depth in sorted(set(plan.rs_depths())):
        plan.set_params(variant=2, depth=depth, tile_s=40, ctas_per_sm=4)
        y = torch.empty_like(x)
        plan.run(x, y, 13, ws)
        assert plan.sync(ws) == 0
        assert torch.equal(y, yn), f"depth {depth}"


@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("shape", [0, 1])
def test_3d_blocked_equals_naive(shape, boundary):
    eb = _eb()
    dims = (23, 37, 90) if boundary == 0 else (24, 36, 96)
    g, c = synth.problem(3, dims, shape, 1, boundary, seed=200 + shape)
    x = torch.from_numpy(g).to(torch.bfloat16).cuda()
    plan = eb.Plan(3, dims, shape, 1, c, eb.BF16, boundary)
    plan.set_rounding(eb.ROUND_STOCHASTIC, seed=4)
    ws = plan.workspace()
    yn = torch.empty_like(x)
    plan.run(x, yn, 7, ws, naive=True)
    assert plan.sync(ws) == 0
    for depth in sorted(set(plan.rs_depths())):
        plan.set_params(variant=2, depth=depth, tile_s=8, ctas_per_sm=4)
        y = torch.empty_like(x)
        plan.run(x, y, 7, ws)
        assert plan.sync(ws) == 0
        assert torch.equal(y, yn), f"depth {depth}"
