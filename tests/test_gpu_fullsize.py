"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times.

* 2D FP64 set on 8192 x 8192, 1000 steps: the parameters are chosen exactly
  as bench.py chooses them (cost-model ranking + short timed tuning), then the
  whole run is checked on sampled outputs the oracle can compute: corner
  windows whose dependency cone (r cells per step) is cut out of the grid and
  stepped by the oracle.  Cells farther than r*T from the cut's artificial
  edge are exact functions of the cut, so the comparison is exact up to
  rounding (relative L-inf 1e-12).
* 3D FP64 set on 512^3, 200 steps: Dirichlet corner windows for the radius-1
  stencils, and for every stencil a periodic run started from a cosine mode,
  checked against the closed form lambda(k)^T (Fourier-mode decay).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2305_07390_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-12


def _eb():
    from paper_2305_07390_gb300 import ebisu
    return ebisu


def tuned_run(eb, ndim, dims, shape, r, c, g, steps, boundary=0, tune=8):
    plan = eb.Plan(ndim, dims, shape, r, c, eb.F64, boundary)
    x = torch.from_numpy(g).cuda()
    y = torch.empty_like(x)
    ws = plan.workspace()
    plan.tune(x, y, min(steps, 16), ws, max_candidates=tune)  # as bench.py does
    plan.run(x, y, steps, ws)
    assert plan.sync(ws) == 0
    return plan, y


def corner_check(g, out, shape, r, c, steps, w, high):
    """Oracle on the cone of a w^d corner window; returns rel L-inf error."""
    nd = g.ndim
    span = w + 2 * r + steps * r
    if high:
        sl = tuple(slice(s - span, s) for s in g.shape)
    else:
        sl = tuple(slice(0, span) for _ in g.shape)
    cut = np.ascontiguousarray(g[sl])
    ref = oracle.run(cut, shape, r, c, synth.DIRICHLET, steps)
    if high:
        win = tuple(slice(span - r - w, span - r) for _ in range(nd))
    else:
        win = tuple(slice(r, r + w) for _ in range(nd))
    dev = out[sl][win]
    ref_w = ref[win]
    return float(np.max(np.abs(dev - ref_w)) / np.max(np.abs(ref_w)))


@pytest.mark.parametrize("shape,r", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)])
def test_2d_fullsize_corners(shape, r):
    eb = _eb()
    dims = (8192, 8192)
    steps = 1000
    g, c = synth.problem(2, dims, shape, r, synth.DIRICHLET, seed=synth.DEFAULT_SEED + 17 * r + shape)
    plan, y = tuned_run(eb, 2, dims, shape, r, c, g, steps)
    out = y.cpu().numpy()
    w = 6
    assert corner_check(g, out, shape, r, c, steps, w, high=False) <= TOL
    if r == 1:
        assert corner_check(g, out, shape, r, c, steps, w, high=True) <= TOL
    # the pad is untouched
    assert np.array_equal(out[:r], g[:r]) and np.array_equal(out[:, -r:], g[:, -r:])


@pytest.mark.parametrize("shape,r", [(0, 1), (1, 1)])
def test_3d_fullsize_dirichlet_corners(shape, r):
    eb = _eb()
    dims = (512, 512, 512)
    steps = 200
    g, c = synth.problem(3, dims, shape, r, synth.DIRICHLET, seed=synth.DEFAULT_SEED + 31 * r + shape)
    plan, y = tuned_run(eb, 3, dims, shape, r, c, g, steps, tune=4)
    out = y.cpu().numpy()
    assert corner_check(g, out, shape, r, c, steps, 4, high=False) <= TOL
    assert corner_check(g, out, shape, r, c, steps, 4, high=True) <= TOL


@pytest.mark.parametrize("shape,r", [(0, 1), (0, 2), (1, 1), (1, 2)])
@pytest.mark.parametrize("k", [(1, 1, 1), (2, 1, 3)])
def test_3d_fullsize_periodic_fourier(shape, r, k):
    eb = _eb()
    dims = (512, 512, 512)
    steps = 200
    c = synth.coefficients(3, shape, r, dims, synth.PERIODIC, seed=synth.DEFAULT_SEED + 7)
    u0 = synth.cosine_mode(dims, k)
    plan, y = tuned_run(eb, 3, dims, shape, r, c, u0, steps, boundary=eb.PERIODIC, tune=3)
    offs = oracle.offsets(3, shape, r)
    lam = sum(ck * np.exp(2j * math.pi * sum(kd * od / nd for kd, od, nd in zip(k, o, dims)))
              for o, ck in zip(offs, c))
    assert abs(lam) ** steps > 1e-3
    # compare on the device in slabs (the 512^3 reference is 1 GB)
    lamT = lam ** steps
    err = 0.0
    xs = torch.arange(512, dtype=torch.float64, device="cuda")
    for z0 in range(0, 512, 64):
        zz, yy, xx = torch.meshgrid(xs[z0:z0 + 64], xs, xs, indexing="ij")
        ph = 2 * math.pi * (k[0] * zz / 512 + k[1] * yy / 512 + k[2] * xx / 512)
        ref = lamT.real * torch.cos(ph) - lamT.imag * torch.sin(ph)
        err = max(err, float(torch.max(torch.abs(y[z0:z0 + 64] - ref))))
    assert err / abs(lamT) <= TOL  # relative L-inf against the mode's amplitude


def bench_tuned_plan(eb, ndim, dims, shape, r, c, x, dtype, tune_steps, candidates):
    """A plan tuned the way bench.py tunes it (cost-model ranking plus a short
    timed run of the best candidates), forced to the fused build it found."""
    plan = eb.Plan(ndim, dims, shape, r, c, dtype, eb.DIRICHLET)
    ws = plan.workspace()
    plan.tune(x, torch.empty_like(x), tune_steps, ws, max_candidates=candidates)
    if plan.params().variant == 1:
        plan.set_params(variant=plan.params().fused_variant)
    return plan, ws


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("shape,r", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)])
def test_2d_fullsize_blocked_equals_naive(shape, r, dtype):
    """The whole 8192^2 grid after 1000 steps, in the benchmark's launch
    configuration, equals the one-step-per-launch kernel bit for bit
    (Section 4.1: tiling reorders the updates without changing them); for
    FP32 storage, the oracle's corner windows of the same run (the values
    the device holds, FP32-rounded coefficients) within 1e-5."""
    eb = _eb()
    dims, steps = (8192, 8192), 1000
    g, c = synth.problem(2, dims, shape, r, synth.DIRICHLET, seed=synth.DEFAULT_SEED + 17 * r + shape)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    plan, ws = bench_tuned_plan(eb, 2, dims, shape, r, c, x, dtype, 48, 16)
    y = torch.empty_like(x)
    plan.run(x, y, steps, ws)
    assert plan.sync(ws) == 0
    yn = torch.empty_like(x)
    plan.run(x, yn, steps, ws, naive=True)
    assert plan.sync(ws) == 0
    assert torch.equal(y, yn), f"params {plan.params().as_dict()}"
    if dtype == eb.F32:
        held = x.double().cpu().numpy()
        c_held = c.astype(np.float32).astype(np.float64)
        out = y.double().cpu().numpy()
        assert corner_check(held, out, shape, r, c_held, steps, 6, high=False) <= 1e-5
        assert corner_check(held, out, shape, r, c_held, steps, 6, high=True) <= 1e-5


@pytest.mark.parametrize("shape,r", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_3d_fullsize_blocked_equals_naive(shape, r):
    """The whole 512^3 FP64 grid after 200 steps, in the benchmark's tuned
    launch configuration, equals the one-step-per-launch kernel bit for bit."""
    eb = _eb()
    dims, steps = (512, 512, 512), 200
    g, c = synth.problem(3, dims, shape, r, synth.DIRICHLET, seed=synth.DEFAULT_SEED + 31 * r + shape)
    x = torch.from_numpy(g).cuda()
    del g
    plan, ws = bench_tuned_plan(eb, 3, dims, shape, r, c, x, eb.F64, 8, 4)
    y = torch.empty_like(x)
    plan.run(x, y, steps, ws)
    assert plan.sync(ws) == 0
    yn = torch.empty_like(x)
    plan.run(x, yn, steps, ws, naive=True)
    assert plan.sync(ws) == 0
    assert torch.equal(y, yn), f"params {plan.params().as_dict()}"


# ---- grids of more than 2^31 stored cells -----------------------------------
# Every element offset past 2^31 needs 64-bit index arithmetic.  The grid is
# generated row block by row block from the seeded stream (counter-based, so
# any row range can be drawn on its own) straight into device memory; the
# oracle's corner cones are drawn the same way.

def _rows(dims_stored, seed, r0, r1):
    """Stored rows (first axis) r0 .. r1-1 of the seeded grid, FP64."""
    inner = int(np.prod(dims_stored[1:]))
    v = synth.uniform01(seed, r0 * inner, (r1 - r0) * inner)
    return v.reshape((r1 - r0,) + tuple(dims_stored[1:]))


@pytest.mark.parametrize("ndim,dims,rs", [
    (2, (46341, 46341), dict(variant=2, depth=8, tile_s=2048, ctas_per_sm=3)),
    (3, (1292, 1292, 1292), dict(variant=2, depth=3, tile_s=0, ctas_per_sm=2))])
def test_more_than_2_to_31_cells(ndim, dims, rs):
    eb = _eb()
    r, shape, steps, seed = 1, 0, 3, 97
    st = synth.stored_shape(dims, r, synth.DIRICHLET)
    assert int(np.prod(st)) > 2 ** 31
    c = synth.coefficients(ndim, shape, r, dims, synth.DIRICHLET, seed)
    x = torch.empty(st, dtype=torch.float32, device="cuda")
    blk = 1024 if ndim == 2 else 64
    for a in range(0, st[0], blk):
        b = min(st[0], a + blk)
        x[a:b] = torch.from_numpy(_rows(st, seed, a, b)).float().cuda()
    plan = eb.Plan(ndim, dims, shape, r, c, eb.F32, eb.DIRICHLET)
    ws = plan.workspace()
    out = {}
    tb = (dict(variant=0, tile_x=64, tile_s=32, depth=3, ctas_per_sm=2) if ndim == 2 else
          dict(variant=0, tile_x=32, tile_y=8, tile_s=16, depth=2, ctas_per_sm=2))
    for name, params, kw in [("naive", None, {"naive": True}), ("shared", tb, {}), ("rs", rs, {})]:
        if params is not None:
            plan.set_params(**params)
        y = torch.empty_like(x)
        plan.run(x, y, steps, ws, **kw)
        assert plan.sync(ws) == 0, name
        out[name] = y
        if name != "naive":
            assert torch.equal(y, out["naive"]), f"{name} differs from the one-step kernel"
            del out[name], y
    y = out["naive"]
    # oracle cones of the first and the last corner window (the last one's
    # offsets lie past 2^31)
    w = 6
    span = w + 2 * r + steps * r
    ch = c.astype(np.float32).astype(np.float64)
    for high in (False, True):
        r0 = st[0] - span if high else 0
        cut_rows = _rows(st, seed, r0, r0 + span).astype(np.float32).astype(np.float64)
        sl = tuple(slice(s - span, s) if high else slice(0, span) for s in st[1:])
        cut = np.ascontiguousarray(cut_rows[(slice(None),) + sl])
        ref = oracle.run(cut, shape, r, ch, synth.DIRICHLET, steps)
        win = tuple(slice(span - r - w, span - r) if high else slice(r, r + w) for _ in range(ndim))
        dev = y[(slice(r0, r0 + span),) + sl].double().cpu().numpy()[win]
        err = float(np.max(np.abs(dev - ref[win])) / np.max(np.abs(ref[win])))
        assert err <= 1e-5, f"corner {'high' if high else 'low'}: {err}"
