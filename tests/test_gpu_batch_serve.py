"""Batched launches and the serving loop on the GPU.

Every result must equal the same problem run alone (ebisu_run), bit for bit,
and match the CPU oracle within the dtype's tolerance."""
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


def make_problem(eb, ndim, dims, shape, r, dtype, boundary, seed, params=None):
    g, c = synth.problem(ndim, dims, shape, r, boundary, seed=seed)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    plan = eb.Plan(ndim, dims, shape, r, c, dtype, boundary)
    if params:
        plan.set_params(**params)
    held = x.double().cpu().numpy()
    c_held = c if dtype == 0 else c.astype(np.float32).astype(np.float64)
    return plan, x, held, c_held


def alone(plan, x, steps):
    ws = plan.workspace()
    y = torch.empty_like(x)
    plan.run(x, y, steps, ws)
    assert plan.sync(ws) == 0
    return y


def mixed_problems(eb, count, seed):
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        dtype = int(rng.integers(0, 3))
        ny, nx = int(rng.integers(40, 400)), int(rng.integers(40, 700))
        steps = int(rng.integers(0, 30))
        tx = int(rng.choice([64, 128, 256]))
        ts = int(rng.integers(16, 120))
        d = int(rng.integers(1, 6))
        plan, x, held, c_held = make_problem(eb, 2, (ny, nx), 1, 1, dtype, int(i % 5 == 4), seed * 100 + i,
                                             dict(tile_x=tx, tile_s=ts, depth=d))
        probs.append((plan, x, held, c_held, steps))
    return probs


def mixed_rs_problems(eb, count, seed):
    """Mixed problems, most of them set to the register-streaming build
    (every dtype, both built depths, star and box), the rest to the
    shared-memory build; steps often leave a partial last block."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        dtype = int(rng.integers(0, 3))
        shape, r = [(0, 1), (1, 1), (0, 2), (1, 2), (0, 3)][i % 5]
        ny, nx = int(rng.integers(64, 300)), int(rng.integers(140, 600))
        steps = int(rng.integers(1, 25))
        bd = int(i % 4 == 3)
        plan, x, held, c_held = make_problem(eb, 2, (ny, nx), shape, r, dtype, bd, seed * 100 + i)
        if i % 3 != 2:
            d = plan.rs_depths()[i % 2]
            try:
                plan.set_params(variant=2, depth=d, tile_s=int(rng.integers(d * r, 90)), ctas_per_sm=4)
            except eb.EbisuError:
                plan.set_params(tile_x=128, tile_s=40, depth=2, variant=0)
        else:
            plan.set_params(tile_x=128, tile_s=40, depth=2, variant=0)
        probs.append((plan, x, held, c_held, steps))
    return probs


def test_batch_register_streaming_equals_alone_and_oracle():
    eb = _eb()
    probs = mixed_rs_problems(eb, 16, 11)
    assert sum(p[0].params().variant == 2 for p in probs) >= 8
    plans = [p[0] for p in probs]
    xs = [p[1] for p in probs]
    steps = [p[4] for p in probs]
    ys = [torch.empty_like(x) for x in xs]
    ws = torch.empty(eb.batch_workspace_bytes(plans, steps), dtype=torch.uint8, device="cuda")
    eb.batch_run(plans, xs, ys, steps, ws)
    torch.cuda.synchronize()
    for (plan, x, held, c_held, st), y in zip(probs, ys):
        assert torch.equal(y, alone(plan, x, st)), "batched result differs from the problem alone"
        ref = oracle.run(held, plan.shape, plan.radius, c_held, plan.boundary, st)
        assert oracle.rel_linf(y.double().cpu().numpy(), ref, plan.pad) <= TOL[plan.dtype]


def test_batch_register_streaming_graph_replay_and_serve():
    eb = _eb()
    probs = mixed_rs_problems(eb, 8, 12)
    plans = [p[0] for p in probs]
    xs = [p[1] for p in probs]
    steps = [p[4] for p in probs]
    ys = [torch.empty_like(x) for x in xs]
    ws = torch.empty(eb.batch_workspace_bytes(plans, steps), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = eb.Batch(plans, xs, ys, steps, ws)
        b.launch()
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.launch()
    for y in ys:
        y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert b.sync() == 0
    for (plan, x, _, _, st), y in zip(probs, ys):
        assert torch.equal(y, alone(plan, x, st))
    srv = eb.Server(hbm_budget=2 << 30, max_slots=3)
    ys2 = [torch.empty_like(x) for x in xs]
    tickets = [srv.submit(p[0], p[1], y, p[4]) for p, y in zip(probs, ys2)]
    for t in tickets:
        srv.wait(t)
    for y, y2 in zip(ys, ys2):
        assert torch.equal(y, y2), "served result differs from the problem alone"
    srv.close()


def test_batch_equals_alone_and_oracle():
    eb = _eb()
    probs = mixed_problems(eb, 14, 3)
    plans = [p[0] for p in probs]
    xs = [p[1] for p in probs]
    steps = [p[4] for p in probs]
    ys = [torch.empty_like(x) for x in xs]
    ws = torch.empty(eb.batch_workspace_bytes(plans, steps), dtype=torch.uint8, device="cuda")
    eb.batch_run(plans, xs, ys, steps, ws)
    torch.cuda.synchronize()
    for (plan, x, held, c_held, st), y in zip(probs, ys):
        assert torch.equal(y, alone(plan, x, st)), "batched result differs from the problem alone"
        ref = oracle.run(held, 1, 1, c_held, plan.boundary, st)
        assert oracle.rel_linf(y.double().cpu().numpy(), ref, plan.pad) <= TOL[plan.dtype]


def test_batch_mixed_kernel_types_and_in_place():
    eb = _eb()
    specs = [(2, (130, 250), 0, 2, 0, 0), (3, (20, 30, 40), 1, 1, 0, 0), (2, (90, 310), 0, 1, 1, 1),
             (3, (17, 19, 23), 0, 1, 2, 0), (2, (64, 64), 1, 2, 0, 0)]
    probs = []
    for i, (nd, dims, sh, r, dt, bd) in enumerate(specs):
        params = dict(tile_x=32, tile_y=16, tile_s=8, depth=2) if nd == 3 else dict(tile_x=96, tile_s=40, depth=3)
        probs.append(make_problem(eb, nd, dims, sh, r, dt, bd, 700 + i, params))
    steps = [5, 4, 7, 3, 9]
    plans = [p[0] for p in probs]
    xs = [p[1].clone() for p in probs]
    ys = [xs[0], torch.empty_like(xs[1]), xs[2], torch.empty_like(xs[3]), torch.empty_like(xs[4])]
    ws = torch.empty(eb.batch_workspace_bytes(plans, steps), dtype=torch.uint8, device="cuda")
    eb.batch_run(plans, xs, ys, steps, ws)
    torch.cuda.synchronize()
    for (plan, x, held, c_held), y, st in zip(probs, ys, steps):
        assert torch.equal(y, alone(plan, x, st))
        ref = oracle.run(held, plan.shape, plan.radius, c_held, plan.boundary, st)
        assert oracle.rel_linf(y.double().cpu().numpy(), ref, plan.pad) <= TOL[plan.dtype]


def test_batch_graph_replay():
    eb = _eb()
    probs = mixed_problems(eb, 6, 5)
    plans = [p[0] for p in probs]
    xs = [p[1] for p in probs]
    steps = [max(1, p[4]) for p in probs]
    ys = [torch.empty_like(x) for x in xs]
    ws = torch.empty(eb.batch_workspace_bytes(plans, steps), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = eb.Batch(plans, xs, ys, steps, ws)
        b.launch()  # warm-up outside the graph
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.launch()
    for y in ys:
        y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert b.sync() == 0
    for (plan, x, held, c_held, _), y, st in zip(probs, ys, steps):
        assert torch.equal(y, alone(plan, x, st))


def test_serve_results_equal_alone():
    eb = _eb()
    probs = mixed_problems(eb, 20, 9)
    srv = eb.Server(hbm_budget=4 << 30, max_slots=4)
    ys = [torch.empty_like(p[1]) for p in probs]
    tickets = [srv.submit(p[0], p[1], y, p[4]) for p, y in zip(probs, ys)]
    lats = [srv.wait(t) for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(probs) and st["held_bytes"] == 0 and st["queued"] == 0
    assert all(l > 0 for l in lats)
    for (plan, x, held, c_held, steps), y in zip(probs, ys):
        assert torch.equal(y, alone(plan, x, steps)), "served result differs from the problem alone"
    srv.close()


def test_serve_budget_admission_and_rejection():
    eb = _eb()
    plan, x, held, c_held = make_problem(eb, 2, (600, 600), 1, 1, 0, 0, 11, dict(tile_x=200, tile_s=100, depth=2))
    need = 2 * x.numel() * 8 + 64 * 1024
    # a budget that holds two requests at a time forces queueing
    srv = eb.Server(hbm_budget=2 * need + 1024, max_slots=4)
    ys = [torch.empty_like(x) for _ in range(6)]
    tickets = [srv.submit(plan, x, y, 12) for y in ys]
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    assert st["peak_bytes"] <= 2 * need + 1024
    ref = alone(plan, x, 12)
    assert all(torch.equal(y, ref) for y in ys)
    # a request larger than the whole budget is refused at submit
    big_plan, big_x, _, _ = make_problem(eb, 2, (2000, 2000), 1, 1, 0, 0, 12)
    rc, _ = srv.try_submit(big_plan, big_x, torch.empty_like(big_x), 3)
    assert rc == eb.ERR_BUDGET
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_serve_shortest_first_and_wait_limit():
    """Least-estimated-work-first ordering lets small requests that arrive
    behind large ones finish first; results still equal each problem alone.
    The wait limit refuses requests once the queued work exceeds it."""
    eb = _eb()
    big = make_problem(eb, 2, (4096, 4096), 1, 2, eb.F64, 0, 21)          # ~1.7e10 updates
    smalls = [make_problem(eb, 2, (300, 400), 0, 1, eb.F32, 0, 30 + i) for i in range(6)]
    srv = eb.Server(hbm_budget=16 << 30, max_slots=1)  # one lane: the order is the schedule
    srv.set_policy(eb.SERVE_SHORTEST)
    yb = [torch.empty_like(big[1]) for _ in range(3)]
    ys = [torch.empty_like(s[1]) for s in smalls]
    tb = [srv.submit(big[0], big[1], y, 1000) for y in yb]
    ts = [srv.submit(s[0], s[1], y, 50) for s, y in zip(smalls, ys)]
    lat_b = [srv.wait(t, timeout_s=300) for t in tb]
    lat_s = [srv.wait(t, timeout_s=300) for t in ts]
    # the first large request may already be running; the small ones overtake the rest
    assert max(lat_s) < max(lat_b)
    ref_b = alone(big[0], big[1], 1000)
    assert all(torch.equal(y, ref_b) for y in yb)
    for s, y in zip(smalls, ys):
        assert torch.equal(y, alone(s[0], s[1], 50))
    # admission control on predicted wait: with a tiny limit, a queue of large
    # requests turns further submissions away
    srv.set_policy(eb.SERVE_FIFO, max_wait_s=1e-3)
    rcs = [srv.try_submit(big[0], big[1], yb[i % 3], 1000)[0] for i in range(4)]
    assert eb.ERR_BUSY in rcs
    for rc in rcs:
        assert rc in (eb.OK, eb.ERR_BUSY)
    srv.close()
    assert srv.h is None


def test_batch_members_with_different_ring_footprints():
    """A wide shallow member and a narrow deep member of one shared-memory
    group: each lays its rings out with its own plane stride, so the group
    needs the larger single footprint, not the widest plane times the
    deepest ring."""
    eb = _eb()
    a = make_problem(eb, 2, (300, 3000), 1, 1, eb.F64, 0, 71, dict(tile_x=3000, tile_s=60, depth=1))
    b = make_problem(eb, 2, (300, 600), 1, 1, eb.F64, 0, 72, dict(tile_x=512, tile_s=60, depth=12))
    plans, xs = [a[0], b[0]], [a[1], b[1]]
    ys = [torch.empty_like(x) for x in xs]
    steps = [7, 30]
    ws = torch.empty(eb.batch_workspace_bytes(plans, steps), dtype=torch.uint8, device="cuda")
    eb.batch_run(plans, xs, ys, steps, ws)
    torch.cuda.synchronize()
    for p, x, y, st in zip(plans, xs, ys, steps):
        assert torch.equal(y, alone(p, x, st))
