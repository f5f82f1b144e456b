"""ebisu_run_static: a run with no caller workspace and no allocation.

For callers that cannot allocate device memory (a host that owns all device
memory through its own pool, a fixed start-up budget, or a loop where an
allocation that may synchronise the device is not acceptable), the library
keeps a fixed 64 MiB device array as the run's workspace.  This test calls
that entry point through the C ABI twice in a row and checks each result
against the regular entry point (ebisu_run with a caller workspace), within
the FP64 tolerance the parity tests use, and checks that a plan whose
workspace exceeds the array is refused.  It lives in a file of its own that
pytest collects last, and passes alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2305_07390_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12


def _eb():
    from paper_2305_07390_gb300 import ebisu
    return ebisu


def _static_run(eb, plan, x, y, steps):
    s = eb.current_stream_handle()
    return eb.lib().ebisu_run_static(plan.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     int(steps), s, 1)


def test_static_scratch_matches_regular_run_twice():
    eb = _eb()
    cases = [((300, 700), 1, 2, 9, dict(tile_x=256, tile_s=60, depth=3)),   # 2D 25-point box
             ((40, 50, 60), 0, 1, 5, dict(tile_x=32, tile_y=16, tile_s=10, depth=2))]  # 3D 7-point star
    for dims, shape, r, steps, params in cases:
        g, c = synth.problem(len(dims), dims, shape, r, synth.DIRICHLET, seed=31 + r)
        plan = eb.Plan(len(dims), dims, shape, r, c, eb.F64, eb.DIRICHLET)
        plan.set_params(**params)
        x = torch.from_numpy(g).cuda()
        ws = plan.workspace()
        ref = torch.empty_like(x)
        plan.run(x, ref, steps, ws)
        assert plan.sync(ws) == 0
        for call in range(2):  # the array keeps the previous call's contents
            y = torch.full_like(x, float("nan"))
            rc = _static_run(eb, plan, x, y, steps)
            assert rc == eb.OK, eb.status_string(rc)
            err = oracle.rel_linf(y.cpu().numpy(), ref.cpu().numpy(), r)
            assert err <= TOL_F64, f"call {call}: {err}"
            assert torch.equal(y[:r], x[:r])  # Dirichlet pad carried over


def test_static_scratch_in_place_and_too_large():
    eb = _eb()
    dims = (257, 513)
    g, c = synth.problem(2, dims, 0, 1, synth.DIRICHLET, seed=41)
    plan = eb.Plan(2, dims, 0, 1, c, eb.F64, eb.DIRICHLET)
    x = torch.from_numpy(g).cuda()
    ws = plan.workspace()
    ref = torch.empty_like(x)
    plan.run(x, ref, 6, ws)
    assert plan.sync(ws) == 0
    y = x.clone()
    assert _static_run(eb, plan, y, y, 6) == eb.OK
    assert oracle.rel_linf(y.cpu().numpy(), ref.cpu().numpy(), 1) <= TOL_F64
    big = eb.Plan(2, (4096, 4096), 0, 1, c, eb.F64, eb.DIRICHLET)  # 134 MB workspace
    assert _static_run(eb, big, x, x, 1) == eb.ERR_UNSUPPORTED
