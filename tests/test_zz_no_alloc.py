"""ebisu_run_static: a run with no caller workspace and no allocation.

For callers that cannot allocate device memory (a host that owns all device
memory through its own pool, a fixed start-up budget, or a loop where an
allocation that may synchronise the device is not acceptable), the library
keeps a fixed 64 MiB device array as the run's workspace.  These tests call
that entry point through the C ABI twice in a row and check each result
against the regular entry point (ebisu_run with a caller workspace): both
run the same kernel on the same inputs, so the results must be identical.
They cover every path through the array (the shared-memory, register-
streaming and one-step builds; zero, odd and even step counts; in == out,
which on the one-step path first copies the input into the array), the
asynchronous form (wait = 0) followed by ebisu_sync_static, and a plan whose
workspace exceeds the array, which is refused.  The file is collected last
and passes alone or after the other tests.
"""
import ctypes

import pytest

from paper_2305_07390_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _eb():
    from paper_2305_07390_gb300 import ebisu
    return ebisu


def _static_run(eb, plan, x, y, steps, wait=1):
    s = eb.current_stream_handle()
    return eb.lib().ebisu_run_static(plan.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     int(steps), s, int(wait))


def _static_sync(eb):
    return eb.lib().ebisu_sync_static(eb.current_stream_handle())


# (dims, shape, radius, dtype, parameters): the shared-memory build (2D and
# 3D), the register-streaming build (2D and 3D) and the one-step build
CASES = [
    ((300, 700), 1, 2, 0, dict(tile_x=256, tile_s=60, depth=3)),                      # 2D 25-point box
    ((40, 50, 60), 0, 1, 0, dict(tile_x=32, tile_y=16, tile_s=10, depth=2)),          # 3D 7-point star
    ((260, 530), 0, 1, 1, dict(variant=2, depth=4, tile_s=48, ctas_per_sm=4)),        # 2D FP32 registers
    ((20, 24, 90), 0, 1, 1, dict(variant=2, depth=3, tile_s=8, ctas_per_sm=4)),       # 3D FP32 registers
    ((130, 170), 1, 1, 0, dict(variant=1)),                                            # one step per launch
]


def _problem(eb, dims, shape, r, dtype, params, seed):
    g, c = synth.problem(len(dims), dims, shape, r, synth.DIRICHLET, seed=seed)
    plan = eb.Plan(len(dims), dims, shape, r, c, dtype, eb.DIRICHLET)
    plan.set_params(**params)
    x = torch.from_numpy(g).to(eb.torch_dtype(dtype)).cuda()
    return plan, x


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("steps", [0, 5, 6])
def test_static_scratch_matches_regular_run_twice(case, steps):
    eb = _eb()
    dims, shape, r, dtype, params = CASES[case]
    plan, x = _problem(eb, dims, shape, r, dtype, params, seed=31 + case)
    ws = plan.workspace()
    ref = torch.empty_like(x)
    plan.run(x, ref, steps, ws)
    assert plan.sync(ws) == 0
    for call in range(2):  # the array keeps the previous call's contents
        y = torch.full_like(x, float("nan"))
        rc = _static_run(eb, plan, x, y, steps)
        assert rc == eb.OK, eb.status_string(rc)
        assert torch.equal(y, ref), f"call {call} differs from ebisu_run"


@pytest.mark.parametrize("case", [0, 2, 4])
@pytest.mark.parametrize("steps", [5, 6])
def test_static_scratch_in_place(case, steps):
    eb = _eb()
    dims, shape, r, dtype, params = CASES[case]
    plan, x = _problem(eb, dims, shape, r, dtype, params, seed=41 + case)
    ws = plan.workspace()
    ref = torch.empty_like(x)
    plan.run(x, ref, steps, ws)
    assert plan.sync(ws) == 0
    for call in range(2):
        y = x.clone()
        rc = _static_run(eb, plan, y, y, steps)
        assert rc == eb.OK, eb.status_string(rc)
        assert torch.equal(y, ref), f"call {call} differs from ebisu_run"


def test_static_scratch_async_then_status_read():
    eb = _eb()
    for case in (0, 2, 4):
        dims, shape, r, dtype, params = CASES[case]
        plan, x = _problem(eb, dims, shape, r, dtype, params, seed=51 + case)
        ws = plan.workspace()
        ref = torch.empty_like(x)
        plan.run(x, ref, 7, ws)
        assert plan.sync(ws) == 0
        for call in range(2):
            y = torch.full_like(x, float("nan"))
            assert _static_run(eb, plan, x, y, 7, wait=0) == eb.OK
            rc = _static_sync(eb)
            assert rc == eb.OK, eb.status_string(rc)
            assert torch.equal(y, ref), f"case {case} call {call}"


def test_static_scratch_too_large_is_refused():
    eb = _eb()
    dims = (257, 513)
    g, c = synth.problem(2, dims, 0, 1, synth.DIRICHLET, seed=41)
    x = torch.from_numpy(g).cuda()
    big = eb.Plan(2, (4096, 4096), 0, 1, c, eb.F64, eb.DIRICHLET)  # 134 MB workspace
    assert _static_run(eb, big, x, x, 1) == eb.ERR_UNSUPPORTED
