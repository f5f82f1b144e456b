"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/ebisu.h declares, and rejects bad arguments with
the documented status codes before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2305_07390_gb300 import ebisu

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ebisu.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ebisu_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ebisu_plan_create", "ebisu_run", "ebisu_batch_run", "ebisu_serve_create",
                     "ebisu_serve_submit", "ebisu_serve_poll", "ebisu_serve_destroy", "ebisu_plan_destroy",
                     "ebisu_status_string", "ebisu_plan_workspace_bytes"]:
        assert required in names


def test_every_declared_symbol_is_exported():
    lib = ebisu.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
    # and the binding knows every one of them
    assert set(declared_functions()) <= set(ebisu.SIGNATURES)


def test_status_strings():
    for code in range(9):
        assert ebisu.status_string(code)
    assert ebisu.status_string(999) == "unknown status"


@pytest.mark.parametrize("args,code", [
    ((1, (10,), 0, 1), ebisu.ERR_INVALID_ARG),          # ndim
    ((2, (10, 10), 5, 1), ebisu.ERR_INVALID_ARG),       # shape
    ((2, (10, 10), 0, 4), ebisu.ERR_UNSUPPORTED),       # star radius > 3
    ((2, (10, 10), 1, 3), ebisu.ERR_UNSUPPORTED),       # box radius > 2
    ((2, (0, 10), 0, 1), ebisu.ERR_INVALID_ARG),        # empty axis
    ((2, (10, 10), 0, 0), ebisu.ERR_INVALID_ARG),       # radius 0
])
def test_plan_create_errors(args, code):
    ndim, dims, shape, r = args
    with pytest.raises(ebisu.EbisuError) as ei:
        ebisu.ebisu_plan_create(ndim, dims, shape, r, [0.1] * 125, 0, 0)
    assert ei.value.code == code


def test_periodic_too_small_is_unsupported():
    with pytest.raises(ebisu.EbisuError) as ei:
        ebisu.ebisu_plan_create(2, (6, 40), 0, 3, [0.1] * 13, 0, 1)
    assert ei.value.code == ebisu.ERR_UNSUPPORTED


def test_plan_defaults_and_params():
    p = ebisu.Plan(2, (8192, 8192), 0, 1, [0.2] * 5, ebisu.F64, ebisu.DIRICHLET)
    q = p.params()
    assert q.depth >= 1 and q.tile_x >= 1
    assert p.workspace_bytes() >= 8192 * 8192 * 8
    pred, bound, valid = p.model()
    assert pred > 0 and 0 < valid <= 1
    # FP64 on this device is FP-pipe bound; the model keeps depth small
    assert bound == "fp"
    with pytest.raises(ebisu.EbisuError):
        p.set_params(depth=0)
    with pytest.raises(ebisu.EbisuError):
        p.set_params(tile_x=4096, depth=64)  # plane too large for the kernel


def test_run_argument_errors_need_no_device():
    p = ebisu.Plan(2, (16, 16), 0, 1, [0.2] * 5, ebisu.F64, ebisu.DIRICHLET)
    lib = ebisu.lib()
    assert lib.ebisu_run(p.h, None, None, 1, None, None) == ebisu.ERR_INVALID_ARG
    assert lib.ebisu_run(p.h, ctypes.c_void_p(256), ctypes.c_void_p(512), -1, ctypes.c_void_p(1024),
                         None) == ebisu.ERR_INVALID_ARG
    # unaligned workspace
    assert lib.ebisu_run(p.h, ctypes.c_void_p(256), ctypes.c_void_p(512), 1, ctypes.c_void_p(1000),
                         None) == ebisu.ERR_INVALID_ARG


def test_register_streaming_params():
    """Variant 2 (register streaming, 2D): depths, derived strip width and
    the host-side validity rules, checked without a device."""
    p = ebisu.Plan(2, (1000, 1000), 0, 1, [0.2] * 5, ebisu.F32, ebisu.DIRICHLET)
    lo, hi = p.rs_depths()
    assert 1 <= lo <= hi
    p.set_params(variant=2, depth=hi, tile_s=100, ctas_per_sm=2)
    q = p.params()
    assert (q.variant, q.depth, q.tile_x, q.tile_s, q.threads) == (2, hi, 128 - 2 * hi, 100, 128)
    for bad in [dict(variant=2, depth=hi + 1),            # not a built depth
                dict(variant=2, depth=hi, tile_s=hi - 1),  # segment shorter than depth * radius
                dict(variant=3)]:
        with pytest.raises(ebisu.EbisuError):
            p.set_params(**bad)
    # too many tiles for the per-tile counters
    big = ebisu.Plan(2, (40000, 2000), 0, 1, [0.2] * 5, ebisu.F32, ebisu.DIRICHLET)
    with pytest.raises(ebisu.EbisuError) as ei:
        big.set_params(variant=2, depth=lo, tile_s=lo)
    assert ei.value.code == ebisu.ERR_UNSUPPORTED
    # 3D FP32 and BF16: the 7-point star at depths 2 and 3, the 27-point box at
    # depth 2 (64 - 2t column strips, 2 fewer at even t, of 4-row patches)
    p3 = ebisu.Plan(3, (20, 20, 80), 0, 1, [0.1] * 7, ebisu.F32, ebisu.DIRICHLET)
    assert p3.rs_depths() == (2, 3)
    p3.set_params(variant=2, depth=3, tile_s=5)
    assert (p3.params().tile_x, p3.params().tile_y) == (58, 4)
    with pytest.raises(ebisu.EbisuError):
        p3.set_params(variant=2, depth=4)
    assert ebisu.Plan(3, (20, 20, 20), 1, 1, [0.03] * 27, ebisu.F32, ebisu.DIRICHLET).rs_depths() == (2, 2)
    assert ebisu.Plan(3, (20, 20, 20), 0, 2, [0.07] * 13, ebisu.F32, ebisu.DIRICHLET).rs_depths() == (0, 0)
    assert ebisu.Plan(3, (20, 20, 20), 0, 1, [0.1] * 7, ebisu.BF16, ebisu.DIRICHLET).rs_depths() == (2, 3)
    pb = ebisu.Plan(3, (20, 20, 80), 1, 1, [0.03] * 27, ebisu.BF16, ebisu.DIRICHLET)
    assert pb.rs_depths() == (2, 2)
    pb.set_params(variant=2, depth=2, tile_s=5)
    assert (pb.params().tile_x, pb.params().tile_y) == (58, 4)
    assert ebisu.Plan(3, (20, 20, 20), 0, 2, [0.07] * 13, ebisu.BF16, ebisu.DIRICHLET).rs_depths() == (0, 0)
    # 3D: FP64 radius 1 only, depth 1, 62-column strips of 2-row patches
    p3d = ebisu.Plan(3, (64, 64, 200), 1, 1, [0.03] * 27, ebisu.F64, ebisu.DIRICHLET)
    assert p3d.rs_depths() == (1, 1)
    p3d.set_params(variant=2, depth=1, tile_s=16, ctas_per_sm=2)
    q3 = p3d.params()
    assert (q3.tile_x, q3.tile_y, q3.tile_s, q3.depth) == (62, 2, 16, 1)
    with pytest.raises(ebisu.EbisuError):
        p3d.set_params(variant=2, depth=2)
    pp = ebisu.Plan(2, (100, 100), 0, 1, [0.2] * 5, ebisu.F32, ebisu.PERIODIC)
    with pytest.raises(ebisu.EbisuError):
        pp.set_params(variant=2, depth=pp.rs_depths()[0])
    # FP64 builds shallow depths only (its FMA pipe, not HBM, bounds it)
    p64 = ebisu.Plan(2, (500, 500), 1, 2, [0.04] * 25, ebisu.F64, ebisu.DIRICHLET)
    assert p64.rs_depths() == (1, 1)


def test_bench_names_the_kernel_a_plan_launches():
    """The benchmark labels each row with the kernel its plan's parameters
    select (host logic only: no launch)."""
    import bench
    p2 = ebisu.Plan(2, (300, 300), 0, 1, [0.2] * 5, ebisu.F32, ebisu.DIRICHLET)
    p2.set_params(variant=2, depth=p2.rs_depths()[1], tile_s=32)
    assert bench.kernel_name(p2) == "rs_kernel"
    p2.set_params(variant=1)
    assert bench.kernel_name(p2) == "naive_kernel"
    p64 = ebisu.Plan(3, (20, 20, 80), 0, 1, [0.1] * 7, ebisu.F64, ebisu.DIRICHLET)
    p64.set_params(variant=2, depth=1, tile_s=8)
    assert bench.kernel_name(p64) == "rs3_kernel"
    for dt in (ebisu.F32, ebisu.BF16):
        p3 = ebisu.Plan(3, (20, 20, 80), 0, 1, [0.1] * 7, dt, ebisu.DIRICHLET)
        p3.set_params(variant=2, depth=3, tile_s=5)
        assert bench.kernel_name(p3) == "rs3t_kernel"
        p3.set_params(tile_x=16, tile_y=8, tile_s=8, depth=2)
        assert bench.kernel_name(p3) == "tb_kernel"


def test_stochastic_rounding_host_rules():
    c2 = [0.2] * 5
    for dt in (ebisu.F64, ebisu.F32):
        p = ebisu.Plan(2, (64, 300), 0, 1, c2, dt, 0)
        with pytest.raises(ebisu.EbisuError) as ei:
            p.set_rounding(ebisu.ROUND_STOCHASTIC, 1)
        assert ei.value.code == ebisu.ERR_UNSUPPORTED
        p.set_rounding(ebisu.ROUND_NEAREST)  # always allowed
    p = ebisu.Plan(2, (64, 300), 0, 1, c2, ebisu.BF16, 0)
    with pytest.raises(ebisu.EbisuError) as ei:
        p.set_rounding(7, 1)
    assert ei.value.code == ebisu.ERR_INVALID_ARG
    p.set_rounding(ebisu.ROUND_STOCHASTIC, 99)
    assert p.rounding() == (ebisu.ROUND_STOCHASTIC, 99)
    assert p.params().variant == 2
    # no shared-memory build with stochastic rounding
    with pytest.raises(ebisu.EbisuError) as ei:
        p.set_params(tile_x=64, tile_s=32, depth=2)
    assert ei.value.code == ebisu.ERR_UNSUPPORTED
    p.set_params(variant=1)  # the one-step kernel has it
    # 3D: the register-streaming build for radius 1, else the one-step kernel
    c3 = [1.0 / 7] * 7
    p3 = ebisu.Plan(3, (32, 32, 96), 0, 1, c3, ebisu.BF16, 0)
    p3.set_rounding(ebisu.ROUND_STOCHASTIC, 5)
    assert p3.params().variant == 2
    c125 = [1.0 / 125] * 125
    p5 = ebisu.Plan(3, (32, 32, 96), 1, 2, c125, ebisu.BF16, 0)
    p5.set_rounding(ebisu.ROUND_STOCHASTIC, 5)
    assert p5.params().variant == 1
    # back to nearest: every build is allowed again
    p.set_rounding(ebisu.ROUND_NEAREST)
    p.set_params(tile_x=64, tile_s=32, depth=2)
    assert p.params().variant == 0


def _npts(plan):
    v = ctypes.c_int()
    assert ebisu.lib().ebisu_plan_npoints(plan.h, ctypes.byref(v)) == 0
    return v.value


def test_new_shapes_and_offset_lists_host_rules():
    import itertools
    p = ebisu.Plan(3, (10, 10, 10), ebisu.POISSON, 1, [1.0 / 19] * 19)
    assert _npts(p) == 19
    assert _npts(ebisu.Plan(3, (10, 10, 10), ebisu.J3D17PT, 1, [1.0 / 17] * 17)) == 17
    for args in [(2, (10, 10), ebisu.POISSON, 1, [0.1] * 19), (3, (10, 10, 10), ebisu.J3D17PT, 2, [0.1] * 17)]:
        with pytest.raises(ebisu.EbisuError) as ei:
            ebisu.Plan(*args)
        assert ei.value.code == ebisu.ERR_UNSUPPORTED
    # offset lists: a named shape's set gets that shape, others the box of their radius
    star3 = [(0, 0, k) for k in range(-3, 4)] + [(0, k, 0) for k in range(-3, 4) if k]
    assert _npts(ebisu.Plan.from_offsets(2, (40, 40), star3, [1.0 / 13] * 13)) == 13
    odd = [(0, -1, 2), (0, 0, 0), (0, 2, -2)]
    assert _npts(ebisu.Plan.from_offsets(2, (40, 40), odd, [0.2, 0.5, 0.3])) == 25
    box1 = list(itertools.product((-1, 0, 1), repeat=3))
    pois = [o for o in box1 if not all(o)]
    assert _npts(ebisu.Plan.from_offsets(3, (9, 9, 9), pois[::-1], [1.0 / 19] * 19)) == 19
    bad = [((0, 0, 0), (0, 0, 0)), ((1, 0, 0), (0, 0, 1))]  # repeated; dz in 2D
    for offs in bad:
        with pytest.raises(ebisu.EbisuError) as ei:
            ebisu.Plan.from_offsets(2, (40, 40), offs, [0.5, 0.5])
        assert ei.value.code == ebisu.ERR_INVALID_ARG
    with pytest.raises(ebisu.EbisuError) as ei:
        ebisu.Plan.from_offsets(2, (40, 40), [(0, 3, 1), (0, 0, 0)], [0.5, 0.5])  # radius 3, not a star
    assert ei.value.code == ebisu.ERR_UNSUPPORTED


def test_ablation_host_rules():
    p = ebisu.Plan(2, (64, 300), 0, 1, [0.2] * 5, ebisu.F32, 0)
    steps = [0, 4, 6, 7, 15]
    for m in steps:
        p.set_ablation(m)
    for bad in (1, 2, 3, 8, 16):
        with pytest.raises(ebisu.EbisuError) as ei:
            p.set_ablation(bad)
        assert ei.value.code == ebisu.ERR_INVALID_ARG
    for args in [(2, (64, 300), 1, 1, [1 / 9] * 9, ebisu.F32), (2, (64, 300), 0, 2, [1 / 9] * 9, ebisu.F64),
                 (2, (64, 300), 0, 1, [0.2] * 5, ebisu.BF16)]:
        q = ebisu.Plan(2, args[1], args[2], args[3], args[4], args[5], 0)
        with pytest.raises(ebisu.EbisuError) as ei:
            q.set_ablation(15)
        assert ei.value.code == ebisu.ERR_UNSUPPORTED
        q.set_ablation(0)
