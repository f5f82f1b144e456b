"""Thin ctypes binding of the C ABI in ``include/ebisu.h``.

Every function named ``ebisu_*`` here marshals its arguments and calls the C
entry point of the same name; no step of the stencil path runs in Python.
Device memory comes from PyTorch tensors (their ``data_ptr()``), streams from
``torch.cuda`` (their ``cuda_stream`` handle).  :class:`Plan` is a small
convenience wrapper over the same calls.

The library must be built (``__graft_entry__.build()`` or
``python -m paper_2305_07390_gb300.build``); loading fails loudly otherwise.
There is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libebisu.so")

(OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_OOM, ERR_BUDGET, ERR_TIMEOUT, ERR_DEVICE_FAULT,
 ERR_NOT_READY, ERR_BUSY) = range(10)
STAR, BOX, POISSON, J3D17PT = 0, 1, 2, 3
F64, F32, BF16 = 0, 1, 2
DIRICHLET, PERIODIC = 0, 1
ROUND_NEAREST, ROUND_STOCHASTIC = 0, 1
SERVE_FIFO, SERVE_SHORTEST = 0, 1
ABLATE_PREFETCH, ABLATE_LAZY, ABLATE_REGISTER_REUSE, ABLATE_CIRCULAR = 1, 2, 4, 8


class EbisuError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {status_string(code)} ({code})"
        if code == ERR_CUDA:
            msg += f": {last_cuda_error()}"
        super().__init__(msg)


class Params(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("tile_s", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("fused_variant", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ModelIn(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("a_gm", "a_sm", "a_cmp", "d_gm", "d_sm", "d_cmp", "s_cell",
                                               "b_gm", "b_sm", "thr_cmp", "t", "t_dsync", "n_sync",
                                               "tile_x", "tile_y", "rad")] + \
               [("ndim", ctypes.c_int32), ("tiling", ctypes.c_int32)]


class ModelOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("t_gm", "t_sm", "t_cmp", "t_stencil", "p", "v_smtile",
                                               "v_dtile", "pp", "depth_sm", "depth_device",
                                               "min_device_tile")] + \
               [("bound", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_D = ctypes.c_double

# name: (restype, argtypes) -- mirrors include/ebisu.h
SIGNATURES = {
    "ebisu_status_string": (ctypes.c_char_p, [_I]),
    "ebisu_version": (_I, []),
    "ebisu_last_cuda_error": (ctypes.c_char_p, []),
    "ebisu_plan_create": (_I, [_I, ctypes.POINTER(_I64), _I, _I, ctypes.POINTER(_D), _I, _I, ctypes.POINTER(_P)]),
    "ebisu_plan_create_offsets": (_I, [_I, ctypes.POINTER(_I64), _I, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(_D), _I, _I, ctypes.POINTER(_P)]),
    "ebisu_plan_destroy": (_I, [_P]),
    "ebisu_plan_npoints": (_I, [_P, ctypes.POINTER(_I)]),
    "ebisu_plan_grid_elems": (_I, [_P, ctypes.POINTER(_I64)]),
    "ebisu_plan_get_params": (_I, [_P, ctypes.POINTER(Params)]),
    "ebisu_plan_set_params": (_I, [_P, ctypes.POINTER(Params)]),
    "ebisu_plan_rs_depths": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "ebisu_plan_set_rounding": (_I, [_P, _I, ctypes.c_uint64]),
    "ebisu_plan_set_ablation": (_I, [_P, _I]),
    "ebisu_plan_set_coefficient_field": (_I, [_P, _P]),
    "ebisu_plan_get_rounding": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_uint64)]),
    "ebisu_plan_workspace_bytes": (_I, [_P, ctypes.POINTER(_SZ)]),
    "ebisu_run": (_I, [_P, _P, _P, _I64, _P, _P]),
    "ebisu_run_naive": (_I, [_P, _P, _P, _I64, _P, _P]),
    "ebisu_run_static": (_I, [_P, _P, _P, _I64, _P, _I]),
    "ebisu_sync_static": (_I, [_P]),
    "ebisu_sync": (_I, [_P, _P]),
    "ebisu_plan_tune": (_I, [_P, _P, _P, _I64, _P, _I, ctypes.POINTER(_D), _P]),
    "ebisu_plan_tune_share": (_I, [_P, _P, _P, _I64, _P, _I, _D, ctypes.POINTER(_D), _P]),
    "ebisu_plan_model": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "ebisu_cost_model": (_I, [ctypes.POINTER(ModelIn), ctypes.POINTER(ModelOut)]),
    "ebisu_reduce": (_I, [_P, _P, _P, ctypes.POINTER(_D), _P, _P]),
    "ebisu_batch_workspace_bytes": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.POINTER(_SZ)]),
    "ebisu_batch_run": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                             ctypes.POINTER(_I64), _P, _P]),
    "ebisu_batch_create": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                ctypes.POINTER(_I64), _P, _P, ctypes.POINTER(_P)]),
    "ebisu_batch_launch": (_I, [_P, _P]),
    "ebisu_batch_sync": (_I, [_P, _P]),
    "ebisu_batch_destroy": (_I, [_P]),
    "ebisu_serve_create": (_I, [_SZ, _I, ctypes.POINTER(_P)]),
    "ebisu_serve_submit": (_I, [_P, _P, _P, _P, _I64, ctypes.POINTER(ctypes.c_uint64)]),
    "ebisu_serve_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "ebisu_serve_wait": (_I, [_P, ctypes.c_uint64, _D, ctypes.POINTER(_D)]),
    "ebisu_serve_stats": (_I, [_P, ctypes.POINTER(_I64)]),
    "ebisu_serve_cancel": (_I, [_P, ctypes.c_uint64]),
    "ebisu_serve_set_max_queue": (_I, [_P, _I]),
    "ebisu_serve_set_policy": (_I, [_P, _I, _D]),
    "ebisu_serve_destroy": (_I, [_P]),
    "ebisu_probe_device": (_I, [ctypes.POINTER(_D)]),
}

# test hooks exported by the library but not part of the public header
HOOKS = {
    "ebisu_debug_run_stalled": (_I, [_P, _P, _P, _I64, _P, _P]),
}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in {**SIGNATURES, **HOOKS}.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != OK:
        raise EbisuError(rc, where)


def status_string(code: int) -> str:
    return lib().ebisu_status_string(code).decode()


def last_cuda_error() -> str:
    return lib().ebisu_last_cuda_error().decode()


# ---------------------------------------------------------------------------
# same-name wrappers (raw pointers / ints)

def ebisu_plan_create(ndim, dims, shape, radius, coeffs, dtype, boundary):
    h = _P()
    d = (_I64 * ndim)(*[int(x) for x in dims])
    c = (_D * len(coeffs))(*[float(x) for x in coeffs])
    _check(lib().ebisu_plan_create(ndim, d, shape, radius, c, dtype, boundary, ctypes.byref(h)), "ebisu_plan_create")
    return h


def ebisu_plan_destroy(h):
    _check(lib().ebisu_plan_destroy(h), "ebisu_plan_destroy")


def ebisu_run(h, in_ptr, out_ptr, steps, ws_ptr, stream=0):
    _check(lib().ebisu_run(h, in_ptr, out_ptr, int(steps), ws_ptr, stream), "ebisu_run")


def ebisu_run_naive(h, in_ptr, out_ptr, steps, ws_ptr, stream=0):
    _check(lib().ebisu_run_naive(h, in_ptr, out_ptr, int(steps), ws_ptr, stream), "ebisu_run_naive")


def ebisu_sync(ws_ptr, stream=0):
    return int(lib().ebisu_sync(ws_ptr, stream))


def ebisu_cost_model(**kw):
    """Evaluate the Section 5 model; keyword arguments are ModelIn fields."""
    mi = ModelIn()
    for k, v in kw.items():
        setattr(mi, k, v)
    mo = ModelOut()
    _check(lib().ebisu_cost_model(ctypes.byref(mi), ctypes.byref(mo)), "ebisu_cost_model")
    return {f: getattr(mo, f) for f, _ in ModelOut._fields_ if f != "reserved"}


def ebisu_probe_device():
    out = (_D * 6)()
    _check(lib().ebisu_probe_device(out), "ebisu_probe_device")
    keys = ["f64_flops", "f32_flops", "lds_bytes_per_s", "barrier_s", "sms", "sm_hz"]
    return dict(zip(keys, list(out)))


# ---------------------------------------------------------------------------
# torch-facing convenience layer

def _torch():
    import torch
    return torch


def dtype_code(tdtype) -> int:
    torch = _torch()
    if tdtype == torch.float64:
        return F64
    if tdtype == torch.float32:
        return F32
    if tdtype == torch.bfloat16:
        return BF16
    raise ValueError(f"unsupported dtype {tdtype}")


def torch_dtype(code: int):
    torch = _torch()
    return {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}[code]


def current_stream_handle():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def ebisu_plan_create_offsets(ndim, dims, offsets, coeffs, dtype, boundary):
    h = _P()
    flat = [int(v) for o in offsets for v in o]
    d = (_I64 * ndim)(*[int(x) for x in dims])
    o = (ctypes.c_int32 * len(flat))(*flat)
    c = (_D * len(coeffs))(*[float(x) for x in coeffs])
    _check(lib().ebisu_plan_create_offsets(ndim, d, len(coeffs), o, c, dtype, boundary, ctypes.byref(h)),
           "ebisu_plan_create_offsets")
    return h


class Plan:
    """Owns a plan handle; runs on torch CUDA tensors laid out as the C ABI says."""

    def __init__(self, ndim, dims, shape, radius, coeffs, dtype=F64, boundary=DIRICHLET, offsets=None):
        self.ndim, self.dims, self.shape, self.radius = ndim, tuple(int(d) for d in dims), shape, radius
        self.dtype, self.boundary = dtype, boundary
        self.coeffs = [float(c) for c in coeffs]
        if offsets is None:
            self.h = ebisu_plan_create(ndim, dims, shape, radius, coeffs, dtype, boundary)
        else:
            self.h = ebisu_plan_create_offsets(ndim, dims, offsets, coeffs, dtype, boundary)

    @classmethod
    def from_offsets(cls, ndim, dims, offsets, coeffs, dtype=F64, boundary=DIRICHLET):
        """A plan for an explicit offset list ((dz, dy, dx) triples, one weight each)."""
        r = max(max(abs(v) for v in o) for o in offsets)
        return cls(ndim, dims, None, max(r, 1), coeffs, dtype, boundary, offsets=offsets)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.ebisu_plan_destroy(h)
            self.h = None

    @property
    def pad(self):
        return self.radius if self.boundary == DIRICHLET else 0

    @property
    def stored_shape(self):
        return tuple(d + 2 * self.pad for d in self.dims)

    def workspace_bytes(self) -> int:
        n = _SZ()
        _check(lib().ebisu_plan_workspace_bytes(self.h, ctypes.byref(n)), "ebisu_plan_workspace_bytes")
        return n.value

    def workspace(self):
        torch = _torch()
        return torch.empty(self.workspace_bytes(), dtype=torch.uint8, device="cuda")

    def params(self) -> Params:
        p = Params()
        _check(lib().ebisu_plan_get_params(self.h, ctypes.byref(p)), "ebisu_plan_get_params")
        return p

    def set_params(self, **kw):
        """Update the given fields of the plan's parameters.  Explicit tile
        extents (tile_x / tile_y) describe the shared-memory build, so unless
        `variant` is given too they select it (variant 0)."""
        if "variant" not in kw and ("tile_x" in kw or "tile_y" in kw):
            kw = dict(kw, variant=0)
        p = self.params()
        for k, v in kw.items():
            setattr(p, k, int(v))
        _check(lib().ebisu_plan_set_params(self.h, ctypes.byref(p)), "ebisu_plan_set_params")

    def set_rounding(self, rounding, seed=0):
        """Storage rounding: ROUND_NEAREST or (BF16 only) ROUND_STOCHASTIC."""
        _check(lib().ebisu_plan_set_rounding(self.h, int(rounding), ctypes.c_uint64(int(seed))),
               "ebisu_plan_set_rounding")

    def set_coefficient_field(self, field):
        """Per-cell weights: a CUDA tensor of shape (P,) + stored shape in the
        accumulation type (float64 for F64, float32 for F32/BF16), or None."""
        if field is None:
            self._field = None
            _check(lib().ebisu_plan_set_coefficient_field(self.h, None), "ebisu_plan_set_coefficient_field")
            return
        torch = _torch()
        want = torch.float64 if self.dtype == F64 else torch.float32
        assert field.is_cuda and field.dtype == want and field.is_contiguous()
        assert tuple(field.shape[1:]) == self.stored_shape
        self._field = field  # keep it alive while the plan may read it
        _check(lib().ebisu_plan_set_coefficient_field(self.h, ctypes.c_void_p(field.data_ptr())),
               "ebisu_plan_set_coefficient_field")

    def set_ablation(self, mask):
        """Switch elements of the shared-memory build off (EBISU_ABLATE_* mask)."""
        _check(lib().ebisu_plan_set_ablation(self.h, int(mask)), "ebisu_plan_set_ablation")

    def rounding(self):
        r, sd = _I(), ctypes.c_uint64()
        _check(lib().ebisu_plan_get_rounding(self.h, ctypes.byref(r), ctypes.byref(sd)), "ebisu_plan_get_rounding")
        return r.value, sd.value

    def rs_depths(self):
        """Temporal depths built for the register-streaming kernel (variant 2)."""
        a, b = _I(), _I()
        _check(lib().ebisu_plan_rs_depths(self.h, ctypes.byref(a), ctypes.byref(b)), "ebisu_plan_rs_depths")
        return a.value, b.value

    def model(self):
        pred, bound, valid = _D(), _I(), _D()
        _check(lib().ebisu_plan_model(self.h, ctypes.byref(pred), ctypes.byref(bound), ctypes.byref(valid)),
               "ebisu_plan_model")
        return pred.value, ("gmem", "smem", "fp")[bound.value], valid.value

    def _ptrs(self, x, y, ws):
        torch = _torch()
        assert x.is_cuda and y.is_cuda and ws.is_cuda
        assert tuple(x.shape) == self.stored_shape and tuple(y.shape) == self.stored_shape
        assert x.dtype == torch_dtype(self.dtype) and y.dtype == x.dtype
        assert x.is_contiguous() and y.is_contiguous()
        return ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(ws.data_ptr())

    def run(self, x, y, steps, ws, stream=None, naive=False):
        a, b, w = self._ptrs(x, y, ws)
        s = current_stream_handle() if stream is None else stream
        if naive:
            ebisu_run_naive(self.h, a, b, steps, w, s)
        else:
            ebisu_run(self.h, a, b, steps, w, s)

    def run_stalled(self, x, y, steps, ws):
        a, b, w = self._ptrs(x, y, ws)
        _check(lib().ebisu_debug_run_stalled(self.h, a, b, int(steps), w, current_stream_handle()),
               "ebisu_debug_run_stalled")

    def sync(self, ws, stream=None) -> int:
        s = current_stream_handle() if stream is None else stream
        return ebisu_sync(ctypes.c_void_p(ws.data_ptr()), s)

    def tune(self, x, y, steps, ws, max_candidates=4, share=1.0):
        """Autotune on these buffers; `share` < 1: the plan will share the
        GPU (a batch member), see ebisu_plan_tune_share."""
        a, b, w = self._ptrs(x, y, ws)
        best = _D()
        if share == 1.0:
            rc = lib().ebisu_plan_tune(self.h, a, b, int(steps), w, int(max_candidates), ctypes.byref(best),
                                       current_stream_handle())
        else:
            rc = lib().ebisu_plan_tune_share(self.h, a, b, int(steps), w, int(max_candidates), float(share),
                                             ctypes.byref(best), current_stream_handle())
        _check(rc, "ebisu_plan_tune")
        return best.value

    def reduce(self, a, ws, b=None):
        res = (_D * 3)()
        pa = ctypes.c_void_p(a.data_ptr())
        pb = ctypes.c_void_p(b.data_ptr()) if b is not None else None
        _check(lib().ebisu_reduce(self.h, pa, pb, res, ctypes.c_void_p(ws.data_ptr()), current_stream_handle()),
               "ebisu_reduce")
        return float(res[0]), float(res[1]), float(res[2])


# ---------------------------------------------------------------------------
# batches and serving

def _arr(ctype, vals):
    return (ctype * len(vals))(*vals)


def batch_workspace_bytes(plans, steps) -> int:
    n = len(plans)
    out = _SZ()
    _check(lib().ebisu_batch_workspace_bytes(n, _arr(_P, [p.h for p in plans]), _arr(_I64, [int(s) for s in steps]),
                                             ctypes.byref(out)), "ebisu_batch_workspace_bytes")
    return out.value


def batch_run(plans, xs, ys, steps, ws, stream=None):
    """One persistent launch per kernel type over all problems (tensors)."""
    n = len(plans)
    s = current_stream_handle() if stream is None else stream
    _check(lib().ebisu_batch_run(n, _arr(_P, [p.h for p in plans]), _arr(_P, [x.data_ptr() for x in xs]),
                                 _arr(_P, [y.data_ptr() for y in ys]), _arr(_I64, [int(t) for t in steps]),
                                 ctypes.c_void_p(ws.data_ptr()), s), "ebisu_batch_run")


class Batch:
    """Uploaded work tables; launch() enqueues stream operations only (graph capturable)."""

    def __init__(self, plans, xs, ys, steps, ws, stream=None):
        self.h = _P()
        self.ws = ws
        self._keep = (plans, xs, ys)
        s = current_stream_handle() if stream is None else stream
        _check(lib().ebisu_batch_create(len(plans), _arr(_P, [p.h for p in plans]),
                                        _arr(_P, [x.data_ptr() for x in xs]), _arr(_P, [y.data_ptr() for y in ys]),
                                        _arr(_I64, [int(t) for t in steps]), ctypes.c_void_p(ws.data_ptr()), s,
                                        ctypes.byref(self.h)), "ebisu_batch_create")

    def launch(self, stream=None):
        s = current_stream_handle() if stream is None else stream
        _check(lib().ebisu_batch_launch(self.h, s), "ebisu_batch_launch")

    def sync(self, stream=None) -> int:
        s = current_stream_handle() if stream is None else stream
        return int(lib().ebisu_batch_sync(self.h, s))

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.ebisu_batch_destroy(h)
            self.h = None


class Server:
    """Continuous-batching server (host thread + lanes), see ebisu_serve_*."""

    def __init__(self, hbm_budget: int, max_slots: int = 4):
        self.h = _P()
        _check(lib().ebisu_serve_create(int(hbm_budget), int(max_slots), ctypes.byref(self.h)), "ebisu_serve_create")

    def submit(self, plan, x, y, steps) -> int:
        t = ctypes.c_uint64()
        rc = lib().ebisu_serve_submit(self.h, plan.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      int(steps), ctypes.byref(t))
        _check(rc, "ebisu_serve_submit")
        return t.value

    def try_submit(self, plan, x, y, steps):
        """(status, ticket) without raising: rejected requests return their code."""
        t = ctypes.c_uint64()
        rc = lib().ebisu_serve_submit(self.h, plan.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      int(steps), ctypes.byref(t))
        return rc, t.value

    def poll(self, ticket):
        done, lat = _I(), _D()
        rc = lib().ebisu_serve_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(lat))
        _check(rc, "ebisu_serve_poll")
        return bool(done.value), lat.value

    def wait(self, ticket, timeout_s=120.0) -> float:
        lat = _D()
        _check(lib().ebisu_serve_wait(self.h, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(lat)),
               "ebisu_serve_wait")
        return lat.value

    def set_max_queue(self, n: int):
        _check(lib().ebisu_serve_set_max_queue(self.h, int(n)), "ebisu_serve_set_max_queue")

    def set_policy(self, order: int, max_wait_s: float = 0.0):
        _check(lib().ebisu_serve_set_policy(self.h, int(order), float(max_wait_s)), "ebisu_serve_set_policy")

    def cancel(self, ticket) -> int:
        return int(lib().ebisu_serve_cancel(self.h, ctypes.c_uint64(ticket)))

    def stats(self):
        a = (_I64 * 7)()
        _check(lib().ebisu_serve_stats(self.h, a), "ebisu_serve_stats")
        keys = ["submitted", "completed", "rejected", "queued", "running", "peak_bytes", "held_bytes"]
        return dict(zip(keys, list(a)))

    def close(self):
        if self.h is not None and _lib is not None:
            _check(_lib.ebisu_serve_destroy(self.h), "ebisu_serve_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
