"""Plain CPU oracle for Jacobi-style iterative stencils (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The library never does: the two
share no code, and the oracle does not import the library either.

The arithmetic lives in ``oracle.c`` (plain FP64 loops, one full sweep per
time step, Section 2.1 / Listings 1-3 of the paper).  This module only loads
the compiled C file through ctypes and marshals numpy arrays.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
against brute force (dense operator powers), invariants and the closed-form
Fourier-mode decay; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

STAR, BOX, POISSON, J3D17 = 0, 1, 2, 3
DIRICHLET, PERIODIC = 0, 1

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP, no FMA
    contraction so that every term is a separate multiply and add)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_offsets.restype = ctypes.c_int
        lib.oracle_offsets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_run.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        lib.oracle_run_offsets.restype = ctypes.c_int
        lib.oracle_run_offsets.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        lib.oracle_run_varcoef.restype = ctypes.c_int
        lib.oracle_run_varcoef.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int64]
        lib.oracle_reduce.restype = ctypes.c_int
        lib.oracle_reduce.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        _lib = lib
    return _lib


def offsets(ndim: int, shape: int, radius: int) -> np.ndarray:
    """Canonical offsets as an (npts, 3) int array of (dz, dy, dx)."""
    lib = _load()
    n = lib.oracle_offsets(ndim, shape, radius, None, None, None)
    if n < 0:
        raise ValueError("bad stencil description")
    dz = np.zeros(n, np.int32)
    dy = np.zeros(n, np.int32)
    dx = np.zeros(n, np.int32)
    lib.oracle_offsets(ndim, shape, radius, dz.ctypes.data, dy.ctypes.data, dx.ctypes.data)
    return np.stack([dz, dy, dx], axis=1)


def npoints(ndim: int, shape: int, radius: int) -> int:
    return int(_load().oracle_offsets(ndim, shape, radius, None, None, None))


def run(grid: np.ndarray, shape: int, radius: int, coeffs, boundary: int,
        steps: int, nthreads: int = 0) -> np.ndarray:
    """Run `steps` Jacobi steps on a stored grid (padded by `radius` for
    Dirichlet, unpadded for periodic) and return the new stored grid."""
    lib = _load()
    g = np.ascontiguousarray(grid, dtype=np.float64)
    ndim = g.ndim
    pad = radius if boundary == DIRICHLET else 0
    dims = (ctypes.c_int64 * ndim)(*[s - 2 * pad for s in g.shape])
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    if c.size != npoints(ndim, shape, radius):
        raise ValueError("coefficient count does not match the stencil")
    out = np.empty_like(g)
    rc = lib.oracle_run(ndim, dims, shape, radius,
                        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), boundary,
                        g.ctypes.data, out.ctypes.data, int(steps), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_run failed ({rc})")
    return out


def run_offsets(grid: np.ndarray, offsets, radius: int, coeffs, boundary: int, steps: int,
                nthreads: int = 0) -> np.ndarray:
    """`steps` Jacobi steps with an explicit offset list: `offsets` is a
    sequence of (dz, dy, dx) triples (dz = 0 in 2D), summed in the order
    given; `radius` is the pad width (Dirichlet) and bounds every offset."""
    lib = _load()
    g = np.ascontiguousarray(grid, dtype=np.float64)
    o = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 3))
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    if c.size != o.shape[0]:
        raise ValueError("one coefficient per offset")
    pad = radius if boundary == DIRICHLET else 0
    dims = (ctypes.c_int64 * g.ndim)(*[s - 2 * pad for s in g.shape])
    oz, oy, ox = (np.ascontiguousarray(o[:, i]) for i in range(3))
    out = np.empty_like(g)
    rc = lib.oracle_run_offsets(g.ndim, dims, radius, int(o.shape[0]), oz.ctypes.data, oy.ctypes.data,
                                ox.ctypes.data, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), boundary,
                                g.ctypes.data, out.ctypes.data, int(steps), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_run_offsets failed ({rc})")
    return out


def run_varcoef(grid: np.ndarray, shape: int, radius: int, field: np.ndarray, boundary: int,
                steps: int) -> np.ndarray:
    """Jacobi steps with per-cell weights: `field` has shape (npts,) +
    grid.shape, entry [k][x] the weight of offset k (canonical order) at
    cell x (pad entries unused).  Single-threaded plain loops."""
    lib = _load()
    g = np.ascontiguousarray(grid, dtype=np.float64)
    f = np.ascontiguousarray(field, dtype=np.float64)
    if f.shape != (npoints(g.ndim, shape, radius),) + g.shape:
        raise ValueError("field must hold one array per offset, shaped like the grid")
    pad = radius if boundary == DIRICHLET else 0
    dims = (ctypes.c_int64 * g.ndim)(*[s - 2 * pad for s in g.shape])
    out = np.empty_like(g)
    rc = lib.oracle_run_varcoef(g.ndim, dims, shape, radius, f.ctypes.data, boundary, g.ctypes.data,
                                out.ctypes.data, int(steps))
    if rc != 0:
        raise ValueError(f"oracle_run_varcoef failed ({rc})")
    return out


def reduce(grid: np.ndarray, pad: int, other: np.ndarray | None = None):
    """(sum, L2 norm, max |.|) over the interior, of `grid` or `grid - other`."""
    lib = _load()
    g = np.ascontiguousarray(grid, dtype=np.float64)
    dims = (ctypes.c_int64 * g.ndim)(*[s - 2 * pad for s in g.shape])
    res = (ctypes.c_double * 3)()
    o = None
    if other is not None:
        o = np.ascontiguousarray(other, dtype=np.float64)
    rc = lib.oracle_reduce(g.ndim, dims, pad, g.ctypes.data,
                           None if o is None else o.ctypes.data, res)
    if rc != 0:
        raise ValueError("oracle_reduce failed")
    return float(res[0]), float(res[1]), float(res[2])


def rel_linf(a: np.ndarray, ref: np.ndarray, pad: int) -> float:
    """max |a - ref| / max |ref| over the interior (the parity metric)."""
    _, _, num = reduce(a, pad, ref)
    _, _, den = reduce(ref, pad)
    return num / den if den > 0 else num
