"""Seeded synthetic inputs shared by the library's tests, benchmark and oracle checks.

This module holds no stencil arithmetic: it only draws numbers.  The paper's
own inputs (grids "generated by STENCILGEN", Section 7) are not available, so
these generators stand in for them with the same structure: dense grids of
uniform values and fixed coefficient sets (the shapes of Table 2), plus the size and
arrival mixes used by the batched and served workloads.

Random stream: SplitMix64 seeded with `seed`; the i-th draw (i = 0, 1, ...) is
    z = seed + (i + 1) * 0x9E3779B97F4A7C15   (mod 2^64), then the SplitMix64
    finaliser; a double in [0, 1) is (z >> 11) * 2^-53.
One stream per problem: the padded grid first (row-major), then the
coefficients.  Open-interval draws for coefficients use ((z >> 11) + 0.5) * 2^-53.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20230521

STAR, BOX, POISSON, J3D17 = 0, 1, 2, 3
DIRICHLET, PERIODIC = 0, 1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream, as uint64."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1)."""
    z = splitmix64(seed, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_open01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in (0, 1)."""
    z = splitmix64(seed, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def npoints(ndim: int, shape: int, radius: int) -> int:
    """Number of support points (a count only; offsets are not built here)."""
    if shape == STAR:
        return 2 * ndim * radius + 1
    if shape == POISSON:
        return 19
    if shape == J3D17:
        return 17
    return (2 * radius + 1) ** ndim


def stored_shape(dims, radius: int, boundary: int):
    pad = radius if boundary == DIRICHLET else 0
    return tuple(int(d) + 2 * pad for d in dims)


def grid(dims, radius: int, boundary: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Stored grid (padded by `radius` for Dirichlet) of uniform [0,1) values,
    drawn first from the problem's stream."""
    shp = stored_shape(dims, radius, boundary)
    n = int(np.prod(shp))
    return uniform01(seed, 0, n).reshape(shp)


def coefficients(ndim: int, shape: int, radius: int, dims, boundary: int,
                 seed: int = DEFAULT_SEED) -> np.ndarray:
    """Per-offset weights uniform in (0,1), divided by their FP64 sum; drawn
    from the same stream right after the grid."""
    shp = stored_shape(dims, radius, boundary)
    start = int(np.prod(shp))
    c = uniform_open01(seed, start, npoints(ndim, shape, radius))
    return c / c.sum()


def config1_coefficients() -> np.ndarray:
    """2D 5-point star with centre 0.5 and 0.125 on each of N, S, E, W, in the
    canonical (dy, dx) order (-1,0), (0,-1), (0,0), (0,1), (1,0)."""
    return np.array([0.125, 0.125, 0.5, 0.125, 0.125])


def problem(ndim, dims, shape, radius, boundary=DIRICHLET, seed=DEFAULT_SEED):
    """(stored grid, coefficients) for one seeded problem."""
    return (grid(dims, radius, boundary, seed),
            coefficients(ndim, shape, radius, dims, boundary, seed))


def cosine_mode(dims, k) -> np.ndarray:
    """cos(2*pi*sum_d k_d x_d / n_d) on an unpadded periodic grid."""
    axes = [np.arange(n, dtype=np.float64) for n in dims]
    mesh = np.meshgrid(*axes, indexing="ij")
    phase = sum(2.0 * math.pi * kd * xd / nd for kd, xd, nd in zip(k, mesh, dims))
    return np.cos(phase)


def batch_mix(count: int = 512, seed: int = DEFAULT_SEED):
    """Sizes and step counts of the uneven batch: n_x log-uniform in
    [256, 4096], aspect log-uniform in [0.25, 4], n_y = clamp(round(n_x * a),
    256, 4096), steps uniform in {16 .. 512}.  Returns a list of (ny, nx, steps)."""
    u = uniform01(seed ^ 0xB47C, 0, 3 * count).reshape(count, 3)
    out = []
    for a, b, c in u:
        nx = int(round(math.exp(math.log(256) + a * (math.log(4096) - math.log(256)))))
        asp = math.exp(math.log(0.25) + b * (math.log(4.0) - math.log(0.25)))
        ny = int(min(4096, max(256, round(nx * asp))))
        steps = 16 + int(c * (512 - 16 + 1))
        out.append((ny, nx, min(steps, 512)))
    return out


def serve_mix(rate_hz: float, duration_s: float, seed: int = DEFAULT_SEED):
    """Open-loop Poisson arrivals with the served request mix: half 2D (side
    log-uniform in [256, 8192], 5-point star or 9-point box), half 3D (side
    log-uniform in [64, 512], 7-point star or 27-point box); FP64/FP32 50/50;
    steps log-uniform in [10, 1000].  Returns a list of dicts sorted by arrival
    time."""
    n_max = int(rate_hz * duration_s * 2 + 64)
    u = uniform01(seed ^ (int(rate_hz) << 8), 0, 6 * n_max).reshape(n_max, 6)
    t = 0.0
    reqs = []
    for row in u:
        t += -math.log(1.0 - row[0]) / rate_hz
        if t >= duration_s:
            break
        if row[1] < 0.5:
            ndim = 2
            side = int(round(math.exp(math.log(256) + row[2] * (math.log(8192) - math.log(256)))))
            shape = STAR if row[3] < 0.5 else BOX
        else:
            ndim = 3
            side = int(round(math.exp(math.log(64) + row[2] * (math.log(512) - math.log(64)))))
            shape = STAR if row[3] < 0.5 else BOX
        dtype = "f64" if row[4] < 0.5 else "f32"
        steps = int(round(math.exp(math.log(10) + row[5] * (math.log(1000) - math.log(10)))))
        reqs.append(dict(t=t, ndim=ndim, dims=(side,) * ndim, shape=shape, radius=1,
                         dtype=dtype, steps=steps))
    return reqs
