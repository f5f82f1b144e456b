"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Nothing here compares the oracle with itself or with the CUDA path.  The pins:
  * Listings 1-3 written out term by term with numpy slices (2d5pt, 3d7pt, and
    the 1D 3-point special case);
  * brute force: the dense one-step operator built from an independently
    constructed offset set, raised to the T-th power, on 8x8 / 6^3 grids;
  * the closed-form Fourier-mode decay lambda(k)^T under periodic boundaries,
    with non-symmetric coefficients (fixes offset signs and axis order);
  * invariants: constant fields (sum c = 1), linear fields (symmetric c),
    mass conservation (periodic), the Dirichlet pad never changes;
  * mutation checks: three plausible mistakes planted in a copy of the oracle
    source (a dropped term, a flipped x offset, swapped axes) each fail a pin.
"""
import cmath
import ctypes
import itertools
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2305_07390_gb300 import synth

EPS = np.finfo(np.float64).eps

SHAPES_2D = [(synth.STAR, 1), (synth.STAR, 2), (synth.STAR, 3), (synth.BOX, 1), (synth.BOX, 2)]
SHAPES_3D = [(synth.STAR, 1), (synth.STAR, 2), (synth.STAR, 3), (synth.BOX, 1), (synth.BOX, 2),
             (synth.POISSON, 1), (synth.J3D17, 1)]


def independent_offsets(ndim, shape, r):
    """Offset set built from its definition, sorted as (dz, dy, dx) tuples.
    Poisson: the 27-point box without its corners (Table 2: 19 points, 38
    flops); j3d17pt (17 points, 34 flops): the reading of that set -- the
    3x3 box of the z = 0 plane plus the 4 axis neighbours in each of the
    planes z = -1 and z = +1."""
    rng = range(-r, r + 1)
    if ndim == 2:
        pts = [(0, a, b) for a, b in itertools.product(rng, rng)]
    else:
        pts = list(itertools.product(rng, rng, rng))
    if shape == synth.STAR:
        pts = [p for p in pts if sum(1 for v in p if v != 0) <= 1]
    if shape == synth.POISSON:
        pts = [p for p in pts if not all(v != 0 for v in p)]
    if shape == synth.J3D17:
        pts = [p for p in pts if p[0] == 0 or (p[1] != 0) != (p[2] != 0)]
    return sorted(pts)


# --------------------------------------------------------------------------
# offsets


@pytest.mark.parametrize("ndim,shape,r,npts", [
    (2, synth.STAR, 1, 5), (2, synth.STAR, 2, 9), (2, synth.STAR, 3, 13),
    (2, synth.BOX, 1, 9), (2, synth.BOX, 2, 25),
    (3, synth.STAR, 1, 7), (3, synth.STAR, 2, 13), (3, synth.BOX, 1, 27), (3, synth.BOX, 2, 125),
    (3, synth.POISSON, 1, 19), (3, synth.J3D17, 1, 17)])
def test_offset_counts_match_table3(ndim, shape, r, npts):
    # Table 2 (benchmarks): j2d5pt, j2d9pt, 2D r3 star, j2d9pt-gol, j2d25pt,
    # j3d7pt, j3d13pt, j3d27pt, the 125-point box, poisson (order 1, 38
    # flops per cell = 19 points) and j3d17pt (order 1, 34 flops = 17).
    offs = oracle.offsets(ndim, shape, r)
    assert offs.shape == (npts, 3)
    assert [tuple(o) for o in offs] == independent_offsets(ndim, shape, r)
    assert npts == synth.npoints(ndim, shape, r)


# --------------------------------------------------------------------------
# Listings written out


def test_listing2_2d5pt_expansion():
    rng = np.random.default_rng(1)
    g = rng.random((10, 12))
    a, b, c, d, e = rng.random(5)
    # canonical order (dy,dx): (-1,0)=a, (0,-1)=d, (0,0)=b, (0,1)=e, (1,0)=c
    coeffs = [a, d, b, e, c]
    out = oracle.run(g, synth.STAR, 1, coeffs, synth.DIRICHLET, 1)
    ref = g.copy()
    inn = g
    ref[1:-1, 1:-1] = (a * inn[:-2, 1:-1] + b * inn[1:-1, 1:-1] + c * inn[2:, 1:-1]
                       + d * inn[1:-1, :-2] + e * inn[1:-1, 2:])
    np.testing.assert_allclose(out, ref, rtol=4 * EPS, atol=4 * EPS)


def test_listing3_3d7pt_expansion():
    rng = np.random.default_rng(2)
    g = rng.random((7, 8, 9))
    a, b, c, d, e, f, h = rng.random(7)
    # Listing 3: i = z (slowest), j = y, k = x.
    # canonical (dz,dy,dx): (-1,0,0)=a, (0,-1,0)=d, (0,0,-1)=f, (0,0,0)=b,
    # (0,0,1)=h, (0,1,0)=e, (1,0,0)=c
    coeffs = [a, d, f, b, h, e, c]
    out = oracle.run(g, synth.STAR, 1, coeffs, synth.DIRICHLET, 1)
    ref = g.copy()
    s = slice(1, -1)
    ref[s, s, s] = (a * g[:-2, s, s] + b * g[s, s, s] + c * g[2:, s, s]
                    + d * g[s, :-2, s] + e * g[s, 2:, s]
                    + f * g[s, s, :-2] + h * g[s, s, 2:])
    np.testing.assert_allclose(out, ref, rtol=8 * EPS, atol=8 * EPS)


def test_new_sets_symmetry_and_flops():
    # 2 flops per point: Table 2's 38 (poisson) and 34 (j3d17pt)
    assert 2 * oracle.npoints(3, synth.POISSON, 1) == 38
    assert 2 * oracle.npoints(3, synth.J3D17, 1) == 34
    for shape in (synth.POISSON, synth.J3D17):
        pts = {tuple(o) for o in oracle.offsets(3, shape, 1)}
        assert all(max(abs(v) for v in p) <= 1 for p in pts)          # order 1
        assert {tuple(-v for v in p) for p in pts} == pts              # point symmetric
        assert {(p[0], p[2], p[1]) for p in pts} == pts                # y <-> x
    pois = {tuple(o) for o in oracle.offsets(3, synth.POISSON, 1)}
    perms = itertools.permutations(range(3))
    assert all({tuple(p[i] for i in pm) for p in pois} == pois for pm in perms)  # every axis alike
    j17 = {tuple(o) for o in oracle.offsets(3, synth.J3D17, 1)}
    assert j17 == pois - {(-1, 0, 0), (1, 0, 0)}


def test_poisson_with_star_weights_is_the_7_point_star():
    g, c7 = synth.problem(3, (7, 6, 8), synth.STAR, 1, synth.DIRICHLET, seed=14)
    offs = [tuple(o) for o in oracle.offsets(3, synth.POISSON, 1)]
    star = [tuple(o) for o in oracle.offsets(3, synth.STAR, 1)]
    c19 = [c7[star.index(o)] if o in star else 0.0 for o in offs]
    np.testing.assert_array_equal(oracle.run(g, synth.POISSON, 1, c19, synth.DIRICHLET, 4),
                                  oracle.run(g, synth.STAR, 1, c7, synth.DIRICHLET, 4))


def test_j3d17_with_in_plane_weights_is_a_2d_box_per_plane():
    rng = np.random.default_rng(15)
    g = rng.random((6, 9, 10))
    offs = [tuple(o) for o in oracle.offsets(3, synth.J3D17, 1)]
    box = [(0, a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)]
    w = rng.random(9)
    c17 = [w[box.index(o)] if o in box else 0.0 for o in offs]
    out = oracle.run(g, synth.J3D17, 1, c17, synth.DIRICHLET, 3)
    for z in range(1, 5):
        np.testing.assert_allclose(out[z], oracle.run(g[z], synth.BOX, 1, w, synth.DIRICHLET, 3),
                                   rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("boundary", [synth.DIRICHLET, synth.PERIODIC])
@pytest.mark.parametrize("ndim", [2, 3])
def test_offset_list_bruteforce(ndim, boundary):
    # an arbitrary, asymmetric offset list inside the radius-2 box
    rng = np.random.default_rng(16 + ndim)
    full = independent_offsets(ndim, synth.BOX, 2)
    pick = sorted(full[i] for i in rng.choice(len(full), 11, replace=False))
    c = rng.random(11)
    c /= c.sum()
    dims = (9, 8) if ndim == 2 else (5, 5, 6)
    g = synth.grid(dims, 2, boundary, seed=17)
    M = dense_operator(g.shape, pick, c, 2, boundary)
    for T in (1, 3):
        out = oracle.run_offsets(g, pick, 2, c, boundary, T)
        ref = (np.linalg.matrix_power(M, T) @ g.ravel()).reshape(g.shape)
        np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-14)


def dense_operator_varcoef(stored_shape, offs, field, r, boundary):
    """Matrix M with u_s = M u_{s-1}: row i holds cell i's own weights."""
    shp = stored_shape
    ndim = len(shp)
    N = int(np.prod(shp))
    M = np.zeros((N, N))
    pad = r if boundary == synth.DIRICHLET else 0
    for idx in itertools.product(*[range(s) for s in shp]):
        i = np.ravel_multi_index(idx, shp)
        if not all(pad <= v < s - pad for v, s in zip(idx, shp)):
            M[i, i] = 1.0
            continue
        for k, (dz, dy, dx) in enumerate(offs):
            d = (dy, dx) if ndim == 2 else (dz, dy, dx)
            nb = tuple(v + o for v, o in zip(idx, d))
            if boundary == synth.PERIODIC:
                nb = tuple(v % s for v, s in zip(nb, shp))
            M[i, np.ravel_multi_index(nb, shp)] += field[k][idx]
    return M


@pytest.mark.parametrize("boundary", [synth.DIRICHLET, synth.PERIODIC])
@pytest.mark.parametrize("ndim,shape,r", [(2, synth.STAR, 1), (2, synth.BOX, 2), (3, synth.STAR, 1)])
def test_varcoef_bruteforce(ndim, shape, r, boundary):
    rng = np.random.default_rng(30 + ndim + r)
    dims = (8, 7) if ndim == 2 else (5, 4, 6)
    g = synth.grid(dims, r, boundary, seed=31)
    offs = independent_offsets(ndim, shape, r)
    field = rng.random((len(offs),) + g.shape)
    M = dense_operator_varcoef(g.shape, offs, field, r, boundary)
    for T in (1, 3):
        out = oracle.run_varcoef(g, shape, r, field, boundary, T)
        ref = (np.linalg.matrix_power(M, T) @ g.ravel()).reshape(g.shape)
        np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-14)


def test_varcoef_with_uniform_weights_is_the_fixed_stencil():
    g, c = synth.problem(2, (20, 17), synth.BOX, 1, synth.DIRICHLET, seed=32)
    field = np.broadcast_to(c[:, None, None], (len(c),) + g.shape).copy()
    np.testing.assert_array_equal(oracle.run_varcoef(g, synth.BOX, 1, field, synth.DIRICHLET, 5),
                                  oracle.run(g, synth.BOX, 1, c, synth.DIRICHLET, 5, nthreads=1))


def test_varcoef_rows_summing_to_one_keep_a_constant_field():
    rng = np.random.default_rng(33)
    dims = (9, 8, 7)
    w = rng.random((13,) + synth.stored_shape(dims, 2, synth.DIRICHLET))
    w /= w.sum(axis=0, keepdims=True)
    g = np.full(synth.stored_shape(dims, 2, synth.DIRICHLET), 0.625)
    out = oracle.run_varcoef(g, synth.STAR, 2, w, synth.DIRICHLET, 6)
    assert np.max(np.abs(out - 0.625)) <= 6 * 13 * EPS


def test_listing1_1d_special_case():
    # A 2D 5-point star with zero north/south weights is one independent
    # 1D 3-point stencil per row (Listing 1), with fixed end cells.
    rng = np.random.default_rng(3)
    g = rng.random((9, 20))
    a, b, c = 0.3, 0.5, 0.2
    T = 6
    out = oracle.run(g, synth.STAR, 1, [0.0, a, b, c, 0.0], synth.DIRICHLET, T)
    for row in range(1, 8):
        u = g[row].copy()
        for _ in range(T):
            v = u.copy()
            v[1:-1] = a * u[:-2] + b * u[1:-1] + c * u[2:]
            u = v
        np.testing.assert_allclose(out[row], u, rtol=1e-14, atol=1e-14)


# --------------------------------------------------------------------------
# brute force: dense operator powers


def dense_operator(stored_shape, offs, coeffs, r, boundary):
    """Matrix M with u_{s} = M u_{s-1} over the whole stored grid."""
    shp = stored_shape
    ndim = len(shp)
    N = int(np.prod(shp))
    M = np.zeros((N, N))
    pad = r if boundary == synth.DIRICHLET else 0
    for idx in itertools.product(*[range(s) for s in shp]):
        i = np.ravel_multi_index(idx, shp)
        interior = all(pad <= v < s - pad for v, s in zip(idx, shp))
        if not interior:
            M[i, i] = 1.0
            continue
        for (dz, dy, dx), ck in zip(offs, coeffs):
            d = (dy, dx) if ndim == 2 else (dz, dy, dx)
            nb = tuple(v + o for v, o in zip(idx, d))
            if boundary == synth.PERIODIC:
                nb = tuple(v % s for v, s in zip(nb, shp))
            M[i, np.ravel_multi_index(nb, shp)] += ck
    return M


@pytest.mark.parametrize("boundary", [synth.DIRICHLET, synth.PERIODIC])
@pytest.mark.parametrize("shape,r", SHAPES_2D)
def test_bruteforce_2d(shape, r, boundary):
    dims = (8, 8)
    g, c = synth.problem(2, dims, shape, r, boundary, seed=11 + r)
    offs = independent_offsets(2, shape, r)
    M = dense_operator(g.shape, offs, c, r, boundary)
    for T in (1, 3):
        out = oracle.run(g, shape, r, c, boundary, T)
        ref = (np.linalg.matrix_power(M, T) @ g.ravel()).reshape(g.shape)
        np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("boundary", [synth.DIRICHLET, synth.PERIODIC])
@pytest.mark.parametrize("shape,r", SHAPES_3D)
def test_bruteforce_3d(shape, r, boundary):
    dims = (6, 6, 6) if (boundary == synth.DIRICHLET or r < 3) else (7, 7, 7)
    if boundary == synth.DIRICHLET and r >= 2:
        dims = (5, 4, 6)
    g, c = synth.problem(3, dims, shape, r, boundary, seed=21 + r)
    offs = independent_offsets(3, shape, r)
    M = dense_operator(g.shape, offs, c, r, boundary)
    for T in (1, 3):
        out = oracle.run(g, shape, r, c, boundary, T)
        ref = (np.linalg.matrix_power(M, T) @ g.ravel()).reshape(g.shape)
        np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-14)


# --------------------------------------------------------------------------
# closed form: Fourier-mode decay under periodic boundaries


def fourier_check(run, ndim, shape, r, dims, k, T, seed):
    c = synth.coefficients(ndim, shape, r, dims, synth.PERIODIC, seed=seed)
    offs = independent_offsets(ndim, shape, r)
    lam = 0j
    for (dz, dy, dx), ck in zip(offs, c):
        o = (dy, dx) if ndim == 2 else (dz, dy, dx)
        lam += ck * cmath.exp(2j * math.pi * sum(kd * od / nd for kd, od, nd in zip(k, o, dims)))
    # as many steps as keep the mode above 1e-3 of its start (at most T)
    if abs(lam) < 1.0:
        T = max(1, min(T, int(math.log(1e-3) / math.log(abs(lam)))))
    u0 = synth.cosine_mode(dims, k)
    out = run(u0, shape, r, c, synth.PERIODIC, T)
    axes = [np.arange(n, dtype=np.float64) for n in dims]
    mesh = np.meshgrid(*axes, indexing="ij")
    phase = sum(2.0 * math.pi * kd * xd / nd for kd, xd, nd in zip(k, mesh, dims))
    ref = np.real(lam ** T * np.exp(1j * phase))
    assert abs(lam) ** T > 1e-3
    return float(np.max(np.abs(out - ref)))


@pytest.mark.parametrize("shape,r", SHAPES_2D)
@pytest.mark.parametrize("k", [(1, 2), (3, 1)])
def test_fourier_decay_2d(shape, r, k):
    err = fourier_check(oracle.run, 2, shape, r, (24, 20), k, 12, seed=5)
    assert err < 1e-12


@pytest.mark.parametrize("shape,r", SHAPES_3D[:2] + SHAPES_3D[3:])
@pytest.mark.parametrize("k", [(1, 1, 1), (2, 1, 3)])
def test_fourier_decay_3d(shape, r, k):
    err = fourier_check(oracle.run, 3, shape, r, (12, 10, 14), k, 5, seed=6)
    assert err < 1e-12


# --------------------------------------------------------------------------
# invariants


@pytest.mark.parametrize("ndim,shape,r", [(2, s, r) for s, r in SHAPES_2D] + [(3, s, r) for s, r in SHAPES_3D])
def test_constant_field_preserved(ndim, shape, r):
    dims = (17, 13) if ndim == 2 else (7, 9, 8)
    c = synth.coefficients(ndim, shape, r, dims, synth.DIRICHLET, seed=8)
    g = np.full(synth.stored_shape(dims, r, synth.DIRICHLET), 0.75)
    T = 10
    out = oracle.run(g, shape, r, c, synth.DIRICHLET, T)
    P = len(c)
    assert np.max(np.abs(out - 0.75)) <= T * P * EPS


@pytest.mark.parametrize("ndim,shape,r", [(2, synth.STAR, 1), (2, synth.BOX, 2), (3, synth.STAR, 2), (3, synth.BOX, 1)])
def test_linear_field_preserved_by_symmetric_stencil(ndim, shape, r):
    dims = (15, 11) if ndim == 2 else (6, 7, 8)
    offs = independent_offsets(ndim, shape, r)
    # symmetric weights: c(o) = c(-o), summing to 1
    raw = synth.uniform_open01(9, 0, len(offs))
    w = {}
    for o, v in zip(offs, raw):
        key = min(o, tuple(-x for x in o))
        w.setdefault(key, v)
    c = np.array([w[min(o, tuple(-x for x in o))] for o in offs])
    c = c / c.sum()
    if ndim == 2 and shape == synth.STAR and r == 1:
        c = synth.config1_coefficients()
    shp = synth.stored_shape(dims, r, synth.DIRICHLET)
    mesh = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shp], indexing="ij")
    g = 0.25 + sum(0.01 * (d + 1) * m for d, m in enumerate(mesh))
    out = oracle.run(g, shape, r, c, synth.DIRICHLET, 7)
    np.testing.assert_allclose(out, g, rtol=0, atol=1e-13)


@pytest.mark.parametrize("ndim,shape,r", [(2, synth.STAR, 2), (2, synth.BOX, 1), (3, synth.STAR, 1), (3, synth.BOX, 2)])
def test_mass_conserved_periodic(ndim, shape, r):
    dims = (19, 23) if ndim == 2 else (9, 8, 10)
    g, c = synth.problem(ndim, dims, shape, r, synth.PERIODIC, seed=10)
    out = oracle.run(g, shape, r, c, synth.PERIODIC, 9)
    assert abs(math.fsum(out.ravel()) - math.fsum(g.ravel())) <= 1e-12 * math.fsum(g.ravel())


def test_dirichlet_pad_unchanged_and_steps_compose():
    g, c = synth.problem(2, (21, 18), synth.BOX, 2, synth.DIRICHLET, seed=12)
    out5 = oracle.run(g, synth.BOX, 2, c, synth.DIRICHLET, 5)
    mask = np.ones(g.shape, bool)
    mask[2:-2, 2:-2] = False
    assert np.array_equal(out5[mask], g[mask])
    out2 = oracle.run(g, synth.BOX, 2, c, synth.DIRICHLET, 2)
    out23 = oracle.run(out2, synth.BOX, 2, c, synth.DIRICHLET, 3)
    assert np.array_equal(out5, out23)
    assert np.array_equal(oracle.run(g, synth.BOX, 2, c, synth.DIRICHLET, 0), g)


def test_reductions_against_exact_sums():
    rng = np.random.default_rng(13)
    g = rng.standard_normal((40, 50))
    h = rng.standard_normal((40, 50))
    inner = g[3:-3, 3:-3]
    s, l2, linf = oracle.reduce(g, 3)
    assert abs(s - math.fsum(inner.ravel())) <= 1e-15 * np.abs(inner).sum()
    assert abs(l2 - math.sqrt(math.fsum((inner * inner).ravel()))) <= 1e-14 * l2
    assert linf == np.max(np.abs(inner))
    _, _, dinf = oracle.reduce(g, 3, h)
    assert dinf == np.max(np.abs(inner - h[3:-3, 3:-3]))


# --------------------------------------------------------------------------
# planted mistakes: every pin set above must be able to fail


MUTANTS = {
    "dropped_term": ("for (int k = 0; k < npts; k++) {", "for (int k = 0; k < npts - 1; k++) {"),
    "flipped_dx": ("xx = wrap(x + ox[k], n[2]);", "xx = wrap(x - ox[k], n[2]);"),
    "swapped_axes": ("yy = wrap(y + oy[k], n[1]);\n                        xx = wrap(x + ox[k], n[2]);",
                     "yy = wrap(y + ox[k], n[1]);\n                        xx = wrap(x + oy[k], n[2]);"),
}


def _mutant_runner(tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(path), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_run.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]

    def run(grid, shape, r, coeffs, boundary, steps):
        g = np.ascontiguousarray(grid, dtype=np.float64)
        pad = r if boundary == synth.DIRICHLET else 0
        dims = (ctypes.c_int64 * g.ndim)(*[s - 2 * pad for s in g.shape])
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        out = np.empty_like(g)
        rc = lib.oracle_run(g.ndim, dims, shape, r, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            boundary, g.ctypes.data, out.ctypes.data, steps, 1)
        assert rc == 0
        return out
    return run


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_are_caught(tmp_path, name):
    run = _mutant_runner(tmp_path, name)
    err = fourier_check(run, 2, synth.BOX, 1, (24, 20), (1, 2), 12, seed=5)
    assert err > 1e-6, f"mutant {name} passed the Fourier pin"
