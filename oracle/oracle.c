/*
 * oracle.c -- plain, slow CPU reference for Jacobi-style iterative stencils.
 *
 * TEST INFRASTRUCTURE ONLY.  The library never links, loads or calls this
 * file; only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes.  The paper's stencils (Section 2.1, Listings 1-3, and the
 * benchmark list of Table 2) are Jacobi updates: every interior cell of the new
 * time level is a fixed weighted sum of the previous level at fixed offsets,
 *
 *     u_s(x) = sum_k c_k * u_{s-1}(x + o_k),      s = 1 .. T.
 *
 * Temporal blocking (Sections 2.1.2, 3 and 4) only reorders these updates, so
 * the plain definition is the oracle: two full arrays, one loop nest per time
 * step, swap.  FP64 throughout.  The sum is taken in canonical offset order,
 * term by term, with a separate multiply and add (this file is compiled with
 * -ffp-contract=off so that no compiler fuses them).
 *
 * Readings of points the paper leaves open (the paper states no boundary rule
 * and no coefficient values):
 *   - Canonical offsets: the support set sorted lexicographically by
 *     (dz, dy, dx).  Star = the centre plus the axis offsets with |k| <= r;
 *     box = every offset with max|k| <= r.
 *   - Table 2 lists two more 3D order-1 stencils without their offsets:
 *     poisson [order 1, 38 flops: 19 points] and j3d17pt [order 1, 34 flops:
 *     17 points], both within the 27-point box (the paper runs its
 *     comparison systems' 27-point code for them).  Poisson = the box without
 *     its 8 corners (offsets with at most two nonzero components).  No
 *     17-point subset of the box has the cube's full symmetry; the reading
 *     here is the poisson set without the two z-axis neighbours (0,0,+-1):
 *     the full 3x3 box in the z = 0 plane plus the four in-plane axis
 *     neighbours (dy,dx) = (+-1,0), (0,+-1) in each of the planes z = +-1.
 *   - Any other offset set runs through oracle_run_offsets.
 *   - Dirichlet: the array is padded by r cells on every side; the pad holds
 *     its initial values for every step (it is read, never written).
 *   - Periodic: the array is not padded; neighbour indices wrap modulo n.
 *   - Layout: row-major, x fastest; 2D arrays are (y, x), 3D arrays (z, y, x).
 *
 * Entry points return 0 on success and a negative value on a bad argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_STAR 0
#define OR_BOX 1
#define OR_POISSON 2
#define OR_J3D17 3
#define OR_DIRICHLET 0
#define OR_PERIODIC 1

/* Offsets of the support set, canonical order.  Writes npts triples into
 * dz/dy/dx (each may be NULL to only count) and returns npts, or -1. */
int oracle_offsets(int ndim, int shape, int radius, int* dz, int* dy, int* dx)
{
    if ((ndim != 2 && ndim != 3) || radius < 1 || shape < OR_STAR || shape > OR_J3D17)
        return -1;
    if ((shape == OR_POISSON || shape == OR_J3D17) && (ndim != 3 || radius != 1))
        return -1;
    int zr = (ndim == 3) ? radius : 0;
    int n = 0;
    for (int a = -zr; a <= zr; a++)
        for (int b = -radius; b <= radius; b++)
            for (int c = -radius; c <= radius; c++) {
                int nonzero = (a != 0) + (b != 0) + (c != 0);
                if (shape == OR_STAR && nonzero > 1)
                    continue;
                if ((shape == OR_POISSON || shape == OR_J3D17) && nonzero > 2)
                    continue;
                if (shape == OR_J3D17 && a != 0 && b == 0 && c == 0)
                    continue;
                if (dz) dz[n] = a;
                if (dy) dy[n] = b;
                if (dx) dx[n] = c;
                n++;
            }
    return n;
}

static int64_t wrap(int64_t i, int64_t n)
{
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

/* One Jacobi step over the whole grid: dst = S(src).
 * ext[] are the stored extents (padded for Dirichlet), n[] the interior
 * extents; 2D grids are handled as 3D grids with one unpadded plane
 * (zpad = 0, dz = 0). */
static void one_step(const int64_t ext[3], const int64_t n[3], int pad,
                     int zpad, int boundary, int npts, const int* oz, const int* oy,
                     const int* ox, const double* c, const double* src,
                     double* dst, int nthreads)
{
    (void)nthreads;
    int64_t sy = ext[2], sz = ext[1] * ext[2];
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static) collapse(2)
#endif
    for (int64_t z = 0; z < n[0]; z++) {
        for (int64_t y = 0; y < n[1]; y++) {
            for (int64_t x = 0; x < n[2]; x++) {
                double acc = 0.0;
                for (int k = 0; k < npts; k++) {
                    int64_t zz, yy, xx;
                    if (boundary == OR_PERIODIC) {
                        zz = wrap(z + oz[k], n[0]);
                        yy = wrap(y + oy[k], n[1]);
                        xx = wrap(x + ox[k], n[2]);
                    } else {
                        zz = z + oz[k] + zpad;
                        yy = y + oy[k] + pad;
                        xx = x + ox[k] + pad;
                    }
                    double term = c[k] * src[zz * sz + yy * sy + xx];
                    acc = acc + term;
                }
                int64_t zo = (boundary == OR_PERIODIC) ? z : z + zpad;
                int64_t yo = (boundary == OR_PERIODIC) ? y : y + pad;
                int64_t xo = (boundary == OR_PERIODIC) ? x : x + pad;
                dst[zo * sz + yo * sy + xo] = acc;
            }
        }
    }
}

/* Run `steps` Jacobi steps of the stencil with the given offsets.
 *   dims: interior extents, slowest first ((ny, nx) or (nz, ny, nx)).
 *   radius: pad width of a Dirichlet grid; every |offset component| must be
 *   <= radius (2D: dz = 0).
 *   oz/oy/ox/coeffs: npts offsets and their weights, summed in the order
 *   given (callers pass the canonical order).
 *   in/out: stored arrays (padded by `radius` for Dirichlet); `in` is not
 *   modified; out may not alias in.  steps == 0 copies in to out.
 *   nthreads <= 0 means "all available". */
int oracle_run_offsets(int ndim, const int64_t* dims, int radius, int npts, const int* oz,
                       const int* oy, const int* ox, const double* coeffs, int boundary,
                       const double* in, double* out, int64_t steps, int nthreads)
{
    if ((ndim != 2 && ndim != 3) || radius < 1 || npts < 1 || steps < 0 || !dims || !coeffs || !in ||
        !out || in == out || !oz || !oy || !ox)
        return -1;
    if (boundary != OR_DIRICHLET && boundary != OR_PERIODIC)
        return -1;
    for (int k = 0; k < npts; k++) {
        if (abs(oz[k]) > radius || abs(oy[k]) > radius || abs(ox[k]) > radius) return -1;
        if (ndim == 2 && oz[k] != 0) return -1;
    }
    int64_t n[3] = {1, 1, 1};
    for (int d = 0; d < ndim; d++) {
        if (dims[d] < 1) return -1;
        n[3 - ndim + d] = dims[d];
    }
    int pad = (boundary == OR_DIRICHLET) ? radius : 0;
    int64_t ext[3];
    for (int d = 0; d < 3; d++)
        ext[d] = n[d] + ((d >= 3 - ndim) ? 2 * pad : 0);
    int64_t total = ext[0] * ext[1] * ext[2];

    double* tmp = malloc(sizeof(double) * (size_t)total);
    if (!tmp) return -2;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    /* Both buffers start as full copies of the input, so the Dirichlet pad of
     * each holds the initial values for the whole run. */
    memcpy(out, in, sizeof(double) * (size_t)total);
    memcpy(tmp, in, sizeof(double) * (size_t)total);
    /* Ping-pong so that the last step lands in `out`. */
    double* a = (steps % 2 == 0) ? out : tmp;
    double* b = (steps % 2 == 0) ? tmp : out;
    for (int64_t s = 0; s < steps; s++) {
        one_step(ext, n, pad, (ndim == 3) ? pad : 0, boundary, npts, oz, oy, ox,
                 coeffs, a, b, nthreads);
        double* t = a; a = b; b = t;
    }
    free(tmp);
    return 0;
}

/* Run `steps` Jacobi steps of a named stencil (star, box, poisson, j3d17pt;
 * offsets from oracle_offsets, canonical order).  Arguments as for
 * oracle_run_offsets. */
int oracle_run(int ndim, const int64_t* dims, int shape, int radius,
               const double* coeffs, int boundary, const double* in,
               double* out, int64_t steps, int nthreads)
{
    int npts = oracle_offsets(ndim, shape, radius, NULL, NULL, NULL);
    if (npts < 0)
        return -1;
    int* oz = malloc(sizeof(int) * npts);
    int* oy = malloc(sizeof(int) * npts);
    int* ox = malloc(sizeof(int) * npts);
    if (!oz || !oy || !ox) {
        free(oz); free(oy); free(ox);
        return -2;
    }
    oracle_offsets(ndim, shape, radius, oz, oy, ox);
    int rc = oracle_run_offsets(ndim, dims, radius, npts, oz, oy, ox, coeffs, boundary, in, out, steps,
                                nthreads);
    free(oz); free(oy); free(ox);
    return rc;
}

/* Variable coefficients (an extension; the paper's stencils have fixed
 * weights): u_s(x) = sum_k c_k(x) * u_{s-1}(x + o_k), the weights of cell x
 * read from `field`, which holds npts arrays laid out like the stored grid
 * (array k starts at field + k * stored elements; pad entries unused).
 * Offsets of a named shape, canonical order; other arguments as for
 * oracle_run. */
int oracle_run_varcoef(int ndim, const int64_t* dims, int shape, int radius,
                       const double* field, int boundary, const double* in,
                       double* out, int64_t steps)
{
    int npts = oracle_offsets(ndim, shape, radius, NULL, NULL, NULL);
    if (npts < 0 || steps < 0 || !dims || !field || !in || !out || in == out)
        return -1;
    if (boundary != OR_DIRICHLET && boundary != OR_PERIODIC)
        return -1;
    int64_t n[3] = {1, 1, 1};
    for (int d = 0; d < ndim; d++) {
        if (dims[d] < 1) return -1;
        n[3 - ndim + d] = dims[d];
    }
    int pad = (boundary == OR_DIRICHLET) ? radius : 0;
    int zpad = (ndim == 3) ? pad : 0;
    int64_t ext[3];
    for (int d = 0; d < 3; d++)
        ext[d] = n[d] + ((d >= 3 - ndim) ? 2 * pad : 0);
    int64_t total = ext[0] * ext[1] * ext[2];
    int64_t sy = ext[2], sz = ext[1] * ext[2];
    int* oz = malloc(sizeof(int) * npts);
    int* oy = malloc(sizeof(int) * npts);
    int* ox = malloc(sizeof(int) * npts);
    double* tmp = malloc(sizeof(double) * (size_t)total);
    if (!oz || !oy || !ox || !tmp) {
        free(oz); free(oy); free(ox); free(tmp);
        return -2;
    }
    oracle_offsets(ndim, shape, radius, oz, oy, ox);
    memcpy(out, in, sizeof(double) * (size_t)total);
    memcpy(tmp, in, sizeof(double) * (size_t)total);
    double* a = (steps % 2 == 0) ? out : tmp;
    double* b = (steps % 2 == 0) ? tmp : out;
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t z = 0; z < n[0]; z++)
            for (int64_t y = 0; y < n[1]; y++)
                for (int64_t x = 0; x < n[2]; x++) {
                    int64_t zo = (boundary == OR_PERIODIC) ? z : z + zpad;
                    int64_t yo = (boundary == OR_PERIODIC) ? y : y + pad;
                    int64_t xo = (boundary == OR_PERIODIC) ? x : x + pad;
                    int64_t self = zo * sz + yo * sy + xo;
                    double acc = 0.0;
                    for (int k = 0; k < npts; k++) {
                        int64_t zz, yy, xx;
                        if (boundary == OR_PERIODIC) {
                            zz = wrap(z + oz[k], n[0]);
                            yy = wrap(y + oy[k], n[1]);
                            xx = wrap(x + ox[k], n[2]);
                        } else {
                            zz = z + oz[k] + zpad;
                            yy = y + oy[k] + pad;
                            xx = x + ox[k] + pad;
                        }
                        double term = field[(int64_t)k * total + self] * a[zz * sz + yy * sy + xx];
                        acc = acc + term;
                    }
                    b[self] = acc;
                }
        double* t = a; a = b; b = t;
    }
    free(oz); free(oy); free(ox); free(tmp);
    return 0;
}

/* Interior reductions used for verification and reporting (FP64):
 *   res[0] = sum of interior values (Neumaier compensated summation),
 *   res[1] = sqrt(sum of squares)   (compensated),
 *   res[2] = max |value|.
 * `b` may be NULL; otherwise the reductions are of (a - b). */
int oracle_reduce(int ndim, const int64_t* dims, int pad, const double* a,
                  const double* b, double* res)
{
    if ((ndim != 2 && ndim != 3) || !dims || !a || !res || pad < 0)
        return -1;
    int64_t n[3] = {1, 1, 1};
    for (int d = 0; d < ndim; d++) n[3 - ndim + d] = dims[d];
    int64_t ext[3];
    for (int d = 0; d < 3; d++) ext[d] = n[d] + ((d >= 3 - ndim) ? 2 * pad : 0);
    int zp = (ndim == 3) ? pad : 0;
    double s = 0.0, cs = 0.0, q = 0.0, cq = 0.0, m = 0.0;
    for (int64_t z = 0; z < n[0]; z++)
        for (int64_t y = 0; y < n[1]; y++)
            for (int64_t x = 0; x < n[2]; x++) {
                int64_t i = ((z + zp) * ext[1] + (y + pad)) * ext[2] + (x + pad);
                double v = b ? a[i] - b[i] : a[i];
                double t = s + v;
                if (fabs(s) >= fabs(v)) cs += (s - t) + v; else cs += (v - t) + s;
                s = t;
                double v2 = v * v;
                double t2 = q + v2;
                if (fabs(q) >= fabs(v2)) cq += (q - t2) + v2; else cq += (v2 - t2) + q;
                q = t2;
                if (fabs(v) > m) m = fabs(v);
            }
    res[0] = s + cs;
    res[1] = sqrt(q + cq);
    res[2] = m;
    return 0;
}
