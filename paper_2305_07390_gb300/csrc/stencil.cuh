// stencil.cuh -- device-side stencil definition shared by every CUDA kernel.
//
// The update is the Jacobi sweep of Section 2.1 (Listings 1-3, shapes of
// Table 2): new(x) = sum_k c_k * old(x + o_k).  Offsets are generated at
// compile time in canonical order -- lexicographic in (dz, dy, dx) -- and the
// sum is always taken as
//     acc = c_0 * u_0;  acc = fma(c_k, u_k, acc),  k = 1 .. P-1,
// with explicit round-to-nearest intrinsics, so every kernel of the library
// (naive, temporally blocked, batched) produces bit-identical cells.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ebisu {

// Shapes: star (centre + axis offsets |k| <= r), box (every offset with
// max |k| <= r), and two 3D order-1 sets of Table 2: poisson (the 27-point
// box without its corners, 19 points) and j3d17pt (17 points: poisson
// without the z-axis neighbours -- the z = 0 plane's 3x3 box plus the four
// in-plane axis neighbours in each of the planes z = +-1; the paper lists
// only the point count, this is the library's reading).
enum { kStar = 0, kBox = 1, kPoisson = 2, kJ3d17 = 3 };

// ---------------------------------------------------------------------------
// Canonical offsets, expressed in streaming coordinates: `s` is the slowest
// axis (y in 2D, z in 3D) along which tiles are streamed; `p1`, `p2` are the
// in-plane axes (p1 is a dummy axis of extent 1 in 2D, p2 is x).

template <int DIM, int SHAPE, int R>
struct Stencil {
    static constexpr int kR = R;
    static constexpr int kDim = DIM;
    static constexpr int kRP1 = (DIM == 3) ? R : 0;  // radius along p1
    static_assert(SHAPE == kStar || SHAPE == kBox || (DIM == 3 && R == 1), "poisson and j3d17pt: 3D, radius 1");
    // is (a, b, c) = (ds, d1, d2) in the support set?
    static constexpr bool member(int a, int b, int c)
    {
        const int nz = (a != 0) + (b != 0) + (c != 0);
        if (SHAPE == kStar) return nz <= 1;
        if (SHAPE == kPoisson) return nz <= 2;
        if (SHAPE == kJ3d17) return nz <= 2 && !(a != 0 && b == 0 && c == 0);
        return true;
    }
    static constexpr int count()
    {
        int n = 0;
        const int zr = (DIM == 3) ? R : 0;
        for (int a = -zr; a <= zr; ++a)
            for (int b = -R; b <= R; ++b)
                for (int c = -R; c <= R; ++c) n += member(DIM == 3 ? a : 0, b, c) ? 1 : 0;
        return n;
    }
    static constexpr int P = count();
    struct Table {
        int ds[P];
        int d1[P];
        int d2[P];
    };
    static constexpr Table make()
    {
        Table t{};
        int n = 0;
        const int zr = (DIM == 3) ? R : 0;
        for (int a = -zr; a <= zr; ++a)
            for (int b = -R; b <= R; ++b)
                for (int c = -R; c <= R; ++c) {
                    if (!member(a, b, c)) continue;
                    if (DIM == 3) {
                        t.ds[n] = a; t.d1[n] = b; t.d2[n] = c;
                    } else {
                        t.ds[n] = b; t.d1[n] = 0; t.d2[n] = c;
                    }
                    ++n;
                }
        return t;
    }
    static constexpr Table kOff = make();

    // Offsets sharing (ds, d1) -- one row of one plane -- are consecutive in
    // canonical order.  Per offset k: does a new row group start at k, and
    // the d2 range of k's row group.  Built at compile time (kernels copy it
    // into a constexpr local, like kOff, so every lookup folds away).
    struct RowInfo {
        bool start[P];
        int min_d2[P];
        int max_d2[P];
    };
    static constexpr RowInfo make_rows()
    {
        RowInfo r{};
        const Table t = make();
        for (int k = 0; k < P; ++k)
            r.start[k] = (k == 0) || t.ds[k] != t.ds[k - 1] || t.d1[k] != t.d1[k - 1];
        for (int k = 0; k < P; ++k) {
            int b = k;
            while (!r.start[b]) --b;
            int lo = t.d2[b], hi = t.d2[b];
            for (int j = b; j < P && (j == b || !r.start[j]); ++j) {
                lo = t.d2[j] < lo ? t.d2[j] : lo;
                hi = t.d2[j] > hi ? t.d2[j] : hi;
            }
            r.min_d2[k] = lo;
            r.max_d2[k] = hi;
        }
        return r;
    }
};

// ---------------------------------------------------------------------------
// Storage / compute type traits.  C is the accumulation type.

template <class T>
struct DT;

template <>
struct DT<double> {
    using C = double;
    static constexpr bool kSR = false;
    __device__ static __forceinline__ C load(const double* p) { return __ldcg(p); }
    __device__ static __forceinline__ double raw(const double* p) { return __ldcg(p); }
    __device__ static __forceinline__ C load_ro(const double* p) { return __ldg(p); }
    __device__ static __forceinline__ C widen(double v) { return v; }
    __device__ static __forceinline__ double narrow(C v) { return v; }
    __device__ static __forceinline__ C mul(C a, C b) { return __dmul_rn(a, b); }
    __device__ static __forceinline__ C fma(C a, C b, C c) { return __fma_rn(a, b, c); }
    __host__ __device__ static __forceinline__ C coef(double v) { return v; }
};

template <>
struct DT<float> {
    using C = float;
    static constexpr bool kSR = false;
    __device__ static __forceinline__ C load(const float* p) { return __ldcg(p); }
    __device__ static __forceinline__ float raw(const float* p) { return __ldcg(p); }
    __device__ static __forceinline__ C load_ro(const float* p) { return __ldg(p); }
    __device__ static __forceinline__ C widen(float v) { return v; }
    __device__ static __forceinline__ float narrow(C v) { return v; }
    __device__ static __forceinline__ C mul(C a, C b) { return __fmul_rn(a, b); }
    __device__ static __forceinline__ C fma(C a, C b, C c) { return __fmaf_rn(a, b, c); }
    __host__ __device__ static __forceinline__ C coef(double v) { return (float)v; }
};

template <>
struct DT<__nv_bfloat16> {
    using C = float;
    static constexpr bool kSR = false;
    __device__ static __forceinline__ C load(const __nv_bfloat16* p)
    {
        unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p));
        return __uint_as_float(((unsigned)b) << 16);
    }
    __device__ static __forceinline__ __nv_bfloat16 raw(const __nv_bfloat16* p)
    {
        unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p));
        return __ushort_as_bfloat16(b);
    }
    __device__ static __forceinline__ C load_ro(const __nv_bfloat16* p)
    {
        unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p));
        return __uint_as_float(((unsigned)b) << 16);
    }
    __device__ static __forceinline__ C widen(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __forceinline__ __nv_bfloat16 narrow(C v) { return __float2bfloat16_rn(v); }
    __device__ static __forceinline__ C mul(C a, C b) { return __fmul_rn(a, b); }
    __device__ static __forceinline__ C fma(C a, C b, C c) { return __fmaf_rn(a, b, c); }
    __host__ __device__ static __forceinline__ C coef(double v) { return (float)v; }
};

// ---------------------------------------------------------------------------
// Stochastic rounding of FP32 results to BF16 storage (a plan option; the
// paper's kernels are FP64 only).  Round-to-nearest storage discards every
// update smaller than half a BF16 ulp, so long runs stagnate; rounding up
// with probability equal to the discarded fraction of an ulp keeps the
// rounding unbiased.  The random bits are a pure function of (seed, step,
// stored cell index), so every kernel -- blocked, naive, batched -- rounds a
// given cell of a given step the same way, and their results stay identical.
//
//   pcg_hash(v)   : the PCG hash of Jarzynski and Olano ("Hash Functions for
//                   GPU Rendering", JCGT 9(3), 2020): one step of the 32-bit
//                   LCG of the PCG family followed by its RXS-M-XS output
//                   permutation (O'Neill, 2014).  A bijection of 32-bit words.
//   plan key      : K = pcg_hash(lo32(seed) ^ pcg_hash(hi32(seed)))
//   step key      : K_t = pcg_hash(K ^ t), t = 1 .. steps (the step whose
//                   result is being rounded)
//   cell bits     : rnd = pcg_hash(i + K_t), i = the cell's index in the
//                   stored (padded) array, modulo 2^32
//   rounding      : BF16 bits of (bits(x) + (rnd >> 16)) truncated to their
//                   upper 16 bits (x finite).
// The last xor-shift of pcg_hash only changes bits 0-9, so rnd >> 16 equals
// the multiply's upper half; sr_bits16 computes just that.

struct bf16sr {  // storage tag: BF16 values, stochastic rounding
    unsigned short bits;
};

__host__ __device__ __forceinline__ uint32_t pcg_hash(uint32_t v)
{
    const uint32_t s = v * 747796405u + 2891336453u;
    const uint32_t w = ((s >> ((s >> 28) + 4u)) ^ s) * 277803737u;
    return (w >> 22) ^ w;
}

__host__ __device__ __forceinline__ uint32_t sr_plan_key(uint64_t seed)
{
    return pcg_hash((uint32_t)seed ^ pcg_hash((uint32_t)(seed >> 32)));
}

__host__ __device__ __forceinline__ uint32_t sr_step_key(uint32_t plan_key, uint32_t t)
{
    return pcg_hash(plan_key ^ t);
}

// upper 16 bits of pcg_hash(v)
__device__ __forceinline__ uint32_t sr_bits16(uint32_t v)
{
    const uint32_t s = v * 747796405u + 2891336453u;
    const uint32_t w = ((s >> ((s >> 28) + 4u)) ^ s) * 277803737u;
    return w >> 16;
}

// x rounded stochastically to BF16, returned as FP32; `cell_plus_key` is
// i + K_t (modulo 2^32)
__device__ __forceinline__ float sr_round_bf16(float x, uint32_t cell_plus_key)
{
    return __uint_as_float((__float_as_uint(x) + sr_bits16(cell_plus_key)) & 0xFFFF0000u);
}

template <>
struct DT<bf16sr> {
    using C = float;
    static constexpr bool kSR = true;
    __device__ static __forceinline__ C load(const bf16sr* p)
    {
        unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p));
        return __uint_as_float(((unsigned)b) << 16);
    }
    __device__ static __forceinline__ bf16sr raw(const bf16sr* p)
    {
        return bf16sr{__ldcg(reinterpret_cast<const unsigned short*>(p))};
    }
    __device__ static __forceinline__ C load_ro(const bf16sr* p)
    {
        unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p));
        return __uint_as_float(((unsigned)b) << 16);
    }
    __device__ static __forceinline__ C widen(bf16sr v) { return __uint_as_float(((unsigned)v.bits) << 16); }
    // exact for the values these kernels store (already BF16 after rounding
    // or copied from BF16 storage)
    __device__ static __forceinline__ bf16sr narrow(C v)
    {
        return bf16sr{(unsigned short)(__float_as_uint(v) >> 16)};
    }
    __device__ static __forceinline__ C mul(C a, C b) { return __fmul_rn(a, b); }
    __device__ static __forceinline__ C fma(C a, C b, C c) { return __fmaf_rn(a, b, c); }
    __host__ __device__ static __forceinline__ C coef(double v) { return (float)v; }
};

// Periodic index wrap (any i; the common in-range case costs two compares).
__device__ __forceinline__ int64_t wrap_idx(int64_t i, int64_t n)
{
    if (i >= 0 && i < n) return i;
    const int64_t m = i % n;
    return m < 0 ? m + n : m;
}

// Wall-clock time in ns (bounded waits).
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace ebisu
