// kernels_impl.cuh -- naive kernel, pad copy, reductions and the dispatch of
// every kernel template over (ndim, shape, radius) for one storage type.
// Included once per storage type by kern_f64.cu / kern_f32.cu / kern_bf16.cu.
#pragma once
#include <mutex>
#include <unordered_map>

#include "dispatch.h"
#include "tb_kernel.cuh"

namespace ebisu {

// ---------------------------------------------------------------------------
// Naive one-step kernel: one thread per interior cell of each of kNaiveRows
// rows (2D: rows 8 apart, so a warp's loads stay coalesced; 3D: consecutive
// planes), neighbours read from global memory (read-only path), same
// canonical FMA chain as the blocked kernels.  This is the "one time step per
// launch" reference GPU path; several cells per thread keep enough loads in
// flight to stream at the memory bandwidth.

constexpr int kNaiveRows = 4;

template <class T, int DIM, int SHAPE, int R>
__global__ void __launch_bounds__(256) naive_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                    const __grid_constant__ NaiveParams a)
{
    using St = Stencil<DIM, SHAPE, R>;
    using D = DT<T>;
    using C = typename D::C;
    constexpr int P = St::P;
    constexpr auto OFF = St::kOff;
    const int64_t n0 = a.n[0];
    const int n1 = (int)a.n[1], n2 = (int)a.n[2];
    const int q2 = blockIdx.x * 32 + threadIdx.x;
    const int q1 = (DIM == 3) ? (int)(blockIdx.y * 8 + threadIdx.y) : 0;
    if (q2 >= n2 || q1 >= n1) return;
    const int pad = a.pad, pad1 = (DIM == 3) ? a.pad : 0;
    const int64_t lds = a.lds, ld1 = a.ld1;
    // coefficients already in the accumulation type: a per-cell FP64 -> FP32
    // conversion would run on the (slow) FP64 pipe
    auto cf = [&](int k) -> C {
        if constexpr (std::is_same<C, double>::value) return a.coef[k];
        else return a.coef_f[k];
    };
    // unrolled: the rows' loads are all in flight together (at one cell per
    // thread the kernel is bound by memory latency, not bandwidth)
#pragma unroll
    for (int i = 0; i < kNaiveRows; ++i) {
        const int64_t ps = (DIM == 3) ? (int64_t)blockIdx.z * kNaiveRows + i
                                      : ((int64_t)blockIdx.y * kNaiveRows + i) * 8 + threadIdx.y;
        if (ps >= n0) return;
        C acc;
        if (a.periodic) {
            auto at = [&](int k) -> C {
                const int64_t s_ = wrap_idx(ps + OFF.ds[k], n0);
                const int64_t y_ = (DIM == 3) ? wrap_idx(q1 + OFF.d1[k], n1) : 0;
                const int64_t x_ = wrap_idx(q2 + OFF.d2[k], n2);
                return D::load_ro(src + s_ * lds + y_ * ld1 + x_);
            };
            acc = D::mul(cf(0), at(0));
#pragma unroll
            for (int k = 1; k < P; ++k) acc = D::fma(cf(k), at(k), acc);
            const int64_t o = ps * lds + (int64_t)q1 * ld1 + q2;
            if constexpr (D::kSR) acc = sr_round_bf16(acc, (uint32_t)o + a.sr_k);
            dst[o] = D::narrow(acc);
        } else {
            const int64_t c = (ps + pad) * lds + (int64_t)(q1 + pad1) * ld1 + (q2 + pad);
            const T* p = src + c;
            auto at = [&](int k) -> C { return D::load_ro(p + OFF.ds[k] * lds + OFF.d1[k] * ld1 + OFF.d2[k]); };
            acc = D::mul(cf(0), at(0));
#pragma unroll
            for (int k = 1; k < P; ++k) acc = D::fma(cf(k), at(k), acc);
            if constexpr (D::kSR) acc = sr_round_bf16(acc, (uint32_t)c + a.sr_k);
            dst[c] = D::narrow(acc);
        }
    }
}

// ---------------------------------------------------------------------------
// Variable coefficients: the same one-step sweep with the weights of cell x
// read from `field` (P arrays laid out like the stored grid, array k at
// field + k * fstride, in the accumulation type).  Each step reads P weights
// per cell, which no temporal blocking can spare (they are not produced by
// the previous step), so plans with a coefficient field run this kernel.

template <class T, int DIM, int SHAPE, int R>
__global__ void __launch_bounds__(256) naive_vc_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                       const typename DT<T>::C* __restrict__ field,
                                                       int64_t fstride, const __grid_constant__ NaiveParams a)
{
    using St = Stencil<DIM, SHAPE, R>;
    using D = DT<T>;
    using C = typename D::C;
    constexpr int P = St::P;
    constexpr auto OFF = St::kOff;
    const int64_t n0 = a.n[0];
    const int n1 = (int)a.n[1], n2 = (int)a.n[2];
    const int q2 = blockIdx.x * 32 + threadIdx.x;
    const int q1 = (DIM == 3) ? (int)(blockIdx.y * 8 + threadIdx.y) : 0;
    if (q2 >= n2 || q1 >= n1) return;
    const int pad = a.pad, pad1 = (DIM == 3) ? a.pad : 0;
    const int64_t lds = a.lds, ld1 = a.ld1;
#pragma unroll
    for (int i = 0; i < kNaiveRows; ++i) {
        const int64_t ps = (DIM == 3) ? (int64_t)blockIdx.z * kNaiveRows + i
                                      : ((int64_t)blockIdx.y * kNaiveRows + i) * 8 + threadIdx.y;
        if (ps >= n0) return;
        int64_t o;
        C acc;
        if (a.periodic) {
            o = ps * lds + (int64_t)q1 * ld1 + q2;
            auto at = [&](int k) -> C {
                const int64_t s_ = wrap_idx(ps + OFF.ds[k], n0);
                const int64_t y_ = (DIM == 3) ? wrap_idx(q1 + OFF.d1[k], n1) : 0;
                const int64_t x_ = wrap_idx(q2 + OFF.d2[k], n2);
                return D::load_ro(src + s_ * lds + y_ * ld1 + x_);
            };
            acc = D::mul(__ldg(field + o), at(0));
#pragma unroll
            for (int k = 1; k < P; ++k) acc = D::fma(__ldg(field + k * fstride + o), at(k), acc);
        } else {
            o = (ps + pad) * lds + (int64_t)(q1 + pad1) * ld1 + (q2 + pad);
            const T* p = src + o;
            auto at = [&](int k) -> C { return D::load_ro(p + OFF.ds[k] * lds + OFF.d1[k] * ld1 + OFF.d2[k]); };
            acc = D::mul(__ldg(field + o), at(0));
#pragma unroll
            for (int k = 1; k < P; ++k) acc = D::fma(__ldg(field + k * fstride + o), at(k), acc);
        }
        dst[o] = D::narrow(acc);
    }
}

// ---------------------------------------------------------------------------
// Copy the Dirichlet pad of `src` into up to two destinations.  Pad cells are
// enumerated directly: the 2*pad pad planes along s, the pad rows of interior
// planes, then the pad cells of interior rows (stored coordinates).

template <class T>
__global__ void pad_copy_kernel(const T* __restrict__ src, T* d0, T* d1, PadParams a)
{
    const int64_t E1 = a.n[1] + 2 * a.pad1, E2 = a.n[2] + 2 * a.pad;
    const int64_t A = 2 * (int64_t)a.pad * E1 * E2;
    const int64_t B = a.n[0] * 2 * (int64_t)a.pad1 * E2;
    const int64_t Cn = a.n[0] * a.n[1] * 2 * (int64_t)a.pad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A + B + Cn;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t ps, y, x;
        if (i < A) {
            const int64_t pl = i / (E1 * E2), rem = i % (E1 * E2);
            ps = (pl < a.pad) ? pl : a.n[0] + pl;
            y = rem / E2;
            x = rem % E2;
        } else if (i < A + B) {
            const int64_t j = i - A;
            const int64_t pl = j / (2 * a.pad1 * E2), rem = j % (2 * a.pad1 * E2);
            ps = a.pad + pl;
            const int64_t rr = rem / E2;
            y = (rr < a.pad1) ? rr : a.n[1] + rr;
            x = rem % E2;
        } else {
            const int64_t j = i - A - B;
            const int64_t row = j / (2 * a.pad), c = j % (2 * a.pad);
            ps = a.pad + row / a.n[1];
            y = a.pad1 + row % a.n[1];
            x = (c < a.pad) ? c : a.n[2] + c;
        }
        const int64_t o = ps * a.lds + y * a.ld1 + x;
        const T v = src[o];
        if (d0) d0[o] = v;
        if (d1) d1[o] = v;
    }
}

// ---------------------------------------------------------------------------
// FP64 reductions over the interior with a fixed tree: block b owns cells
// [b*kRedChunk, (b+1)*kRedChunk) in a fixed thread order, writes one partial
// (sum, sum of squares, max |.|); one block then folds the partials in a
// fixed order.  The result does not depend on timing.

constexpr int kRedThreads = 256;
constexpr int kRedChunk = 4096;

template <class T>
__global__ void __launch_bounds__(kRedThreads) reduce_partial_kernel(const T* __restrict__ a,
                                                                     const T* __restrict__ b,
                                                                     double* part, PadParams g)
{
    using D = DT<T>;
    __shared__ double s0[kRedThreads], s1[kRedThreads], s2[kRedThreads];
    const int64_t cells = g.n[0] * g.n[1] * g.n[2];
    const int64_t beg = (int64_t)blockIdx.x * kRedChunk;
    double sum = 0.0, sq = 0.0, mx = 0.0;
    for (int k = 0; k < kRedChunk / kRedThreads; ++k) {
        const int64_t i = beg + (int64_t)k * kRedThreads + threadIdx.x;
        if (i >= cells) break;
        const int64_t x = i % g.n[2], y = (i / g.n[2]) % g.n[1], s = i / (g.n[2] * g.n[1]);
        const int64_t o = (s + g.pad) * g.lds + (y + g.pad1) * g.ld1 + (x + g.pad);
        double v = (double)D::load_ro(a + o);
        if (b) v -= (double)D::load_ro(b + o);
        sum += v;
        sq = fma(v, v, sq);
        mx = fmax(mx, fabs(v));
    }
    s0[threadIdx.x] = sum;
    s1[threadIdx.x] = sq;
    s2[threadIdx.x] = mx;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s0[threadIdx.x] += s0[threadIdx.x + w];
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = s0[0];
        part[3 * blockIdx.x + 1] = s1[0];
        part[3 * blockIdx.x + 2] = s2[0];
    }
}

// ---------------------------------------------------------------------------
// dispatch over (ndim, shape, radius)

#define EBISU_FOR_EACH_STENCIL(X) \
    X(2, kStar, 1) X(2, kStar, 2) X(2, kStar, 3) X(2, kBox, 1) X(2, kBox, 2) \
    X(3, kStar, 1) X(3, kStar, 2) X(3, kStar, 3) X(3, kBox, 1) X(3, kBox, 2) \
    X(3, kPoisson, 1) X(3, kJ3d17, 1)

constexpr int kTBThreads = 256;
constexpr int kTBStage = 16;
constexpr int kTBILP = 4;

// Two builds of the blocked kernel per stencil:
//   variant 0: up to 128 registers (2 resident CTAs); prefetch 2 planes in
//              3D, 3 in 2D FP64 (2048-wide FP64 rows still fit twice per SM)
//              and 4 in 2D FP32/BF16;
//   variant 1 (FP64 only): up to 64 registers and 2 planes of prefetch, so
//              that 4 CTAs fit on an SM.  The FP64 pipe only stays busy when
//              enough warps are resident to cover the per-plane barrier.
// tb_variant_prefetch() must agree with prefetch_planes() on the host.
template <class T, int DIM, int SHAPE, int R, int V>
struct TBInst {
    static constexpr int PF = (V == 1 || DIM == 3) ? 2 : (sizeof(T) == 8 ? 3 : 4);
    static constexpr int MINB = (V == 1) ? 4 : 2;
    // 4-wide compute for the FP32-arithmetic types (FP32, BF16 storage);
    // measured slower than the scalar path for FP64, whose FP64 pipe, not the
    // shared-memory issue, is the bound
    static constexpr int VEC = sizeof(T) == 8 ? 0 : 1;
    // independent FMA chains per thread: the FP64 pipe's dependent-issue
    // latency needs more of them than FP32 (128-register build only)
    static constexpr int ILP = (sizeof(T) == 8 && V == 0) ? 8 : kTBILP;
    static const void* ptr()
    {
        return (const void*)&tb_kernel<T, DIM, SHAPE, R, kTBThreads, ILP, PF, kTBStage, MINB, VEC>;
    }
};

template <class T>
static const void* tb_kernel_ptr(int dim, int shape, int r, int variant)
{
#define X(D_, S_, R_) \
    if (dim == D_ && shape == S_ && r == R_) { \
        if constexpr (sizeof(T) == 8) { \
            if (variant == 1) return TBInst<T, D_, S_, R_, 1>::ptr(); \
        } \
        return TBInst<T, D_, S_, R_, 0>::ptr(); \
    }
    EBISU_FOR_EACH_STENCIL(X)
#undef X
    return nullptr;
}

template <class T>
static const void* naive_kernel_ptr(int dim, int shape, int r)
{
#define X(D_, S_, R_) \
    if (dim == D_ && shape == S_ && r == R_) return (const void*)&naive_kernel<T, D_, S_, R_>;
    EBISU_FOR_EACH_STENCIL(X)
#undef X
    return nullptr;
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than what was set before, so that launches inside a stream capture make no
// attribute calls once a warm-up launch has set the limit.
static cudaError_t ensure_smem_limit(const void* k, size_t smem)
{
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> limit;
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[k];
    if (smem <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

template <class T>
static cudaError_t tb_launch_t(int dim, int shape, int r, int variant, const TBParams& p, int grid, size_t smem,
                               cudaStream_t st)
{
    const void* k = tb_kernel_ptr<T>(dim, shape, r, variant);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(k, dim3(grid), dim3(kTBThreads), args, smem, st);
}

template <class T>
static cudaError_t tb_occupancy_t(int dim, int shape, int r, int variant, size_t smem, int* blocks)
{
    const void* k = tb_kernel_ptr<T>(dim, shape, r, variant);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kTBThreads, smem);
}

template <class T>
static cudaError_t naive_launch_t(int dim, int shape, int r, const void* src, void* dst,
                                  const NaiveParams& p, cudaStream_t st)
{
    const void* k = naive_kernel_ptr<T>(dim, shape, r);
    if (!k) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((p.n[2] + 31) / 32), 1, 1);
    if (dim == 3) {
        grid.y = (unsigned)((p.n[1] + 7) / 8);
        grid.z = (unsigned)((p.n[0] + kNaiveRows - 1) / kNaiveRows);
    } else {
        grid.y = (unsigned)((p.n[0] + 8 * kNaiveRows - 1) / (8 * kNaiveRows));
    }
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    void* args[] = {(void*)&src, (void*)&dst, (void*)&p};
    return cudaLaunchKernel(k, grid, dim3(32, 8), args, 0, st);
}

template <class T>
static cudaError_t naive_vc_launch_t(int dim, int shape, int r, const void* src, void* dst, const void* field,
                                     int64_t fstride, const NaiveParams& p, cudaStream_t st)
{
    const void* k = nullptr;
#define X(D_, S_, R_) \
    if (dim == D_ && shape == S_ && r == R_) k = (const void*)&naive_vc_kernel<T, D_, S_, R_>;
    EBISU_FOR_EACH_STENCIL(X)
#undef X
    if (!k) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((p.n[2] + 31) / 32), 1, 1);
    if (dim == 3) {
        grid.y = (unsigned)((p.n[1] + 7) / 8);
        grid.z = (unsigned)((p.n[0] + kNaiveRows - 1) / kNaiveRows);
    } else {
        grid.y = (unsigned)((p.n[0] + 8 * kNaiveRows - 1) / (8 * kNaiveRows));
    }
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    void* args[] = {(void*)&src, (void*)&dst, (void*)&field, (void*)&fstride, (void*)&p};
    return cudaLaunchKernel(k, grid, dim3(32, 8), args, 0, st);
}

template <class T>
static cudaError_t pad_copy_t(const void* src, void* d0, void* d1, const PadParams& p, cudaStream_t st)
{
    const int64_t E1 = p.n[1] + 2 * p.pad1, E2 = p.n[2] + 2 * p.pad;
    const int64_t total = 2 * (int64_t)p.pad * E1 * E2 + p.n[0] * 2 * (int64_t)p.pad1 * E2 +
                          p.n[0] * p.n[1] * 2 * (int64_t)p.pad;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    pad_copy_kernel<T><<<(unsigned)blocks, 256, 0, st>>>((const T*)src, (T*)d0, (T*)d1, p);
    return cudaGetLastError();
}

template <class T>
static cudaError_t reduce_partial_t(const void* a, const void* b, double* part, const PadParams& p,
                                    int64_t* nparts, cudaStream_t st)
{
    const int64_t cells = p.n[0] * p.n[1] * p.n[2];
    const int64_t blocks = (cells + kRedChunk - 1) / kRedChunk;
    *nparts = blocks;
    if (blocks == 0) return cudaSuccess;
    reduce_partial_kernel<T><<<(unsigned)blocks, kRedThreads, 0, st>>>((const T*)a, (const T*)b, part, p);
    return cudaGetLastError();
}

}  // namespace ebisu

#define EBISU_DEFINE_DTYPE_ENTRY(T, NAME)                                                        \
    namespace ebisu {                                                                            \
    cudaError_t tb_launch_##NAME(int d, int s, int r, int v, const TBParams& p, int g, size_t sm, \
                                 cudaStream_t st)                                                \
    {                                                                                            \
        return tb_launch_t<T>(d, s, r, v, p, g, sm, st);                                         \
    }                                                                                            \
    cudaError_t tb_occupancy_##NAME(int d, int s, int r, int v, size_t sm, int* b)               \
    {                                                                                            \
        return tb_occupancy_t<T>(d, s, r, v, sm, b);                                             \
    }                                                                                            \
    cudaError_t naive_launch_##NAME(int d, int s, int r, const void* a, void* b,                 \
                                    const NaiveParams& p, cudaStream_t st)                       \
    {                                                                                            \
        return naive_launch_t<T>(d, s, r, a, b, p, st);                                          \
    }                                                                                            \
    cudaError_t pad_copy_##NAME(const void* s, void* d0, void* d1, const PadParams& p,           \
                                cudaStream_t st)                                                 \
    {                                                                                            \
        return pad_copy_t<T>(s, d0, d1, p, st);                                                  \
    }                                                                                            \
    cudaError_t naive_vc_launch_##NAME(int d, int s, int r, const void* a, void* b, const void* f, \
                                       int64_t fs, const NaiveParams& p, cudaStream_t st)        \
    {                                                                                            \
        return naive_vc_launch_t<T>(d, s, r, a, b, f, fs, p, st);                                \
    }                                                                                            \
    cudaError_t reduce_partial_##NAME(const void* a, const void* b, double* part,                \
                                      const PadParams& p, int64_t* n, cudaStream_t st)           \
    {                                                                                            \
        return reduce_partial_t<T>(a, b, part, p, n, st);                                        \
    }                                                                                            \
    }
