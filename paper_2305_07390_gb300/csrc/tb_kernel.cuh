// tb_kernel.cuh -- persistent temporally blocked stencil kernel (2D and 3D).
//
// What the paper's method does, and how this kernel maps it to sm_103a:
//  * Tile by tile (Section 4.1): a CTA owns one large output tile at a time
//    and runs all `depth` fused time steps of it before taking the next one;
//    tiles come from a device-wide work queue (an atomic counter), so one
//    persistent launch covers every tile of every temporal block.
//  * N.5-D streaming (Section 2.1.3): the tile is streamed along the slowest
//    axis (y in 2D, z in 3D); each streamed plane (a row in 2D) passes
//    through all time levels while it is on chip.
//  * Circular multi-queue (Section 4.2): every time level keeps a ring of
//    planes in shared memory; a plane's slot is its index modulo the ring
//    length (a compile-time constant, so the modulo is a multiply-shift).
//  * Lazy streaming (Section 4.3.2): level s lags level s-1 by r+1 planes, so
//    everything a level reads was written before the previous barrier and a
//    streamed plane costs exactly one __syncthreads.
//  * Prefetching (Section 4.3.1): input planes are copied global -> shared
//    with cp.async PF planes ahead of use (Little's law: enough bytes in
//    flight to cover the memory latency at the bandwidth the tile needs).
//  * Overlapped tiling (Section 2.1.2, SM tiling): each level computes only
//    the trapezoid it needs, shrinking by r per level, so the redundant work
//    is the paper's 1 - V_SMtile and nothing more.
//  * Dependencies between temporal blocks replace the grid barrier: an item
//    of block b waits (bounded spin on %globaltimer) until every tile of block
//    b-1 of the same problem is done.  Items are popped in order, so a wait
//    only ever targets items held by running CTAs: no deadlock and no
//    co-residency requirement.
//  * Dirichlet pads are re-imposed at every level: a pad cell of level s is
//    copied from the same position of level s-1's ring (and level 0 loaded it
//    from global memory), so no intermediate level ever computes a pad cell.
//    Periodic neighbours wrap when level 0 is loaded.
#pragma once
#include <type_traits>

#include "common.h"
#include "stencil.cuh"

namespace ebisu {

template <int R, int PF>
struct RingGeom {
    static constexpr int Q0 = 2 * R + 1 + PF;  // input ring (level 0)
    static constexpr int Q = 2 * R + 2;        // rings of levels 1 .. d-1
};

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Exact quotient i / d for 0 <= i < 2^22 and 1 <= d < 2^16 by a multiply and
// a shift: with m = ceil(2^40 / d), i*m / 2^40 exceeds i/d by less than
// i / 2^40 < 2^-18 < 1/d, so the floor is exact.  No conversion instructions.
struct Divisor {
    uint64_t m;
    int d;
};
__device__ __forceinline__ Divisor make_divisor(int d)
{
    return Divisor{((1ull << 40) + (uint64_t)d - 1) / (uint64_t)d, d};
}
__device__ __forceinline__ int fast_div(int i, const Divisor& v)
{
    return (int)(((uint64_t)(unsigned)i * v.m) >> 40);
}

enum { kLoadElem = 0, kLoadPairs = 1, kLoadStaged = 2 };

// Four consecutive ring values (16-byte aligned for float, 32-byte for double).
__device__ __forceinline__ void load_quad(const float* p, float* w)
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
__device__ __forceinline__ void load_quad(const double* p, double* w)
{
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}
// BF16: four values in one 8-byte shared load / store (8-byte aligned)
__device__ __forceinline__ void load_quad(const __nv_bfloat16* p, float* w)
{
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    w[0] = __uint_as_float(u.x << 16);
    w[1] = __uint_as_float(u.x & 0xffff0000u);
    w[2] = __uint_as_float(u.y << 16);
    w[3] = __uint_as_float(u.y & 0xffff0000u);
}
__device__ __forceinline__ void store_quad(__nv_bfloat16* p, const __nv_bfloat16* v)
{
    const unsigned a = (unsigned)__bfloat16_as_ushort(v[0]) | ((unsigned)__bfloat16_as_ushort(v[1]) << 16);
    const unsigned b = (unsigned)__bfloat16_as_ushort(v[2]) | ((unsigned)__bfloat16_as_ushort(v[3]) << 16);
    *reinterpret_cast<uint2*>(p) = make_uint2(a, b);
}
// 16-byte (FP32) / 8-byte (BF16) global store of an aligned quad
__device__ __forceinline__ void store_quad_global(float* p, const float* v)
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store_quad_global(double* p, const double* v)
{
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void store_quad_global(__nv_bfloat16* p, const __nv_bfloat16* v)
{
    const unsigned a = (unsigned)__bfloat16_as_ushort(v[0]) | ((unsigned)__bfloat16_as_ushort(v[1]) << 16);
    const unsigned b = (unsigned)__bfloat16_as_ushort(v[2]) | ((unsigned)__bfloat16_as_ushort(v[3]) << 16);
    *reinterpret_cast<uint2*>(p) = make_uint2(a, b);
}
__device__ __forceinline__ void store_quad(float* p, const float* v)
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store_quad(double* p, const double* v)
{
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// Free columns before every ring row: the 4-wide reads of the vector path
// may start up to 4 columns left of a row without leaving the slot.
constexpr int kRingMargin = 4;

// Ablation builds (the paper's Section 7.4 breakdown, measured one element
// at a time; ABL = 0 in every production build):
//   kAblNoPrefetch : each input plane is loaded and waited for in the
//                    iteration that uses it (no planes in flight ahead);
//   kAblNoLazy     : level s lags level s-1 by r planes, one barrier after
//                    every level (instead of lag r+1, one barrier per plane);
//   kAblNoRegReuse : FP32/BF16 compute one cell per thread from shared
//                    memory (no four-cells-per-thread register reuse);
//   kAblNoCircular : every queue shifts down one slot per streamed plane by
//                    copying (instead of circular indexing); implies the two
//                    above, the state the queue is introduced in.
enum { kAblNoPrefetch = 1, kAblNoLazy = 2, kAblNoRegReuse = 4, kAblNoCircular = 8 };

template <class T, int DIM, int SHAPE, int R, int NT, int ILP, int PF, int STG, int MINB, int VEC, int ABL = 0>
__global__ void __launch_bounds__(NT, MINB) tb_kernel(const __grid_constant__ TBParams prm)
{
    using St = Stencil<DIM, SHAPE, R>;
    using D = DT<T>;
    using C = typename D::C;
    constexpr int P = St::P;
    constexpr int Q0 = RingGeom<R, PF>::Q0;
    constexpr int Q = RingGeom<R, PF>::Q;
    constexpr int RP1 = St::kRP1;
    // coefficients in registers when they are few, else broadcast from shared memory
    constexpr bool kCoefRegs = (P * sizeof(typename DT<T>::C) <= (MINB >= 4 ? 40 : 128));
    constexpr auto OFF = St::kOff;
    constexpr auto ROWS = St::make_rows();
    // 4-wide path (chosen per storage type by the build, see kernels_impl.cuh)
    constexpr bool kVec = (VEC != 0) && !(ABL & kAblNoRegReuse);
    constexpr bool kShift = (ABL & kAblNoCircular) != 0;
    constexpr bool kNoPF = kShift || (ABL & kAblNoPrefetch) != 0;
    constexpr bool kNoLazy = kShift || (ABL & kAblNoLazy) != 0;
    static_assert(ABL == 0 || sizeof(T) >= 4, "ablation builds: 4- and 8-byte storage");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const ring = reinterpret_cast<T*>(smem_raw);
    __shared__ GridDesc sg;
    __shared__ C s_coef[kCoefRegs ? 1 : P];
    __shared__ int s_cmd[4];

    const int tid = threadIdx.x;
    Control* const ctl = prm.ctl;

    for (;;) {
        // ---- pop the next work item ---------------------------------------
        if (tid == 0) {
            int64_t it = -1;
            if (*(volatile int*)&ctl->status == 0) it = (int64_t)atomicAdd(&ctl->next_item, 1u);
            int g = 0, b = 0, tl = 0;
            if (it >= 0 && it < prm.nitems) {
                if (prm.items) {
                    g = prm.items[3 * it + 0];
                    b = prm.items[3 * it + 1];
                    tl = prm.items[3 * it + 2];
                } else {
                    b = (int)(it / prm.g.ntiles);
                    tl = (int)(it % prm.g.ntiles);
                }
            } else {
                it = -1;
            }
            s_cmd[0] = (it < 0) ? -1 : g;
            s_cmd[1] = b;
            s_cmd[2] = tl;
            s_cmd[3] = (int)it;
        }
        __syncthreads();
        const int gi = s_cmd[0];
        const int blk = s_cmd[1];
        const int tile = s_cmd[2];
        const int item = s_cmd[3];
        if (gi < 0) return;
        {   // copy the problem descriptor into shared memory
            const GridDesc* srcd = prm.grids ? (prm.grids + gi) : &prm.g;
            const int* w = reinterpret_cast<const int*>(srcd);
            int* dsm = reinterpret_cast<int*>(&sg);
            for (int i = tid; i < (int)(sizeof(GridDesc) / sizeof(int)); i += NT) dsm[i] = w[i];
        }
        __syncthreads();

        // ---- wait until the previous temporal block is complete -------------
        if (tid == 0) {
            int ok = 1;
            if (blk > 0 || prm.debug_stall) {
                const unsigned target = (unsigned)blk * (unsigned)sg.ntiles + (prm.debug_stall ? 1u : 0u);
                const unsigned* cnt = &ctl->done[sg.grid_id];
                if (ld_acquire_u32(cnt) < target) {
                    const uint64_t t0 = global_ns();
                    unsigned ns = 32;
                    while (ld_acquire_u32(cnt) < target) {
                        if (*(volatile int*)&ctl->status != 0) { ok = 0; break; }
                        if (global_ns() - t0 > (uint64_t)prm.timeout_ns) {
                            atomicCAS(&ctl->status, 0, 6 /* EBISU_ERR_TIMEOUT */);
                            atomicExch(&ctl->wait_where, (unsigned)item);
                            ok = 0;
                            break;
                        }
                        __nanosleep(ns);
                        ns = ns < 1024 ? ns * 2 : ns;
                    }
                }
            }
            s_cmd[0] = ok;
        }
        __syncthreads();
        if (!s_cmd[0]) return;

        // ---- geometry of this item ------------------------------------------
        const int plane_cap = sg.plane_cap > 0 ? sg.plane_cap : prm.smem_plane;  // ring plane stride
        const bool last = (blk == sg.nblocks - 1);
        const int d = last ? sg.last_depth : sg.depth;
        const bool dst_is_out = ((sg.nblocks - 1 - blk) % 2) == 0;
        T* const dst = reinterpret_cast<T*>(dst_is_out ? sg.out : sg.ws);
        const T* const src = (blk == 0) ? reinterpret_cast<const T*>(sg.src0)
                                        : reinterpret_cast<const T*>(dst_is_out ? sg.ws : sg.out);
        const bool per = sg.periodic != 0;
        const int64_t n0 = sg.n[0];
        const int n1 = (int)sg.n[1], n2 = (int)sg.n[2];
        const int pad = sg.pad;
        const int pad1 = (DIM == 3) ? pad : 0;
        const int64_t lds = sg.lds;
        const int ld1 = (int)sg.ld1;
        // 4- and 8-byte types always use element copies (compile-time)
        const int mode = (sizeof(T) == 2) ? sg.load_mode : (int)kLoadElem;
        const int t2i = tile % sg.nt[2];
        const int t1i = (tile / sg.nt[2]) % sg.nt[1];
        const int tsi = tile / (sg.nt[2] * sg.nt[1]);
        const int64_t as = (int64_t)tsi * sg.tile[0], bs = min(as + sg.tile[0], n0);
        const int a1 = t1i * sg.tile[1], b1 = min(a1 + sg.tile[1], n1);
        const int a2 = t2i * sg.tile[2], b2 = min(a2 + sg.tile[2], n2);

        // coefficients
        C cr[kCoefRegs ? P : 1];
        if constexpr (kCoefRegs) {
#pragma unroll
            for (int k = 0; k < P; ++k) cr[k] = D::coef(sg.coef[k]);
        } else {
            for (int k = tid; k < P; k += NT) s_coef[k] = D::coef(sg.coef[k]);
            __syncthreads();
        }

        // region of time level s along each axis: [a - r(d-s), b + r(d-s)),
        // clipped to the padded array for Dirichlet grids.
        auto lo_s = [&](int64_t a, int rr, int s, int padax) -> int64_t {
            const int64_t v = a - (int64_t)rr * (d - s);
            return per ? v : max(v, (int64_t)-padax);
        };
        auto hi_s = [&](int64_t b, int64_t n, int rr, int s, int padax) -> int64_t {
            const int64_t v = b + (int64_t)rr * (d - s);
            return per ? v : min(v, n + padax);
        };
        const int64_t slo0 = lo_s(as, R, 0, pad), shi0 = hi_s(bs, n0, R, 0, pad);
        const int lo01 = (int)lo_s(a1, RP1, 0, pad1), hi01 = (int)hi_s(b1, n1, RP1, 0, pad1);
        const int lo02 = (int)lo_s(a2, R, 0, pad), hi02 = (int)hi_s(b2, n2, R, 0, pad);
        const int E1 = hi01 - lo01, E2 = hi02 - lo02;
        // ring row: kRingMargin free columns, the row (+1 for the pair-load
        // shift), then room for the 4-wide reads of the vector path (up to
        // 7 columns past the row's last quad start); multiple of 4
        const int E2p = (E2 + kRingMargin + 7 + 3) & ~3;
        const int plane0 = E1 * E2;
        if (E1 * E2p > plane_cap || (mode == kLoadStaged && plane0 > STG * NT)) {
            if (tid == 0) atomicCAS(&ctl->status, 0, 7 /* EBISU_ERR_DEVICE_FAULT */);
            return;
        }
        const Divisor divE2 = make_divisor(E2);
        const int safe_off = (E1 / 2) * E2p + E2 / 2;  // >= R away from every plane edge

        // stored element offset of (ps, q1, q2), interior coordinates
        auto gplane = [&](int64_t ps) -> int64_t {
            if (per) return wrap_idx(ps, n0) * lds;
            return (ps + pad) * lds;
        };
        auto ginplane = [&](int q1, int q2) -> int64_t {
            if (per) {
                const int64_t y = (DIM == 3) ? wrap_idx(q1, n1) : 0;
                return y * ld1 + wrap_idx(q2, n2);
            }
            return (int64_t)(q1 + pad1) * ld1 + (q2 + pad);
        };
        // plane of level s streamed at iteration j is slo0 + j - lag(s)
        auto lag = [&](int s) -> int64_t {
            if constexpr (kNoLazy) return (int64_t)R * s;
            return s == 0 ? 0 : (int64_t)R + (int64_t)(s - 1) * (R + 1);
        };
        int64_t jcur = 0;  // the streaming iteration (shifting queues only)
        // ring slot of plane ps at level lev (0 = input ring)
        auto ring_plane = [&](int lev, int64_t ps) -> T* {
            if constexpr (kShift) {
                // the newest plane of a level sits in its last slot
                const int qq = (lev == 0) ? Q0 : Q;
                const int slot = qq - 1 - (int)(slo0 + jcur - lag(lev) - ps);
                if (lev == 0) return ring + (size_t)slot * plane_cap + kRingMargin;
                return ring + ((size_t)Q0 + (size_t)(lev - 1) * Q + slot) * plane_cap + kRingMargin;
            }
            const unsigned rel = (unsigned)(ps - slo0);
            if (lev == 0) return ring + (size_t)(rel % Q0) * plane_cap + kRingMargin;
            return ring + ((size_t)Q0 + (size_t)(lev - 1) * Q + (rel % Q)) * plane_cap + kRingMargin;
        };
        // shift of a level-0 plane in pair-load mode: parity of its first
        // stored element (every row of a plane shares it, see host checks)
        auto pshift = [&](int64_t ps) -> int {
            if (mode != kLoadPairs) return 0;
            return (int)((gplane(ps) + ginplane(lo01, lo02)) & 1);
        };

        // ---- first temporal block: fill the Dirichlet pads of the buffers ---
        if (blk == 0 && !per && (sg.halo_dst0 || sg.halo_dst1)) {
            T* h0 = reinterpret_cast<T*>(sg.halo_dst0);
            T* h1 = reinterpret_cast<T*>(sg.halo_dst1);
            const T* s0 = reinterpret_cast<const T*>(sg.src0);
            const bool t12 = (DIM == 3 && (a1 == 0 || b1 == n1)) || a2 == 0 || b2 == n2;
            const bool touches = (as == 0) || (bs == n0) || t12;
            if (touches) {
                const int64_t xs0 = (as == 0) ? -pad : as, xs1 = (bs == n0) ? n0 + pad : bs;
                const int x10 = (a1 == 0) ? -pad1 : a1, x11 = (b1 == n1) ? n1 + pad1 : b1;
                const int x20 = (a2 == 0) ? -pad : a2, x21 = (b2 == n2) ? n2 + pad : b2;
                const int w1 = x11 - x10, w2 = x21 - x20;
                for (int64_t ps = xs0; ps < xs1; ++ps) {
                    const bool hp = (ps < 0 || ps >= n0);
                    if (!hp && !t12) continue;
                    const int64_t pb = gplane(ps);
                    for (int i = tid; i < w1 * w2; i += NT) {
                        const int q1 = x10 + i / w2, q2 = x20 + i % w2;
                        if (!(hp || q1 < 0 || q1 >= n1 || q2 < 0 || q2 >= n2)) continue;
                        const int64_t g = pb + ginplane(q1, q2);
                        const T v = D::raw(s0 + g);
                        if (h0) h0[g] = v;
                        if (h1) h1[g] = v;
                    }
                }
            }
        }

        // ---- level-0 plane loads --------------------------------------------
        // Element mode: one cp.async per element (any alignment, wraps).
        // Pair mode (2-byte types): 4-byte cp.async of aligned element pairs;
        //   the plane is stored shifted by the parity of its first element.
        // Staged mode: registers, loaded one iteration ahead (fallback).
        constexpr int kStg = (sizeof(T) == 2) ? STG : 1;
        T stage[kStg];
        auto issue_plane = [&](int64_t ps) {
            T* rp = ring_plane(0, ps);
            const int64_t pb = gplane(ps);
            if (mode == kLoadElem) {
                for (int i = tid; i < plane0; i += NT) {
                    const int r1 = (DIM == 3) ? fast_div(i, divE2) : 0;
                    const int c2 = i - r1 * E2;
                    cp_async(rp + r1 * E2p + c2, src + pb + ginplane(lo01 + r1, lo02 + c2), (int)sizeof(T));
                }
            } else if (mode == kLoadPairs) {
                const int sh = pshift(ps);
                const int npair = (E2 + sh + 1) >> 1;
                const int64_t last_elem = sg.total_elems - 1;
                for (int i = tid; i < E1 * npair; i += NT) {
                    const int r1 = (DIM == 3) ? i / npair : 0;
                    const int k = i - r1 * npair;
                    const int64_t g0 = pb + ginplane(lo01 + r1, lo02) - sh + 2 * k;
                    T* sp = rp + r1 * E2p + 2 * k;
                    if (g0 + 1 <= last_elem) {
                        cp_async(sp, src + g0, 4);
                    } else {
                        sp[0] = D::raw(src + g0);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < kStg; ++k) {
                    const int i = tid + k * NT;
                    if (i < plane0) {
                        const int r1 = (DIM == 3) ? fast_div(i, divE2) : 0;
                        const int c2 = i - r1 * E2;
                        stage[k] = D::raw(src + pb + ginplane(lo01 + r1, lo02 + c2));
                    }
                }
            }
        };
        auto finish_staged = [&](int64_t ps) {
            T* rp = ring_plane(0, ps);
#pragma unroll
            for (int k = 0; k < kStg; ++k) {
                const int i = tid + k * NT;
                if (i < plane0) {
                    const int r1 = (DIM == 3) ? fast_div(i, divE2) : 0;
                    rp[r1 * E2p + (i - r1 * E2)] = stage[k];
                }
            }
        };

        // ---- one plane of time level s (1 <= s <= d) ---------------------------
        auto compute_plane = [&](int s, int64_t ps) {
            const int l1 = (int)lo_s(a1, RP1, s, pad1), h1 = (int)hi_s(b1, n1, RP1, s, pad1);
            const int l2 = (int)lo_s(a2, R, s, pad), h2 = (int)hi_s(b2, n2, R, s, pad);
            const int R2 = h2 - l2;
            const int cnt = (h1 - l1) * R2;
            const Divisor divR2 = make_divisor(R2);
            const bool to_global = (s == d);
            T* const outp = to_global ? nullptr : ring_plane(s, ps);
            T* const gout = to_global ? dst + gplane(ps) : nullptr;
            const int sh_c = (s == 1) ? pshift(ps) : 0;
            const T* const self = ring_plane(s - 1, ps) + sh_c;
            const bool pad_plane = !per && (ps < 0 || ps >= n0);
            // any pad cell in this plane's region?
            const bool edge = !per && (pad_plane || l1 < 0 || h1 > n1 || l2 < 0 || h2 > n2);
            if (pad_plane) {  // keep the input values: copy from the level below
                for (int i = tid; i < cnt; i += NT) {
                    const int r1 = (DIM == 3) ? fast_div(i, divR2) : 0;
                    const int off = (l1 + r1 - lo01) * E2p + (l2 + (i - r1 * R2) - lo02);
                    outp[off] = self[off];
                }
                return;
            }
            const T* base[2 * R + 1];
#pragma unroll
            for (int k = 0; k < 2 * R + 1; ++k) {
                const int64_t pk = ps + k - R;
                base[k] = ring_plane(s - 1, pk) + ((s == 1) ? pshift(pk) : 0);
            }
            // cell index i -> (q1, q2) of this level's region
            auto cell = [&](int i, int& q1, int& q2) {
                const int r1 = (DIM == 3) ? fast_div(i, divR2) : 0;
                q1 = l1 + r1;
                q2 = l2 + (i - r1 * R2);
            };
            auto is_pad = [&](int q1, int q2) -> bool {
                return edge && (q1 < 0 || q1 >= n1 || q2 < 0 || q2 >= n2);
            };
            // U cells per thread, slots i0, i0 + NT, ... (U is compile-time)
            auto group = [&](auto UC, int i0) {
                constexpr int U = decltype(UC)::value;
                int rd[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * NT;
                    int q1, q2;
                    cell(i < cnt ? i : 0, q1, q2);
                    const bool comp = (i < cnt) && !is_pad(q1, q2);
                    rd[u] = comp ? (q1 - lo01) * E2p + (q2 - lo02) : safe_off;
                }
                C acc[U];
                {
                    const C c0 = kCoefRegs ? cr[0] : s_coef[0];
                    const T* bp = base[OFF.ds[0] + R] + OFF.d1[0] * E2p + OFF.d2[0];
#pragma unroll
                    for (int u = 0; u < U; ++u) acc[u] = D::mul(c0, D::widen(bp[rd[u]]));
                }
#pragma unroll
                for (int k = 1; k < P; ++k) {
                    const C ck = kCoefRegs ? cr[k] : s_coef[k];
                    const T* bp = base[OFF.ds[k] + R] + OFF.d1[k] * E2p + OFF.d2[k];
#pragma unroll
                    for (int u = 0; u < U; ++u) acc[u] = D::fma(ck, D::widen(bp[rd[u]]), acc[u]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * NT;
                    if (i >= cnt) continue;
                    int q1, q2;
                    cell(i, q1, q2);
                    const int off = (q1 - lo01) * E2p + (q2 - lo02);
                    const bool pc = is_pad(q1, q2);
                    const T v = pc ? self[off] : D::narrow(acc[u]);
                    if (to_global) {
                        if (!pc) gout[ginplane(q1, q2)] = v;
                    } else {
                        outp[off] = v;
                    }
                }
            };
            static_assert(ILP == 4 || ILP == 8, "slot dispatch below handles ILP 4 and 8");
            for (int i0 = tid; i0 < cnt; i0 += ILP * NT) {
                // slots that hold at least one cell of this warp (warp-uniform),
                // so a short last pass issues no FMAs for empty slots
                const int wbase = i0 - (tid & 31);
                const int uw = min(ILP, (cnt - wbase + NT - 1) / NT);
                if (uw >= ILP)
                    group(std::integral_constant<int, ILP>{}, i0);
                else if (ILP == 8 && uw > 4)
                    group(std::integral_constant<int, (ILP == 8 ? 6 : 1)>{}, i0);
                else if (uw >= 3)
                    group(std::integral_constant<int, (ILP == 8 ? 4 : 3)>{}, i0);
                else if (uw == 2)
                    group(std::integral_constant<int, 2>{}, i0);
                else
                    group(std::integral_constant<int, 1>{}, i0);
            }
        };


        // ---- four consecutive cells per thread (FP32 and BF16 storage) ---------
        // Each thread owns ring columns [4j, 4j+4) of a row and reads its
        // neighbourhood as aligned 4-wide shared loads (one per needed quad of
        // each stencil row), selecting neighbours from registers; the FMA
        // chain of every cell is the canonical one, so results are identical
        // to the scalar path and to the naive kernel.
        auto compute_plane_vec = [&](int s, int64_t ps) {
            const int l1 = (int)lo_s(a1, RP1, s, pad1), h1 = (int)hi_s(b1, n1, RP1, s, pad1);
            const int l2 = (int)lo_s(a2, R, s, pad), h2 = (int)hi_s(b2, n2, R, s, pad);
            const int c0 = l2 - lo02, c1 = h2 - lo02;  // ring columns of the region
            const int jq0 = c0 >> 2, nq = ((c1 - 1) >> 2) - jq0 + 1;
            const int items = (h1 - l1) * nq;
            const Divisor divnq = make_divisor(nq);
            const bool to_global = (s == d);
            T* const outp = to_global ? nullptr : ring_plane(s, ps);
            T* const gout = to_global ? dst + gplane(ps) : nullptr;
            const T* const self = ring_plane(s - 1, ps);
            const bool pad_plane = !per && (ps < 0 || ps >= n0);
            const bool edge = !per && (pad_plane || l1 < 0 || h1 > n1 || l2 < 0 || h2 > n2);
            const T* base[2 * R + 1];
            int shk[2 * R + 1];  // pair-load shift of each input plane (level 1, 2-byte storage)
#pragma unroll
            for (int k = 0; k < 2 * R + 1; ++k) {
                base[k] = ring_plane(s - 1, ps + k - R);
                shk[k] = (s == 1) ? pshift(ps + k - R) : 0;
            }
            const int sh_self = (sizeof(T) == 2 && s == 1) ? pshift(ps) : 0;
            for (int it = tid; it < items; it += NT) {
                const int r1 = (DIM == 3) ? fast_div(it, divnq) : 0;
                const int cb = 4 * (jq0 + it - r1 * nq);  // ring column of the first cell
                const int q1 = l1 + r1;
                const int rowoff = (q1 - lo01) * E2p;
                C acc[4];
                // a pad row of a 3D plane keeps its input values; its
                // neighbour rows may lie outside the ring, so read nothing
                const bool pad_row = !per && DIM == 3 && (q1 < 0 || q1 >= n1);
                if (!pad_plane && !pad_row) {
                    C w[12];
#pragma unroll
                    for (int k = 0; k < P; ++k) {
                        // a shifted plane (sh = 1) holds column c at c + 1
                        const int sh = (sizeof(T) == 2) ? shk[OFF.ds[k] + R] : 0;
                        if (ROWS.start[k]) {
                            const T* rp = base[OFF.ds[k] + R] + rowoff + OFF.d1[k] * E2p + cb;
                            load_quad(rp, w + 4);
                            if (ROWS.min_d2[k] < 0) load_quad(rp - 4, w);
                            if (ROWS.max_d2[k] > 0 || sh) load_quad(rp + 4, w + 8);
                        }
                        const C ck = kCoefRegs ? cr[k] : s_coef[k];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const C v = sh ? w[5 + m + OFF.d2[k]] : w[4 + m + OFF.d2[k]];
                            acc[m] = (k == 0) ? D::mul(ck, v) : D::fma(ck, v, acc[m]);
                        }
                    }
                }
                // Interior quad (the common case): all four cells inside the
                // region, no pad cell, one contiguous run in global memory.
                const bool inner = (cb >= c0) && (cb + 4 <= c1) && !edge &&
                                   (!per || (lo02 + cb >= 0 && lo02 + cb + 4 <= n2 && q1 >= 0 && q1 < n1));
                if (inner) {
                    T res[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) res[m] = D::narrow(acc[m]);
                    if (to_global) {
                        T* gp = gout + ginplane(q1, lo02 + cb);
                        if ((reinterpret_cast<uintptr_t>(gp) & (4 * sizeof(T) - 1)) == 0) {
                            store_quad_global(gp, res);
                        } else {
#pragma unroll
                            for (int m = 0; m < 4; ++m) gp[m] = res[m];
                        }
                    } else {
                        store_quad(outp + rowoff + cb, res);
                    }
                    continue;
                }
                // general quad: cells outside the region are skipped, pad cells
                // keep the level below's value
                T res[4];
                bool keep[4], padc[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int col = cb + m;
                    const int q2 = lo02 + col;
                    keep[m] = (col >= c0) && (col < c1);
                    padc[m] = edge && (pad_plane || q1 < 0 || q1 >= n1 || q2 < 0 || q2 >= n2);
                    res[m] = padc[m] ? self[rowoff + col + sh_self] : D::narrow(acc[m]);
                }
                if (to_global) {
                    // per-cell addresses: on periodic grids a quad may straddle
                    // the wrap, so its cells are not one contiguous run
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (keep[m] && !padc[m]) gout[ginplane(q1, lo02 + cb + m)] = res[m];
                } else {
                    T* op = outp + rowoff + cb;
                    if (keep[0] && keep[3]) {
                        store_quad(op, res);
                    } else {
#pragma unroll
                        for (int m = 0; m < 4; ++m)
                            if (keep[m]) op[m] = res[m];
                    }
                }
            }
        };

        // ---- stream the tile ----------------------------------------------------
        const int64_t lastp = bs - 1;  // last plane of level d
        const int64_t niter = lastp - slo0 + lag(d) + 1;
        if constexpr (kNoPF) {
            // ablation: planes are loaded in the iteration that uses them
#pragma unroll 1
            for (int64_t j = 0; j < niter; ++j) {
                jcur = j;
                const int64_t pcur = slo0 + j;
                if (pcur < shi0) issue_plane(pcur);
                cp_async_commit();
                cp_async_wait<0>();
                __syncthreads();
                for (int s = 1; s <= d; ++s) {
                    const int64_t ps = slo0 + j - lag(s);
                    if (ps >= lo_s(as, R, s, pad) && ps < hi_s(bs, n0, R, s, pad)) {
                        if constexpr (kVec)
                            compute_plane_vec(s, ps);
                        else
                            compute_plane(s, ps);
                    }
                    if (kNoLazy && s < d) __syncthreads();
                }
                if constexpr (kShift) {
                    // every queue moves down one slot (slot k+1 -> k)
                    __syncthreads();
                    for (int lev = 0; lev < d; ++lev) {
                        const int qq = (lev == 0) ? Q0 : Q;
                        T* const base = (lev == 0) ? ring : ring + ((size_t)Q0 + (size_t)(lev - 1) * Q) * plane_cap;
                        for (int i = tid; i < plane_cap; i += NT)
                            for (int k = 0; k + 1 < qq; ++k) base[(size_t)k * plane_cap + i] = base[(size_t)(k + 1) * plane_cap + i];
                    }
                }
                __syncthreads();
            }
        } else if (mode != kLoadStaged) {
            // prologue: PF planes in flight, one commit group each
#pragma unroll 1
            for (int k = 0; k < PF; ++k) {
                if (slo0 + k < shi0) issue_plane(slo0 + k);
                cp_async_commit();
            }
        } else {
            issue_plane(slo0);
            finish_staged(slo0);
        }
        for (int64_t j = 0; j < (kNoPF ? 0 : niter); ++j) {
            if (mode != kLoadStaged) cp_async_wait<PF - 1>();
            __syncthreads();
            const int64_t pnext = slo0 + j + ((mode != kLoadStaged) ? PF : 1);
            const bool have_next = pnext < shi0;
            if (mode != kLoadStaged) {
                if (have_next) issue_plane(pnext);
                cp_async_commit();
            } else if (have_next) {
                issue_plane(pnext);
            }
            for (int s = 1; s <= d; ++s) {
                const int64_t ps = slo0 + j - lag(s);
                if (ps >= lo_s(as, R, s, pad) && ps < hi_s(bs, n0, R, s, pad)) {
                    if constexpr (kVec)
                        compute_plane_vec(s, ps);
                    else
                        compute_plane(s, ps);
                }
                if (kNoLazy && s < d) __syncthreads();  // ablation: a barrier per level
            }
            if (mode == kLoadStaged && have_next) finish_staged(pnext);
        }
        if (mode != kLoadStaged) cp_async_wait<0>();

        // ---- publish completion ---------------------------------------------
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            red_release_add_u32(&ctl->done[sg.grid_id], 1u);
        }
    }
}

}  // namespace ebisu
