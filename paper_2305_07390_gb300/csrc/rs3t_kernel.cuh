// rs3t_kernel.cuh -- register-streaming temporally blocked kernel for 3D
// radius-1 grids (7-point star, 27-point box) in FP32 or BF16 storage with
// FP32 arithmetic (temporal depth t >= 2).
//
// FP32 3D stencils are memory-bound at depth 1 (the naive kernel streams at
// the HBM rate), so they need the paper's temporal blocking (Section 4) with
// t > 1.  This kernel does it in registers, like rs_kernel.cuh in 2D:
//  * One warp owns a 64-column x 4-row output patch of the xy plane -- lane l
//    holds columns 2l, 2l+1 -- and streams it along z (N.5-D streaming).
//  * Time level s (0 = input) covers the patch's rows widened by t - s rows
//    on each side (overlapped tiling along y inside the warp, Section 2.1.2)
//    and all 64 columns (along x the valid part shrinks by one column per
//    level: strips advance by 64 - 2t columns).  Each level s < t keeps its
//    last three planes in registers (the circular multi-queue of Section
//    4.2, along z; the plane loop is unrolled three times so every queue
//    slot is a fixed register) and computes plane z - s when level 0
//    receives plane z (lag 1 per level: one warp owns the whole patch, so
//    no barrier separates the levels).
//  * x neighbours come from the adjacent lanes by warp shuffles: for the
//    star only the centre row's, for the box every row of the three planes
//    (each row shuffled once per level and step, kept while the next three
//    output rows use it); all other neighbours are in this lane's registers.
//  * Level-0 planes are staged 4 planes ahead in shared memory by per-lane
//    cp.async (each lane copies and later reads back only its own cells).
//  * Dirichlet pad cells keep their input value at every level (copied from
//    the level below); levels past the last block's depth pass values on.
//  * Tiles (strip, band, z segment) of block b wait only for their 3 x 3 x 3
//    neighbours of block b-1 (a tile's inputs reach t cells past its output,
//    at most one patch, strip or segment away).
#pragma once
#include <type_traits>

#include "common.h"
#include "stencil.cuh"

namespace ebisu {

// packed two-cell FP32 FMAs (sm_100 family) for the terms without an x offset
#ifndef EBISU_RS3T_PACKED_FMA
#define EBISU_RS3T_PACKED_FMA 1
#endif
constexpr bool kRS3TPackedFma = EBISU_RS3T_PACKED_FMA != 0;

template <class T, int SHAPE, int D>
struct RS3TGeom {
    using C = typename DT<T>::C;
    static constexpr int VX = 2;   // columns per lane
    static constexpr int TY = 4;   // output rows per warp
    static constexpr int U = 3;    // planes queued per level (2r + 1, r = 1)
    static constexpr int PFS = 4;  // level-0 planes in flight (shared memory)
    static constexpr int rows(int s) { return TY + 2 * (D - s); }  // rows of level s
    static constexpr int off(int s)  // first register of level s's queue
    {
        int o = 0;
        for (int q = 0; q < s; ++q) o += U * rows(q) * VX;
        return o;
    }
    static constexpr int RING = off(D);  // levels 0 .. D-1
    static constexpr int regs() { return RING + rows(1) * VX + (SHAPE != kStar ? 18 : 0) + 80; }
    static constexpr int minb()
    {
        const int e = (regs() + 7) & ~7;
        const int b = 65536 / (kRSThreads * e);
        return b < 1 ? 1 : (b > 8 ? 8 : b);
    }
};

// cp.async of one 4-byte element; src_size 0 writes zeros and reads nothing.
template <class T>
__device__ __forceinline__ void rs3t_cp_async(T* smem, const T* gmem, int src_size)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gmem), "r"(src_size) : "memory");
}

// Step keys of a block's levels for stochastic rounding; empty otherwise.
template <bool SR, int D>
struct RS3TStepKeys {
    __device__ __forceinline__ RS3TStepKeys(uint32_t, int) {}
};
template <int D>
struct RS3TStepKeys<true, D> {
    uint32_t k[D];
    __device__ __forceinline__ RS3TStepKeys(uint32_t plan_key, int blk)
    {
#pragma unroll
        for (int s = 1; s <= D; ++s) k[s - 1] = sr_step_key(plan_key, (uint32_t)(blk * D + s));
    }
};

template <class T, int SHAPE, int D>
__global__ void __launch_bounds__(kRSThreads, RS3TGeom<T, SHAPE, D>::minb())
    rs3t_kernel(const __grid_constant__ RS3Params prm)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 2, "FP32 or BF16 storage");
    using G = RS3TGeom<T, SHAPE, D>;
    using Dt = DT<T>;
    using C = typename Dt::C;
    using St = Stencil<3, SHAPE, 1>;
    constexpr int P = St::P;
    constexpr int VX = G::VX, TY = G::TY, U = G::U, PFS = G::PFS;
    constexpr int Y0 = G::rows(0);  // rows loaded per plane
    constexpr auto OFF = St::kOff;  // (dz, dy, dx) in canonical order
    constexpr unsigned FULL = 0xffffffffu;

    const int lane = threadIdx.x & 31;
    Control* const ctl = prm.ctl;
    const bool per = prm.periodic != 0;
    const int n0 = (int)prm.n[0], n1 = (int)prm.n[1], n2 = (int)prm.n[2];
    const int pad = prm.pad;
    const int64_t lds = prm.lds, ld1 = prm.ld1;
    const int S = prm.S, H = prm.H, nstrips = prm.nstrips, nbands = prm.nbands, nsegs = prm.nsegs;
    const long long ntiles = (long long)nstrips * nbands * nsegs;

    C ring[G::RING];
    // queue register of (level s < D, slot, row, column)
    auto Q = [&](int s, int slot, int row, int v) -> C& {
        return ring[G::off(s) + (slot * G::rows(s) + row) * VX + v];
    };
    __shared__ __align__(16) T s_stage[kRSWarps * PFS * 32 * Y0 * VX];
    T* const my_stage = s_stage + ((threadIdx.x >> 5) * PFS * 32 + lane) * (Y0 * VX);

    for (;;) {
        long long it = -1;
        if (lane == 0 && *(volatile int*)&ctl->status == 0) it = (long long)atomicAdd(&ctl->next_item, 1u);
        it = __shfl_sync(FULL, it, 0);
        if (it < 0 || it >= prm.nitems) return;
        const int blk = (int)(it / ntiles);
        const int tile = (int)(it - (long long)blk * ntiles);
        const int strip = tile % nstrips;
        const int band = (tile / nstrips) % nbands;
        const int seg = tile / (nstrips * nbands);

        // ---- wait for the 3 x 3 x 3 neighbouring tiles of the previous block ---
        int ok = 1;
        if (lane < 27 && (blk > 0 || prm.debug_stall)) {
            int sz = seg + lane / 9 - 1, sy = band + (lane / 3) % 3 - 1, sx = strip + lane % 3 - 1;
            bool exists = true;
            if (per) {
                sz = (sz + nsegs) % nsegs;
                sy = (sy + nbands) % nbands;
                sx = (sx + nstrips) % nstrips;
            } else {
                exists = sz >= 0 && sz < nsegs && sy >= 0 && sy < nbands && sx >= 0 && sx < nstrips;
            }
            if (exists) {
                const unsigned target = (unsigned)blk + (prm.debug_stall ? 1u : 0u);
                const unsigned* cnt = &ctl->done[((int64_t)sz * nbands + sy) * nstrips + sx];
                if (ld_acquire_u32(cnt) < target) {
                    const uint64_t t0 = global_ns();
                    unsigned ns = 32;
                    while (ld_acquire_u32(cnt) < target) {
                        if (*(volatile int*)&ctl->status != 0) { ok = 0; break; }
                        if (global_ns() - t0 > (uint64_t)prm.timeout_ns) {
                            atomicCAS(&ctl->status, 0, 6 /* EBISU_ERR_TIMEOUT */);
                            atomicExch(&ctl->wait_where, (unsigned)it);
                            ok = 0;
                            break;
                        }
                        __nanosleep(ns);
                        ns = ns < 1024 ? ns * 2 : ns;
                    }
                }
            }
        }
        if (!__all_sync(FULL, ok)) return;

        // ---- geometry ----------------------------------------------------------
        const bool lastb = (blk == prm.nblocks - 1);
        const int deff = lastb ? prm.depth_last : D;  // levels above deff pass values on
        const bool dst_is_out = ((prm.nblocks - 1 - blk) & 1) == 0;
        T* const dst = reinterpret_cast<T*>(dst_is_out ? prm.out : prm.ws);
        const T* const src = (blk == 0) ? reinterpret_cast<const T*>(prm.src0)
                                        : reinterpret_cast<const T*>(dst_is_out ? prm.ws : prm.out);
        const int xs = strip * S, xe = min(xs + S, n2);
        // this lane's first column (even depths: the patch starts one column
        // further left, so that with the pad of 1 a lane's pair is 8-byte
        // aligned; the host's strip width leaves room for it)
        constexpr int SH = (D % 2 == 0) ? 1 : 0;
        const int cb = xs - D - SH + VX * lane;
        const int ya = band * TY;           // first output row
        const int za = seg * H, zb = min(za + H, n0);
        const int lo0 = per ? za - D : max(za - D, -pad);
        const int hi0 = per ? zb + D : min(zb + D, n0 + pad);
        const int niter = zb + D - lo0;  // level D's last plane zb-1 arrives last
        // level-0 rows ya - D .. ya - D + Y0 - 1 and this lane's columns:
        // which exist, where they are stored
        unsigned rowok = 0, colok = 0, padc = 0, outc = 0;
#pragma unroll
        for (int i = 0; i < Y0; ++i) {
            const int y = ya - D + i;
            if (per || (y >= -pad && y < n1 + pad)) rowok |= 1u << i;
        }
#pragma unroll
        for (int v = 0; v < VX; ++v) {
            const int c = cb + v;
            if (per || (c >= -pad && c < n2 + pad)) colok |= 1u << v;
            if (!per && (c < 0 || c >= n2)) padc |= 1u << v;
            if (c >= xs && c < xe) outc |= 1u << v;
        }
        // in-plane stored offsets (32-bit: the host keeps a plane below 2^31
        // elements) of loaded row i and of this lane's column v
        int rowoff[Y0], coloff[VX];
#pragma unroll
        for (int i = 0; i < Y0; ++i) {
            int y = ya - D + i;
            if (per) y = (y < 0) ? y + n1 : (y >= n1 ? y - n1 : y);  // one wrap at most (n1 >= 16)
            rowoff[i] = (y + pad) * (int)ld1;
        }
#pragma unroll
        for (int v = 0; v < VX; ++v) {
            int c = cb + v;
            if (per) c = (c < 0) ? c + n2 : (c >= n2 ? c - n2 : c);  // one wrap at most (n2 >= 72)
            coloff[v] = c + pad;
        }
        // a lane's two columns as one copy (8 bytes FP32, 4 bytes BF16) when
        // both exist and every row starts them on a pair boundary (aligned
        // buffer, even row pitch -- hence even plane pitch -- and even column)
        // stochastic rounding (BF16-SR storage): the step keys of this block's
        // levels (an empty object for the other storage types, so that their
        // code is exactly the plain form)
        const RS3TStepKeys<Dt::kSR, D> srk(prm.sr_key, blk);
        constexpr int PB = 2 * (int)sizeof(T);  // bytes of a lane's column pair
        const bool pairs = !per && colok == 3u && ((ld1 & 1) == 0) && ((coloff[0] & 1) == 0) &&
                           ((reinterpret_cast<uintptr_t>(src) & (PB - 1)) == 0);
        auto issue_plane = [&](int slot, int z) {
            T* const sp = my_stage + slot * (32 * Y0 * VX);
            if (z < hi0) {
                const int zw = per ? ((z < 0) ? z + n0 : (z >= n0 ? z - n0 : z)) : z + pad;
                const T* const pp = src + (int64_t)zw * lds;
                if (pairs) {
#pragma unroll
                    for (int i = 0; i < Y0; ++i) {
                        const bool okr = (rowok >> i) & 1u;
                        const unsigned sa = (unsigned)__cvta_generic_to_shared(sp + i * VX);
                        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(sa),
                                     "l"(okr ? pp + (rowoff[i] + coloff[0]) : src), "n"(PB), "r"(okr ? PB : 0)
                                     : "memory");
                    }
                } else if constexpr (sizeof(T) == 2) {
                    // 2-byte cells have no cp.async form: plain loads into the
                    // lane's own slots (read back only by this thread)
                    unsigned short* const sp16 = reinterpret_cast<unsigned short*>(sp);
                    const unsigned short* const pp16 = reinterpret_cast<const unsigned short*>(pp);
#pragma unroll
                    for (int i = 0; i < Y0; ++i)
#pragma unroll
                        for (int v = 0; v < VX; ++v) {
                            const bool okc = ((rowok >> i) & (colok >> v)) & 1u;
                            sp16[i * VX + v] = okc ? __ldg(pp16 + (rowoff[i] + coloff[v])) : (unsigned short)0;
                        }
                } else {
#pragma unroll
                    for (int i = 0; i < Y0; ++i)
#pragma unroll
                        for (int v = 0; v < VX; ++v) {
                            const bool okc = ((rowok >> i) & (colok >> v)) & 1u;
                            rs3t_cp_async<T>(sp + i * VX + v, okc ? pp + (rowoff[i] + coloff[v]) : src,
                                                okc ? 4 : 0);
                        }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };

        // ---- stream along z ------------------------------------------------------
        // Every level computes a plane at every step; planes and rows outside a
        // level's region hold garbage that no kept value depends on.
#pragma unroll
        for (int q = 0; q < PFS; ++q) issue_plane(q, lo0 + q);
        for (int j0 = 0; j0 < niter; j0 += U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int zi = lo0 + j0 + u;  // plane arriving at level 0
                {
                    const int slot = (j0 + u) & (PFS - 1);
                    asm volatile("cp.async.wait_group %0;" ::"n"(PFS - 1) : "memory");
                    const T* const sp = my_stage + slot * (32 * Y0 * VX);
#pragma unroll
                    for (int i = 0; i < Y0; ++i)
#pragma unroll
                        for (int v = 0; v < VX; ++v) Q(0, u, i, v) = Dt::widen(sp[i * VX + v]);
                    issue_plane(slot, zi + PFS);
                }
#pragma unroll
                for (int s = 1; s <= D; ++s) {
                    const int zs = zi - s;                      // plane of level s computed now
                    const int cs = ((u - s) % U + U) % U;       // queue slot of plane zs
                    const int sp_ = ((u - s - 1) % U + U) % U;  // slot of plane zs - 1
                    const int sn = ((u - s + 1) % U + U) % U;   // slot of plane zs + 1
                    const int ys = ya - (D - s);  // global row of level s's row 0
                    const bool copy = (s > deff) || (!per && (zs < 0 || zs >= n0));
                    // x neighbours of level s-1 rows: WL = left lane's last
                    // column, WR = right lane's first column, per plane
                    // (0: zs-1, 1: zs, 2: zs+1) and row
                    C WL[3][G::rows(0)], WR[3][G::rows(0)];
                    auto shuffle_row = [&](int pl, int r) {
                        const int sl = pl == 0 ? sp_ : (pl == 1 ? cs : sn);
                        WL[pl][r] = __shfl_up_sync(FULL, Q(s - 1, sl, r, VX - 1), 1);
                        WR[pl][r] = __shfl_down_sync(FULL, Q(s - 1, sl, r, 0), 1);
                    };
#pragma unroll
                    for (int i = 0; i < G::rows(s); ++i) {
                        const int ib = i + 1;  // the same row in level s-1
                        if constexpr (SHAPE != kStar) {
                            // rows ib-1 .. ib+1 of all three planes; the first
                            // two were shuffled for earlier rows
                            if (i == 0) {
#pragma unroll
                                for (int pl = 0; pl < 3; ++pl) {
                                    shuffle_row(pl, 0);
                                    shuffle_row(pl, 1);
                                }
                            }
#pragma unroll
                            for (int pl = 0; pl < 3; ++pl) shuffle_row(pl, ib + 1);
                        } else {
                            shuffle_row(1, ib);  // the star: the centre row only
                        }
                        const int y = ys + i;
                        const bool prow = !per && (y < 0 || y >= n1);
                        C acc[VX];
#pragma unroll
                        for (int k = 0; k < P; ++k) {
                            const int dz = OFF.ds[k], dy = OFF.d1[k], dx = OFF.d2[k];
                            const int pl = dz + 1, r = ib + dy;
                            const int sl = pl == 0 ? sp_ : (pl == 1 ? cs : sn);
                            const C ck = prm.coef_f[k];
                            // dx = 0: the lane's pair is one register pair --
                            // both cells in one packed FMA (per-element round
                            // to nearest, the same result as two scalar FMAs)
                            if (kRS3TPackedFma && dx == 0) {
                                const float2 c2 = make_float2(ck, ck);
                                const float2 v2 = make_float2(Q(s - 1, sl, r, 0), Q(s - 1, sl, r, 1));
                                const float2 r2 = (k == 0) ? __fmul2_rn(c2, v2)
                                                           : __ffma2_rn(c2, v2, make_float2(acc[0], acc[1]));
                                acc[0] = r2.x;
                                acc[1] = r2.y;
                                continue;
                            }
#pragma unroll
                            for (int v = 0; v < VX; ++v) {
                                const int cx = v + dx;
                                const C val = (cx < 0) ? WL[pl][r] : (cx >= VX ? WR[pl][r] : Q(s - 1, sl, r, cx));
                                acc[v] = (k == 0) ? Dt::mul(ck, val) : Dt::fma(ck, val, acc[v]);
                            }
                        }
#pragma unroll
                        for (int v = 0; v < VX; ++v) {
                            const bool keep = copy || prow || ((padc >> v) & 1u);
                            C o;
                            if constexpr (Dt::kSR) {
                                // the cell's index in the stored array picks its random bits
                                const int zw = per ? ((zs < 0) ? zs + n0 : (zs >= n0 ? zs - n0 : zs)) : zs + pad;
                                const uint32_t cell = (uint32_t)((int64_t)zw * lds) + (uint32_t)rowoff[i + s] +
                                                      (uint32_t)coloff[v];
                                o = keep ? Q(s - 1, cs, ib, v) : sr_round_bf16(acc[v], cell + srk.k[s - 1]);
                            } else {
                                o = keep ? Q(s - 1, cs, ib, v) : Dt::widen(Dt::narrow(acc[v]));
                            }
                            if (s < D) {
                                Q(s < D ? s : 0, cs, i, v) = o;
                            } else if (zs >= za && zs < zb && i < TY && ya + i < n1 && ((outc >> v) & 1u)) {
                                T* const pz = dst + (per ? (int64_t)zs * lds : (int64_t)(zs + pad) * lds);
                                pz[rowoff[D + i] + coloff[v]] = Dt::narrow(o);
                            }
                        }
                    }
                }
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");  // the slots are reused by the next item

        // ---- publish completion of this tile -------------------------------------
        __threadfence();
        __syncwarp();
        if (lane == 0) red_release_add_u32(&ctl->done[tile], 1u);
    }
}

}  // namespace ebisu
