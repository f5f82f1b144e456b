// rs_kernel.cuh -- register-streaming temporally blocked kernel (2D grids).
//
// The same method as tb_kernel.cuh (t Jacobi steps fused per temporal block,
// tile by tile, the tile streamed along y and every time level kept on chip,
// Sections 2.1 and 4), with the on-chip storage moved from shared memory to
// registers and the tile narrowed to what one warp holds:
//  * One warp owns a strip of 128 columns (lane l holds columns 4l .. 4l+3)
//    and streams it down a segment of rows.  Each time level s < t keeps its
//    last 2r+1 rows in registers (the circular multi-queue of Section 4.2,
//    one queue per level, indexed by row mod 2r+1; the row loop is unrolled
//    2r+1 times so every queue index is a compile-time register name).
//  * Level s computes row y - s*r when level 0 receives row y: with one warp
//    per strip no barrier separates the levels, so the lag is r per level
//    (the shared-memory kernel needs r+1 to hide its per-plane barrier).
//  * Horizontal neighbours come from the adjacent lanes by warp shuffles:
//    star stencils shuffle the r edge cells of the centre row when they use
//    it; box stencils keep every queued row widened by r cells per side,
//    shuffled once when the row is produced.
//  * Overlapped tiling (Section 2.1.2) at warp granularity: the valid part of
//    a strip shrinks by r columns per level and side, so strips advance by
//    S = 128 - 2*t*r columns; rows overlap the same way along y.
//  * Level-0 rows are loaded PF rows ahead into registers (Section 4.3.1's
//    prefetching, without a shared-memory stage).
//  * Tiles of block b wait only for the (up to) eight neighbouring tiles of
//    block b-1 -- the tiles whose outputs their inputs overlap -- through one
//    completion counter per tile.  Those are also the only tiles of block b-1
//    that read the region a tile of block b overwrites in the ping-pong
//    buffer, so the same wait orders both hazards.  Items are popped in
//    (block, tile) order and every warp of the grid is resident, so a wait
//    only targets items already held by running warps: no deadlock.
//  * Dirichlet pad cells keep their input value at every level (copied from
//    the level below); periodic neighbours wrap when level 0 is loaded.
#pragma once
#include <type_traits>

#include "common.h"
#include "stencil.cuh"

namespace ebisu {

// packed two-cell FP32 FMAs (sm_100 family) in the register-streaming kernel
#ifndef EBISU_RS_PACKED_FMA
#define EBISU_RS_PACKED_FMA 1
#endif
constexpr bool kRSPackedFma = EBISU_RS_PACKED_FMA != 0;

template <class T, int SHAPE, int R>
struct RSGeom {
    using C = typename DT<T>::C;
    static constexpr int U = 2 * R + 1;                       // rows queued per level
    static constexpr bool EXT = (SHAPE == kBox);              // rows stored with halo
    static constexpr int RW = EXT ? 4 + 2 * R : 4;            // values per queued row
    // Level-0 rows in flight.  PFS rows staged in shared memory by cp.async
    // (each lane copies and later reads back only its own columns, so no
    // barrier is needed).  2-byte storage is below cp.async's 4-byte
    // minimum, so a BF16 lane copies the 4-byte-aligned pairs covering its
    // columns (one pair more than it needs) and reads back from the row's
    // parity.  The 25-point box (measured faster with its 5 rows in
    // registers): PF rows in registers (PF divides U).
    static constexpr bool ASYNC = !(EXT && R == 2);
    static constexpr int SW = (sizeof(T) == 2) ? RW + 2 : RW;  // elements of a lane's staging slot
    static constexpr int PFS = (sizeof(T) == 8) ? 4 : 8;
    static constexpr int PF = ASYNC ? 1 : ((sizeof(C) == 8) ? 1 : U);
    static constexpr int WORDS = (int)sizeof(C) / 4;
    // registers a thread needs at depth D: the queues, the rows in flight,
    // the star's widened centre row, the accumulators, and about 56 for
    // addresses, loop state and the item's geometry (the 25-point box keeps
    // more of its rows' values live across its 100 FMAs: found by compiling)
    static constexpr int P = Stencil<2, SHAPE, R>::P;
    static constexpr bool SR = DT<T>::kSR;  // stochastic rounding: step keys and a column key
    static constexpr int regs(int D, bool batch)
    {
        return (D * U * RW + (ASYNC ? 0 : PF * RW) + (EXT ? 0 : 4 + 2 * R) + 4 + (batch ? P : 0)) * WORDS + 56 +
               ((EXT && R == 2) ? 48 : 0) + (batch ? 16 : 0) + (SR ? D + 4 : 0);
    }
    static constexpr int minb(int D, bool batch)
    {
        const int e = (regs(D, batch) + 7) & ~7;
        const int b = 65536 / (kRSThreads * e);
        return b < 1 ? 1 : (b > 8 ? 8 : b);
    }
};

// cp.async of one 4- or 8-byte element; src_size 0 writes zeros and reads nothing.
template <int BYTES>
__device__ __forceinline__ void rs_cp_async(void* smem, const void* gmem, int src_size)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(sa), "l"(gmem), "n"(BYTES), "r"(src_size)
                 : "memory");
}
__device__ __forceinline__ void rs_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void rs_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class T, int SHAPE, int R, int D, bool BATCH>
__global__ void __launch_bounds__(kRSThreads, RSGeom<T, SHAPE, R>::minb(D, BATCH))
    rs_kernel(const __grid_constant__ RSParams prm)
{
    using G = RSGeom<T, SHAPE, R>;
    using Dt = DT<T>;
    using C = typename Dt::C;
    using St = Stencil<2, SHAPE, R>;
    constexpr int P = St::P;
    constexpr int U = G::U;
    constexpr int RW = G::RW;
    constexpr int PF = G::PF;
    constexpr bool EXT = G::EXT;
    constexpr int X0 = EXT ? R : 0;  // position of cell 0 in a queued row
    constexpr auto OFF = St::kOff;   // ds = row offset, d2 = column offset
    static_assert(U % PF == 0, "prefetch slots must divide the unrolled row count");
    static_assert(R <= 3 && 2 * D * R < kRSCols, "strip too narrow for this depth");
    constexpr unsigned FULL = 0xffffffffu;

    const int lane = threadIdx.x & 31;
    Control* const ctl = prm.ctl;
    // coefficients: in the parameter bank for a single problem (FMAs take
    // them as operands), in registers (loaded per item) for a batch
    C cr[BATCH ? P : 1] = {};
    auto coef = [&](int k) -> C {
        if constexpr (BATCH) return cr[k];
        else if constexpr (sizeof(C) == 8) return prm.g.coef[k];
        else return prm.g.coef_f[k];
    };

    constexpr bool ASYNC = G::ASYNC;
    constexpr int PFS = G::PFS;
    C ring[D][U][RW];                 // levels 0 .. D-1; level D goes to global memory
    C stage[ASYNC ? 1 : PF][RW];      // level-0 rows in flight (registers)
    // level-0 rows in flight (shared memory): [warp][slot][lane][column]
    constexpr int SW = G::SW;
    __shared__ __align__(16) T s_stage[ASYNC ? kRSWarps * PFS * 32 * SW : 1];
    T* const my_stage = s_stage + (ASYNC ? ((threadIdx.x >> 5) * PFS * 32 + lane) * SW : 0);

    for (;;) {
        // ---- pop an item: (problem, temporal block, tile) ---------------------
        long long it = -1;
        int gi = 0, blk = 0, tile = 0;
        if (lane == 0 && *(volatile int*)&ctl->status == 0) it = (long long)atomicAdd(&ctl->next_item, 1u);
        it = __shfl_sync(FULL, it, 0);
        if (it < 0 || it >= prm.nitems) return;
        if constexpr (BATCH) {
            int v = 0;
            if (lane < 3) v = prm.items[3 * it + lane];
            gi = __shfl_sync(FULL, v, 0);
            blk = __shfl_sync(FULL, v, 1);
            tile = __shfl_sync(FULL, v, 2);
        } else {
            const long long ntiles = (long long)prm.g.nstrips * prm.g.nsegs;
            blk = (int)(it / ntiles);
            tile = (int)(it - (long long)blk * ntiles);
        }
        const RSGrid* const gd = BATCH ? prm.grids + gi : &prm.g;
        const bool per = gd->periodic != 0;
        const int64_t n0 = gd->n0;
        const int n2 = gd->n2;
        const int pad = gd->pad;
        const int64_t lds = gd->lds;
        const int S = gd->S, H = gd->H, nstrips = gd->nstrips, nsegs = gd->nsegs, nblocks = gd->nblocks;
        unsigned* const done = &ctl->done[gd->tile_base];
        if constexpr (BATCH) {
#pragma unroll
            for (int k = 0; k < P; ++k) {
                if constexpr (sizeof(C) == 8) cr[k] = gd->coef[k];
                else cr[k] = gd->coef_f[k];
            }
        }
        const int seg = tile / nstrips;
        const int strip = tile - seg * nstrips;

        // ---- wait for the neighbouring tiles of the previous block -------------
        // lanes 0..8 each watch one of the 3 x 3 neighbours (bounded waits)
        int ok = 1;
        if (lane < 9 && (blk > 0 || prm.debug_stall)) {
            int sg = seg + lane / 3 - 1, sx = strip + lane % 3 - 1;
            bool exists = true;
            if (per) {
                sg = (sg + nsegs) % nsegs;
                sx = (sx + nstrips) % nstrips;
            } else {
                exists = sg >= 0 && sg < nsegs && sx >= 0 && sx < nstrips;
            }
            if (exists) {
                const unsigned target = (unsigned)blk + (prm.debug_stall ? 1u : 0u);
                const unsigned* cnt = &done[(int64_t)sg * nstrips + sx];
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

        // ---- geometry ------------------------------------------------------------
        const bool lastb = (blk == nblocks - 1);
        const int deff = lastb ? gd->depth_last : D;  // levels above deff pass values through
        const bool dst_is_out = ((nblocks - 1 - blk) & 1) == 0;
        T* const dst = reinterpret_cast<T*>(dst_is_out ? gd->out : gd->ws);
        const T* const src = (blk == 0) ? reinterpret_cast<const T*>(gd->src0)
                                        : reinterpret_cast<const T*>(dst_is_out ? gd->ws : gd->out);
        const int xs = strip * S;              // first output column of the strip
        const int xe = min(xs + S, n2);        // end of the output columns
        const int cb = xs - D * R + 4 * lane;  // column of this lane's cell 0
        // rows (int: the host keeps n0 + 2 * pad below 2^31)
        const int ya = seg * H;
        const int yb = min(ya + H, (int)n0);
        const int n0i = (int)n0;
        // rows of level s: [ya - r(D-s), yb + r(D-s)), clipped to the padded
        // grid; level 0 is loaded over [lo0, hi0)
        const int lo0 = per ? ya - R * D : max(ya - R * D, -pad);
        const int hi0 = per ? yb + R * D : min(yb + R * D, n0i + pad);
        const int niter = yb + D * R - lo0;  // level D's last row arrives last

        // ---- first temporal block: give the buffers later blocks write the
        // input's Dirichlet pad (this tile's share: the pad cells next to its
        // output region).  A tile of block 1 that reads such a cell reaches
        // at most t*r cells past its own output, so the writer is one of the
        // 3 x 3 neighbours it waits for.
        if (blk == 0 && !per && (gd->pad_dst0 || gd->pad_dst1)) {
            const bool fs = strip == 0, ls = strip == nstrips - 1, fg = seg == 0, lg = seg == nsegs - 1;
            if (fs || ls || fg || lg) {
                const T* const s0 = reinterpret_cast<const T*>(gd->src0);
                T* const h0 = reinterpret_cast<T*>(gd->pad_dst0);
                T* const h1 = reinterpret_cast<T*>(gd->pad_dst1);
                const int x0 = fs ? -pad : xs, x1 = ls ? n2 + pad : xe;
                const int y0 = fg ? -pad : ya, y1 = lg ? (int)n0 + pad : yb;
                auto copy_cell = [&](int y, int c) {
                    const int64_t g = (int64_t)(y + pad) * lds + (c + pad);
                    const T v = Dt::raw(s0 + g);
                    if (h0) h0[g] = v;
                    if (h1) h1[g] = v;
                };
                for (int y = y0; y < y1; ++y) {
                    if (y < 0 || y >= (int)n0) {  // a pad row: all of the tile's columns
                        for (int c = x0 + lane; c < x1; c += 32) copy_cell(y, c);
                    } else {                      // an interior row: its pad columns
                        if (fs && lane < pad) copy_cell(y, -pad + lane);
                        if (ls && lane < pad) copy_cell(y, n2 + lane);
                    }
                }
            }
        }

        // loaded columns cb - X0 .. cb - X0 + RW - 1: which exist (Dirichlet:
        // inside the padded row), and whether they are one contiguous run
        // (periodic: no wrap inside this lane's columns)
        const int c0 = cb - X0;
        unsigned lvm = 0;
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            const int c = c0 + q;
            if (per || ((c >= -pad) && (c < n2 + pad))) lvm |= 1u << q;
        }
        const int cw0 = per ? (c0 < 0 ? c0 + n2 : (c0 >= n2 ? c0 - n2 : c0)) : 0;  // wrapped c0
        const bool contig = cw0 + RW <= n2;
        unsigned padm = 0, outm = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int c = cb + m;
            if (!per && (c < 0 || c >= n2)) padm |= 1u << m;
            if (c >= xs && c < xe) outm |= 1u << m;
        }
        // Most tiles touch no boundary and belong to a full-depth block.  For
        // the short FP32/BF16 stencils (5 and 9 points) those run a lean copy
        // of the loop without pad, copy or wrap handling; everything else
        // runs the general loop.  For FP64 (FMA-pipe bound) and the 13- and
        // 25-point stencils a second copy of the loop only costs registers
        // (measured).  Each copy's row body is branch-free, so the compiler
        // can interleave the levels' instructions freely.
        constexpr bool kLean = (sizeof(C) == 4) && (P <= 9);
        bool general = true;
        if constexpr (kLean) {
            const bool lane_edge = per ? !contig : (padm != 0u || lvm != (1u << RW) - 1u);
            // (the last block needs the pass-through copies only when it is shallower)
            general = __any_sync(FULL, lane_edge) || (lastb && gd->depth_last < D) ||
                      (!per && (ya - R * D < 0 || yb + R * D > n0i));
        }

        // 2-byte storage: every pair copy of this tile lies inside the array
        // when the tile is Dirichlet, loads interior rows only and every
        // lane's columns lie inside the padded row (the copies then start at
        // (y+pad)*lds - 1 >= 0 and end at most one element into the next
        // stored row), so its copies need no bounds checks
        bool stage_in = false;
        if constexpr (sizeof(T) == 2) {
            stage_in = !per && !__any_sync(FULL, lvm != (1u << RW) - 1u) && ya - R * D >= 0 &&
                       yb + R * D <= n0i;
        }

        // level-0 row y (general loop: rows past the loaded region are
        // prefetched for the ramp-down steps and never used, so skipped)
        auto load_row = [&](C(&v)[RW], int y) {
            if (y >= hi0) return;
            if (per) {
                // one wrap at most: the host keeps n0 >= 64 and n2 >= 136
                const int yw = (y < 0) ? y + n0i : (y >= n0i ? y - n0i : y);
                const T* rp = src + (int64_t)yw * lds;
                if (contig) {
#pragma unroll
                    for (int q = 0; q < RW; ++q) v[q] = Dt::load(rp + cw0 + q);
                } else {
#pragma unroll
                    for (int q = 0; q < RW; ++q) {
                        const int c = cw0 + q;
                        v[q] = Dt::load(rp + (c >= n2 ? c - n2 : c));
                    }
                }
            } else {
                const T* rp = src + (int64_t)(y + pad) * lds + (c0 + pad);
#pragma unroll
                for (int q = 0; q < RW; ++q) v[q] = ((lvm >> q) & 1u) ? Dt::load(rp + q) : C(0);
            }
        };
        // Shared-memory staging (FP32/FP64): row y's columns go to this
        // lane's slot by cp.async (zero-filled where the column does not
        // exist); rows past the loaded region are skipped (general loop) or
        // clamped into it (lean loop).  One commit group per row, always.
        // 2-byte storage: the first stored element of this lane's columns in
        // row y (periodic: wrapped; only for lanes without a wrap inside)
        auto elem0 = [&](int y) -> int64_t {
            if (per) {
                const int yw = (y < 0) ? y + n0i : (y >= n0i ? y - n0i : y);
                return (int64_t)yw * lds + cw0;
            }
            return (int64_t)(y + pad) * lds + (c0 + pad);
        };
        const int64_t total = (int64_t)(n0i + 2 * pad) * lds;  // stored elements of the grid
        auto issue_row = [&](int slot, int y, const bool G, const bool lean) {
            T* const sp = my_stage + slot * (32 * SW);
            bool skip = false;
            if (lean) y = min(y, hi0 - 1);
            else skip = (y >= hi0);
            if (!skip && sizeof(T) == 2) {
                if (per && G && !contig) {
                    // a wrap inside the lane's columns: element loads into the slot
                    const int yw = (y < 0) ? y + n0i : (y >= n0i ? y - n0i : y);
                    const T* rp = src + (int64_t)yw * lds;
#pragma unroll
                    for (int q = 0; q < RW; ++q) {
                        const int c = cw0 + q;
                        sp[q] = Dt::raw(rp + (c >= n2 ? c - n2 : c));
                    }
                } else {
                    // the pairs [a, a + SW) with a the element below the first
                    // column rounded down to even; pairs outside the array are
                    // zero-filled (their cells lie outside the padded row), and
                    // an odd-sized array's last element, whose pair would end
                    // past the array, is copied alone
                    const int64_t a = elem0(y) & ~(int64_t)1;
                    // (the lean loop's interior tiles, !G, have the
                    // property by construction; the general loop tests it
                    // per tile)
                    if ((!G && !per) || (!lean && stage_in)) {
#pragma unroll
                        for (int q = 0; q < SW; q += 2) rs_cp_async<4>(sp + q, src + (a + q), 4);
                    } else {
#pragma unroll
                        for (int q = 0; q < SW; q += 2) {
                            const int64_t e = a + q;
                            const bool ok = e >= 0 && e + 1 < total;
                            if (!ok && e >= 0 && e < total) {
                                sp[q] = Dt::raw(src + e);
                            } else {
                                rs_cp_async<4>(sp + q, ok ? src + e : src, ok ? 4 : 0);
                            }
                        }
                    }
                }
            } else if (!skip) {
                if (per) {
                    const int yw = (y < 0) ? y + n0i : (y >= n0i ? y - n0i : y);
                    const T* rp = src + (int64_t)yw * lds;
#pragma unroll
                    for (int q = 0; q < RW; ++q) {
                        const int c = cw0 + q;
                        rs_cp_async<sizeof(T)>(sp + q, rp + ((!G || contig) ? c : (c >= n2 ? c - n2 : c)), sizeof(T));
                    }
                } else {
                    const T* rp = src + (int64_t)(y + pad) * lds + (c0 + pad);
#pragma unroll
                    for (int q = 0; q < RW; ++q) {
                        const bool ok = !G || ((lvm >> q) & 1u);
                        rs_cp_async<sizeof(T)>(sp + q, ok ? rp + q : src, ok ? (int)sizeof(T) : 0);
                    }
                }
            }
            rs_cp_commit();
        };
        // the oldest row in flight into level 0's queue slot u
        auto take_row = [&](int u, int slot, int y, const bool G, const bool lean) {
            rs_cp_wait<PFS - 1>();
            const T* const sp = my_stage + slot * (32 * SW);
            // a lane's slot starts on a multiple of RW elements: 16-byte
            // loads for four floats (or two doubles), 8-byte loads for pairs
            if constexpr (sizeof(T) == 2) {
                // the row's parity (the same clamp as when it was issued)
                if (lean) y = min(y, hi0 - 1);
                const int par = (per && G && !contig) ? 0 : (int)(elem0(y) & 1);
                const unsigned short* const s16 = reinterpret_cast<const unsigned short*>(sp) + par;
#pragma unroll
                for (int q = 0; q < RW; ++q) ring[0][u][q] = __uint_as_float((unsigned)s16[q] << 16);
            } else if constexpr (sizeof(T) == 4 && RW % 4 == 0) {
#pragma unroll
                for (int q = 0; q < RW; q += 4) {
                    const float4 v = *reinterpret_cast<const float4*>(sp + q);
                    ring[0][u][q] = v.x;
                    ring[0][u][q + 1] = v.y;
                    ring[0][u][q + 2] = v.z;
                    ring[0][u][q + 3] = v.w;
                }
            } else if constexpr ((sizeof(T) == 4 || sizeof(T) == 8) && RW % 2 == 0) {
                using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
#pragma unroll
                for (int q = 0; q < RW; q += 2) {
                    const V2 v = *reinterpret_cast<const V2*>(sp + q);
                    ring[0][u][q] = v.x;
                    ring[0][u][q + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < RW; ++q) ring[0][u][q] = Dt::widen(sp[q]);
            }
        };

        // One level's row, split in two parts of the canonical FMA chain:
        // the head (every term whose row is older than the newest row of the
        // level below) and the tail (the terms on that newest row, last in
        // canonical order).  All levels' heads are independent of this
        // step's other levels, so they are issued first, back to back; only
        // the short tails form a chain through the levels.
        // (star: the centre row's r edge cells come from the adjacent lanes)
        constexpr int kTail = P - (EXT ? 2 * R + 1 : 1);  // first term on row +r
        // box stencils: only while the ring is shallow (t*r <= 4); at depth 6
        // the register pairs the packed form needs cost more than the halved
        // FMA count (measured: 9-point box t = 6 -6%, 25-point box t = 2 +9%)
        // (BF16 storage, 13-point star: the packed form spills under the
        // register cap, so it keeps scalar FMAs)
        constexpr bool kPair = (sizeof(C) == 4) && kRSPackedFma && (!EXT || D * R <= 4) &&
                               !(sizeof(T) == 2 && !EXT && R == 3);
        // The accumulators of levels below t are the queue slots they fill
        // (the slot's old row is dead by then), so no copy follows the FMAs.
        C accD[4];  // level t's row (to global memory)
        auto acc_ref = [&](int s, int cs, int m) -> C& {
            return (s < D) ? ring[s < D ? s : 0][cs][X0 + m] : accD[m];
        };
        // A level's result rounded to the storage type: to nearest even, or
        // (BF16-SR storage) stochastically with the bits of the cell's
        // stored index and step -- the key of level s's step, the column part
        // of this lane's first cell (periodic: wrapped) and the row's part.
        uint32_t srk[Dt::kSR ? D : 1];
        uint32_t sr_col = 0;
        if constexpr (Dt::kSR) {
#pragma unroll
            for (int s = 1; s <= D; ++s) srk[s - 1] = sr_step_key(gd->sr_key, (uint32_t)(blk * D + s));
            sr_col = (uint32_t)(per ? (cb < 0 ? cb + n2 : (cb >= n2 ? cb - n2 : cb)) : cb + pad);
        }
        auto round_cell = [&](int s, int y, int m, C a) -> C {
            if constexpr (Dt::kSR) {
                const int yw = per ? (y < 0 ? y + n0i : (y >= n0i ? y - n0i : y)) : y + pad;
                uint32_t c = sr_col + (uint32_t)m;
                if (per && c >= (uint32_t)n2) c -= (uint32_t)n2;
                return sr_round_bf16(a, (uint32_t)yw * (uint32_t)lds + c + srk[s - 1]);
            } else {
                return Dt::widen(Dt::narrow(a));
            }
        };
        // a level's four results rounded (BF16 to nearest: two packed
        // conversions, each element rounded on its own as by one conversion)
        auto round_row = [&](int s, int y, int cs, C(&o)[4]) {
            if constexpr (!Dt::kSR && sizeof(T) == 2) {
#pragma unroll
                for (int q2 = 0; q2 < 2; ++q2) {
                    const __nv_bfloat162 p = __floats2bfloat162_rn(acc_ref(s, cs, 2 * q2), acc_ref(s, cs, 2 * q2 + 1));
                    const unsigned w = *reinterpret_cast<const unsigned*>(&p);
                    o[2 * q2] = __uint_as_float(w << 16);
                    o[2 * q2 + 1] = __uint_as_float(w & 0xffff0000u);
                }
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) o[m] = round_cell(s, y, m, acc_ref(s, cs, m));
            }
        };

        auto level_row = [&](int s, int cs, const bool head) {
            C e[EXT ? 1 : 4 + 2 * R];
            if (!EXT && head) {
#pragma unroll
                for (int m = 0; m < 4; ++m) e[R + m] = ring[s - 1][cs][EXT ? 0 : m];
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    e[EXT ? 0 : i] = __shfl_up_sync(FULL, ring[s - 1][cs][4 - R + i], 1);
                    e[EXT ? 0 : R + 4 + i] = __shfl_down_sync(FULL, ring[s - 1][cs][i], 1);
                }
            }
#pragma unroll
            for (int k = 0; k < P; ++k) {
                if ((k < kTail) != head) continue;
                const int dy = OFF.ds[k], dx = OFF.d2[k];
                const int rs = (cs + dy + U) % U;
                const C ck = coef(k);
                // FP32 arithmetic: where a term's four values are two
                // register pairs of a queued row (star: dx even), two cells
                // per packed FMA (per-element round to nearest: the same
                // result as two scalar FMAs)
                if constexpr (kPair) {
                    if (((EXT ? X0 + dx : dx) & 1) == 0) {
                        const float2 ck2 = make_float2(ck, ck);
#pragma unroll
                        for (int q2 = 0; q2 < 2; ++q2) {
                            C v[2];
#pragma unroll
                            for (int w = 0; w < 2; ++w) {
                                const int m = 2 * q2 + w;
                                v[w] = EXT ? ring[s - 1][rs][X0 + m + dx]
                                           : ((dy == 0) ? e[R + m + dx] : ring[s - 1][rs][m]);
                            }
                            C& a0 = acc_ref(s, cs, 2 * q2);
                            C& a1 = acc_ref(s, cs, 2 * q2 + 1);
                            const float2 r2 = (k == 0) ? __fmul2_rn(ck2, make_float2(v[0], v[1]))
                                                       : __ffma2_rn(ck2, make_float2(v[0], v[1]), make_float2(a0, a1));
                            a0 = r2.x;
                            a1 = r2.y;
                        }
                        continue;
                    }
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    C v;
                    if constexpr (EXT) v = ring[s - 1][rs][X0 + m + dx];
                    else v = (dy == 0) ? e[R + m + dx] : ring[s - 1][rs][m];
                    C& a = acc_ref(s, cs, m);
                    a = (k == 0) ? Dt::mul(ck, v) : Dt::fma(ck, v, a);
                }
            }
        };
        // hand a level's row on: into its queue (box: with shuffled halo
        // cells), or to global memory for the last level
        auto put_row = [&](int s, int cs, int y, const C(&o)[4]) {
            if (s < D) {
#pragma unroll
                for (int m = 0; m < 4; ++m) ring[s][cs][X0 + m] = o[m];
                if constexpr (EXT) {
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        ring[s][cs][i] = __shfl_up_sync(FULL, o[4 - R + i], 1);
                        ring[s][cs][X0 + 4 + i] = __shfl_down_sync(FULL, o[i], 1);
                    }
                }
            } else {
                const unsigned st = (y >= ya && y < yb) ? outm : 0u;
                T* const rp = dst + (per ? (int64_t)y * lds : (int64_t)(y + pad) * lds + pad) + cb;
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if ((st >> m) & 1u) rp[m] = Dt::narrow(o[m]);
            }
        };

        // ---- stream the strip ----------------------------------------------------
        // Every level computes a row at every step.  A row outside its level's
        // region (the ramp at the segment's ends, rows past the padded grid,
        // the steps after the last) holds garbage that no kept value depends
        // on: a row y of level s+1 inside its region reads rows y-r .. y+r of
        // level s, all inside level s's region.  Only level-t rows inside the
        // segment are stored.
        if constexpr (kLean) {
            // both copies from one template (this form measured fastest for
            // the short stencils); rows past the region are clamped into it
            auto load_row2 = [&](C(&v)[RW], int y, const bool G) {
                y = min(y, hi0 - 1);
                if (per) {
                    const int yw = (y < 0) ? y + n0i : (y >= n0i ? y - n0i : y);
                    const T* rp = src + (int64_t)yw * lds;
                    if (!G || contig) {
#pragma unroll
                        for (int q = 0; q < RW; ++q) v[q] = Dt::load(rp + cw0 + q);
                    } else {
#pragma unroll
                        for (int q = 0; q < RW; ++q) {
                            const int c = cw0 + q;
                            v[q] = Dt::load(rp + (c >= n2 ? c - n2 : c));
                        }
                    }
                } else {
                    const T* rp = src + (int64_t)(y + pad) * lds + (c0 + pad);
#pragma unroll
                    for (int q = 0; q < RW; ++q) v[q] = (!G || ((lvm >> q) & 1u)) ? Dt::load(rp + q) : C(0);
                }
            };
            auto stream = [&](auto GEN) {
                constexpr bool G = decltype(GEN)::value;
                if constexpr (ASYNC) {
#pragma unroll
                    for (int q = 0; q < PFS; ++q) issue_row(q, lo0 + q, G, true);
                } else {
#pragma unroll
                    for (int q = 0; q < PF; ++q) load_row2(stage[q], lo0 + q, G);
                }
                for (int j0 = 0; j0 < niter; j0 += U) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int yi = lo0 + j0 + u;  // level-0 row arriving now
                        if constexpr (ASYNC) {
                            const int slot = (j0 + u) & (PFS - 1);
                            take_row(u, slot, yi, G, true);
                            issue_row(slot, yi + PFS, G, true);
                        } else {
#pragma unroll
                            for (int q = 0; q < RW; ++q) ring[0][u][q] = stage[u % PF][q];
                            load_row2(stage[u % PF], yi + PF, G);
                        }
#pragma unroll
                        for (int s = 1; s <= D; ++s) level_row(s, ((u - s * R) % U + U) % U, true);
#pragma unroll
                        for (int s = 1; s <= D; ++s) {
                            const int y = yi - s * R;                  // row of level s computed now
                            const int cs = ((u - s * R) % U + U) % U;  // queue slot of row y
                            C o[4];
                            level_row(s, cs, false);
                            round_row(s, y, cs, o);
                            if constexpr (G) {
                                const bool copy = (s > deff) || (!per && (y < 0 || y >= n0i));
                                const unsigned keep = copy ? 0xfu : padm;
#pragma unroll
                                for (int m = 0; m < 4; ++m)
                                    if ((keep >> m) & 1u) o[m] = ring[s - 1][cs][X0 + m];
                            }
                            put_row(s, cs, y, o);
                        }
                    }
                }
            };
            if (general)
                stream(std::true_type{});
            else
                stream(std::false_type{});
        } else {
            if constexpr (ASYNC) {
#pragma unroll
                for (int q = 0; q < PFS; ++q) issue_row(q, lo0 + q, true, false);
            } else {
#pragma unroll
                for (int q = 0; q < PF; ++q) load_row(stage[q], lo0 + q);
            }
            for (int j0 = 0; j0 < niter; j0 += U) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int yi = lo0 + j0 + u;  // level-0 row arriving now
                    if constexpr (ASYNC) {
                        const int slot = (j0 + u) & (PFS - 1);
                        take_row(u, slot, yi, true, false);
                        issue_row(slot, yi + PFS, true, false);
                    } else {
#pragma unroll
                        for (int q = 0; q < RW; ++q) ring[0][u][q] = stage[u % PF][q];
                        load_row(stage[u % PF], yi + PF);
                    }
#pragma unroll
                    for (int s = 1; s <= D; ++s) level_row(s, ((u - s * R) % U + U) % U, true);
#pragma unroll
                    for (int s = 1; s <= D; ++s) {
                        const int y = yi - s * R;                  // row of level s computed now
                        const int cs = ((u - s * R) % U + U) % U;  // queue slot of row y
                        // pad rows and the levels past the last block's depth
                        // keep the value below; pad columns likewise
                        const bool copy = (s > deff) || (!per && (y < 0 || y >= n0i));
                        const unsigned keep = copy ? 0xfu : padm;
                        C o[4];
                        level_row(s, cs, false);
                        round_row(s, y, cs, o);
#pragma unroll
                        for (int m = 0; m < 4; ++m)
                            if ((keep >> m) & 1u) o[m] = ring[s - 1][cs][X0 + m];
                        put_row(s, cs, y, o);
                    }
                }
            }
        }

        if constexpr (ASYNC) rs_cp_wait<0>();  // the slots are reused by the next item

        // ---- publish completion of this tile -------------------------------------
        __threadfence();
        __syncwarp();
        if (lane == 0) red_release_add_u32(&done[tile], 1u);
    }
}

}  // namespace ebisu
