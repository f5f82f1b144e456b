// rs3_kernel.cuh -- register-streaming kernel for 3D grids at temporal depth 1.
//
// On this part FP64 stencils are bound by the FP64 pipe, so the tuner runs
// them at depth 1 (Eq. 17's desired depth is below 1).  At depth 1 the
// shared-memory kernel's per-plane barrier and shared-memory latency keep the
// pipe ~half idle in 3D; this kernel removes both, like the 2D register-
// streaming kernel (rs_kernel.cuh):
//  * One warp owns a 64-column x 2-row patch of the
//    xy plane -- lane l holds columns 2l, 2l+1 of every row -- and streams it
//    along z (Section 2.1.3's N.5-D streaming).
//  * The last 2r+1 input planes of the patch, each with r rows of y halo
//    above and below, are kept in registers (the z queue; the plane loop is
//    unrolled 2r+1 times so every queue slot is a fixed register); the next
//    plane is loaded one step ahead.
//  * x neighbours come from the adjacent lanes by warp shuffles; the patch's
//    outermost r columns are overlap (strips advance by 64 - 2r columns).
//  * Tiles (strip, band, z segment) of step b wait only for their 3 x 3 x 3
//    neighbours of step b-1 (per-tile counters, bounded waits); the
//    neighbours are also the only readers of what a tile overwrites.
//  * Output cells are interior cells only; Dirichlet pads are read, never
//    written (the host copies the input's pad to the written buffers).
#pragma once
#include <type_traits>

#include "common.h"
#include "stencil.cuh"

namespace ebisu {

template <class T, int SHAPE, int R>
struct RS3Geom {
    using C = typename DT<T>::C;
    static constexpr int VX = 2;                 // columns per lane
    static constexpr int TY = 2;                 // output rows per warp
    static constexpr int YR = TY + 2 * R;        // loaded rows per plane
    static constexpr int U = 2 * R + 1;          // planes queued
    static constexpr int WORDS = (int)sizeof(C) / 4;
    // star stencils read the y halo only on the centre plane: the queue keeps
    // the TY core rows of each plane, and the centre plane's 2r halo rows are
    // loaded one step ahead of their use
    static constexpr bool STARQ = (SHAPE == kStar);
    static constexpr int QR = STARQ ? TY : YR;  // rows kept per queued plane
    static constexpr int Q0 = STARQ ? R : 0;    // loaded-row index of queue row 0
    static constexpr int regs()
    {
        return (U * QR * VX + QR * VX + (STARQ ? 4 * R * VX : 0) + TY * VX + 4 * R) * WORDS + 112;
    }
    static constexpr int minb()
    {
        const int e = (regs() + 7) & ~7;
        const int b = 65536 / (kRSThreads * e);
        return b < 1 ? 1 : (b > 8 ? 8 : b);
    }
};

template <class T, int SHAPE, int R>
__global__ void __launch_bounds__(kRSThreads, RS3Geom<T, SHAPE, R>::minb())
    rs3_kernel(const __grid_constant__ RS3Params prm)
{
    using G = RS3Geom<T, SHAPE, R>;
    using Dt = DT<T>;
    using C = typename Dt::C;
    using St = Stencil<3, SHAPE, R>;
    constexpr int P = St::P;
    constexpr int VX = G::VX, TY = G::TY, YR = G::YR, U = G::U;
    constexpr bool STARQ = G::STARQ;
    constexpr int QR = G::QR, Q0 = G::Q0;
    constexpr int NH = STARQ ? 2 * R : 1;  // halo rows of the centre plane (star)
    constexpr auto OFF = St::kOff;  // ds = dz, d1 = dy, d2 = dx
    constexpr auto ROWS = St::make_rows();  // offsets sharing (dz, dy) are consecutive
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(R <= VX, "x neighbours must come from the adjacent lanes only");

    const int lane = threadIdx.x & 31;
    Control* const ctl = prm.ctl;
    const bool per = prm.periodic != 0;
    const int n0 = (int)prm.n[0], n1 = (int)prm.n[1], n2 = (int)prm.n[2];
    const int pad = prm.pad;
    const int64_t lds = prm.lds, ld1 = prm.ld1;
    const int S = prm.S, H = prm.H, nstrips = prm.nstrips, nbands = prm.nbands, nsegs = prm.nsegs;
    const long long ntiles = (long long)nstrips * nbands * nsegs;
    auto coef = [&](int k) -> C {
        if constexpr (sizeof(C) == 8) return prm.coef[k];
        else return prm.coef_f[k];
    };

    C q[U][QR][VX];     // the z queue
    C stage[QR][VX];    // the next plane
    C hcur[NH][VX];     // star: halo rows of this step's centre plane
    C hnext[NH][VX];    // star: halo rows of the next step's centre plane

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

        // ---- wait for the 3 x 3 x 3 neighbouring tiles of the previous step ----
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
        const bool dst_is_out = ((prm.nblocks - 1 - blk) & 1) == 0;
        T* const dst = reinterpret_cast<T*>(dst_is_out ? prm.out : prm.ws);
        const T* const src = (blk == 0) ? reinterpret_cast<const T*>(prm.src0)
                                        : reinterpret_cast<const T*>(dst_is_out ? prm.ws : prm.out);
        const int xs = strip * S, xe = min(xs + S, n2);
        const int cb = xs - R + VX * lane;  // this lane's first column
        const int ya = band * TY;           // first output row
        const int za = seg * H, zb = min(za + H, n0);
        const int lo0 = per ? za - R : max(za - R, -pad);
        const int hi0 = per ? zb + R : min(zb + R, n0 + pad);
        const int niter = zb + R - lo0;  // the last output plane zb-1 needs plane zb-1+r
        // in-plane stored offset of loaded row i (0 .. YR-1), column v of this
        // lane, and whether the cell exists (Dirichlet: inside the padded grid)
        unsigned rowok = 0, colok = 0;
#pragma unroll
        for (int i = 0; i < YR; ++i) {
            const int y = ya - R + i;
            if (per || (y >= -pad && y < n1 + pad)) rowok |= 1u << i;
        }
#pragma unroll
        for (int v = 0; v < VX; ++v) {
            const int c = cb + v;
            if (per || (c >= -pad && c < n2 + pad)) colok |= 1u << v;
        }
        auto cell_off = [&](int i, int v) -> int64_t {
            int y = ya - R + i, c = cb + v;
            if (per) {  // one wrap at most: the host keeps n1 >= 16 and n2 >= 72
                y = (y < 0) ? y + n1 : (y >= n1 ? y - n1 : y);
                c = (c < 0) ? c + n2 : (c >= n2 ? c - n2 : c);
                return (int64_t)y * ld1 + c;
            }
            return (int64_t)(y + pad) * ld1 + (c + pad);
        };
        unsigned outm = 0;  // output cells of this lane: bit i*VX+v
#pragma unroll
        for (int i = 0; i < TY; ++i)
#pragma unroll
            for (int v = 0; v < VX; ++v)
                if (ya + i < n1 && cb + v >= xs && cb + v < xe) outm |= 1u << (i * VX + v);

        auto plane_ptr = [&](int z) -> const T* {
            const int zw = per ? ((z < 0) ? z + n0 : (z >= n0 ? z - n0 : z)) : z + pad;
            return src + (int64_t)zw * lds;
        };
        auto load_plane = [&](int z) {
            if (z >= hi0) return;  // past the loaded region: never used
            const T* const pp = plane_ptr(z);
#pragma unroll
            for (int i = 0; i < QR; ++i)
#pragma unroll
                for (int v = 0; v < VX; ++v)
                    stage[i][v] = (((rowok >> (Q0 + i)) & (colok >> v)) & 1u) ? Dt::load(pp + cell_off(Q0 + i, v))
                                                                               : C(0);
        };
        // star: halo rows (loaded rows 0..r-1 and r+TY..YR-1) of plane z
        auto load_halo = [&](int z) {
            if (z < lo0 || z >= hi0) return;  // outside the loaded region: never used
            const T* const pp = plane_ptr(z);
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                const int fr = (h < R) ? h : TY + h;
#pragma unroll
                for (int v = 0; v < VX; ++v)
                    hnext[h][v] = (((rowok >> fr) & (colok >> v)) & 1u) ? Dt::load(pp + cell_off(fr, v)) : C(0);
            }
        };

        // ---- stream along z ------------------------------------------------------
        load_plane(lo0);
        for (int j0 = 0; j0 < niter; j0 += U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int zi = lo0 + j0 + u;  // plane arriving now
#pragma unroll
                for (int i = 0; i < QR; ++i)
#pragma unroll
                    for (int v = 0; v < VX; ++v) q[u][i][v] = stage[i][v];
                load_plane(zi + 1);
                const int z = zi - R;  // output plane of this step
                if constexpr (STARQ) {
#pragma unroll
                    for (int h = 0; h < NH; ++h)
#pragma unroll
                        for (int v = 0; v < VX; ++v) hcur[h][v] = hnext[h][v];
                    load_halo(z + 1);
                }
                // x neighbours: for every (plane, row) group of offsets that
                // reaches past this lane's pair, the pair of the adjacent lanes
                // (shuffled once per group, used by all its offsets)
                C acc[TY][VX];
                C lft[TY][VX], rgt[TY][VX];
                // star: the one group that needs them (the centre plane's
                // centre rows) is shuffled first, so the shuffles' latency
                // overlaps the FMAs of the offsets before it
                constexpr bool kHoist = (SHAPE == kStar);
                if constexpr (kHoist) {
                    const int sl = ((u - R) % U + U) % U;
#pragma unroll
                    for (int i = 0; i < TY; ++i)
#pragma unroll
                        for (int w = 0; w < VX; ++w) {
                            lft[i][w] = __shfl_up_sync(FULL, q[sl][R + i - Q0][w], 1);
                            rgt[i][w] = __shfl_down_sync(FULL, q[sl][R + i - Q0][w], 1);
                        }
                }
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const int dz = OFF.ds[k], dy = OFF.d1[k], dx = OFF.d2[k];
                    const int sl = ((u - R + dz) % U + U) % U;  // queue slot of plane z + dz
                    const C ck = coef(k);
                    if (!kHoist && ROWS.start[k] && (ROWS.min_d2[k] < 0 || ROWS.max_d2[k] > 0)) {
#pragma unroll
                        for (int i = 0; i < TY; ++i)
#pragma unroll
                            for (int w = 0; w < VX; ++w) {
                                lft[i][w] = __shfl_up_sync(FULL, q[sl][R + i + dy - Q0][w], 1);
                                rgt[i][w] = __shfl_down_sync(FULL, q[sl][R + i + dy - Q0][w], 1);
                            }
                    }
#pragma unroll
                    for (int i = 0; i < TY; ++i) {
                        const int fr = R + i + dy;  // loaded row
#pragma unroll
                        for (int v = 0; v < VX; ++v) {
                            const int cx = v + dx;
                            C val;
                            if (cx < 0) {
                                val = lft[i][cx + VX];
                            } else if (cx >= VX) {
                                val = rgt[i][cx - VX];
                            } else if (STARQ && (fr < Q0 || fr >= Q0 + QR)) {
                                val = hcur[STARQ ? ((fr < R) ? fr : fr - TY) : 0][cx];  // centre-plane halo row
                            } else {
                                val = q[sl][fr - Q0][cx];
                            }
                            acc[i][v] = (k == 0) ? Dt::mul(ck, val) : Dt::fma(ck, val, acc[i][v]);
                        }
                    }
                }
                if (z >= za && z < zb) {
                    T* const pz = dst + (per ? (int64_t)z * lds : (int64_t)(z + pad) * lds);
#pragma unroll
                    for (int i = 0; i < TY; ++i)
#pragma unroll
                        for (int v = 0; v < VX; ++v)
                            if ((outm >> (i * VX + v)) & 1u) pz[cell_off(R + i, v)] = Dt::narrow(acc[i][v]);
                }
            }
        }

        // ---- publish completion of this tile -------------------------------------
        __threadfence();
        __syncwarp();
        if (lane == 0) red_release_add_u32(&ctl->done[tile], 1u);
    }
}

}  // namespace ebisu
