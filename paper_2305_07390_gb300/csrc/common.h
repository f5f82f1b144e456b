// common.h -- structures shared by the host orchestration and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>

namespace ebisu {

constexpr int kMaxPoints = 125;        // 3D box of radius 2
constexpr size_t kControlBytes = 65536; // status word, counters (single run)
constexpr size_t kAlign = 256;

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Control block at the start of every workspace.  Zeroed before each run.
struct Control {
    int status;          // 0 = ok, else an ebisu_status code set by a kernel
    unsigned next_item;  // work-queue head (persistent kernels pop items)
    unsigned wait_where; // diagnostic: item index of the wait that gave up
    unsigned pad_[5];
    unsigned done[1];    // per-problem completed-tile counters (ngrids)
};

// One problem of a (possibly batched) temporally blocked launch, in
// streaming coordinates: s = slowest axis (y in 2D, z in 3D), p1 = y in 3D
// (dummy, extent 1, in 2D), p2 = x.
struct GridDesc {
    const void* src0;    // input of the first temporal block
    void* out;           // final destination
    void* ws;            // ping-pong buffer
    void* halo_dst0;     // buffers whose Dirichlet pad is filled from src0
    void* halo_dst1;     //   during the first temporal block (or null)
    int64_t n[3];        // interior extents (s, p1, p2)
    int64_t lds;         // element stride between consecutive s
    int64_t ld1;         // element stride between consecutive p1
    int32_t pad;         // Dirichlet pad width (= radius), 0 if periodic
    int32_t periodic;
    int32_t tile[3];     // output tile extents (s, p1, p2)
    int32_t nt[3];       // tiles per axis (s, p1, p2)
    int32_t ntiles;
    int32_t depth;       // temporal block depth t
    int32_t nblocks;     // ceil(steps / depth)
    int32_t last_depth;  // depth of the last block
    int32_t grid_id;     // index into Control::done
    int32_t load_mode;   // 0 = element cp.async, 1 = pair cp.async (2-byte
                         // types, rows of a plane share parity), 2 = staged
    int32_t plane_cap;   // elements per ring plane of this problem (its own
                         // stride, so batch members need no common one)
    int32_t reserved_;
    int64_t total_elems; // stored elements of the grid (bounds of pair loads)
    double coef[kMaxPoints];
};

// Kernel parameters of a temporally blocked launch.
struct TBParams {
    GridDesc g;                 // the problem, when `grids` is null
    const GridDesc* grids;      // batched: per-problem descriptors (device)
    const int32_t* items;       // batched: (grid, block, tile) triples (device)
    int64_t nitems;
    Control* ctl;
    int64_t timeout_ns;         // bound on every dependency wait
    int32_t debug_stall;        // test hook: 1 = the first wait targets a
                                // count that is never reached
    int32_t smem_plane;         // elements per ring plane
};

// ---------------------------------------------------------------------------
// Register-streaming build (2D): one warp streams one strip of 128 columns
// (32 lanes x 4 cells) down a segment of rows, every time level of the
// temporal block held in registers.  Tiles of one temporal block depend only
// on their eight neighbours of the previous block (per-tile counters).
constexpr int kRSWarps = 4;            // warps per CTA
constexpr int kRSThreads = 32 * kRSWarps;
constexpr int kRSCols = 128;           // columns a warp holds (loaded region)
// Maximum tiles of one run (one completion counter each in the Control block).
constexpr int64_t kRSMaxTiles = (int64_t)((kControlBytes - 64) / sizeof(unsigned));

// Temporal depths built per storage size and stencil (which = 0: the
// shallower, 1: the deeper).  FP64 is bound by its FMA pipe, so depth only
// adds redundant work there; FP32/BF16 take the deepest ring that still fits
// the register file at two or more resident CTAs.
constexpr int rs_depth(int esize, int shape /*0 star, 1 box*/, int r, int which)
{
    if (esize == 8) return (which && !(shape == 0 && r == 3) && !(shape == 1 && r == 2)) ? 2 : 1;
    if (shape == 0) return r == 1 ? (which ? 8 : 4) : r == 2 ? (which ? 5 : 3) : (which ? 3 : 2);
    return r == 1 ? (which ? 6 : 3) : (which ? 2 : 1);
}

// 3D register-streaming builds: which stencils they cover (FP64 at depth 1:
// the 7- and 13-point stars and the radius-1 boxes; FP32 and BF16
// temporally blocked: radius 1) and the rows of a warp's patch.
constexpr bool rs3_built(int esize, int shape, int r)
{
    return (esize == 8 && (r == 1 || (shape == 0 && r == 2))) || (esize != 8 && r == 1);
}
// rows of a warp's patch (FP64 depth 1: 2; FP32/BF16 temporally blocked: 4)
constexpr int rs3_rows(int esize) { return esize == 8 ? 2 : 4; }
constexpr int kRS3Cols = 64;  // columns a warp holds (32 lanes x 2)
// output columns per 64-column strip: the patch loses t*r columns per side;
// the FP32/BF16 build shifts the patch one column left when r(t-1) is odd so
// that a lane's column pair starts on an even stored column
constexpr int rs3_strip(int esize, int depth, int r)
{
    return kRS3Cols - 2 * depth * r - ((esize != 8 && ((r * (depth - 1)) & 1)) ? 2 : 0);
}
// temporal depths built (FP64: 1; FP32/BF16: 7-point star 2 and 3, the
// other radius-1 stencils 2)
constexpr int rs3_depth(int esize, int shape, int r, int which)
{
    return esize == 8 ? 1 : ((which && shape == 0 && r == 1) ? 3 : 2);
}

// Depth the register-streaming build defaults to (FP32/BF16 storage): the
// faster of the two built depths on 8192^2 grids (measured on GB300).
constexpr int rs_preferred_depth(int esize, int shape, int r)
{
    if (esize == 8) return 1;
    if (shape == 0) return r == 1 ? (esize == 4 ? 8 : 4) : (r == 2 ? 3 : 2);
    return r == 1 ? (esize == 4 ? 6 : 3) : 2;
}

// One problem of a register-streaming launch.
struct RSGrid {
    const void* src0;   // input of the first temporal block
    void* out;          // final destination
    void* ws;           // ping-pong buffer
    void* pad_dst0;     // buffers whose Dirichlet pad is filled from src0
    void* pad_dst1;     //   during the first temporal block (or null)
    int64_t n0;         // interior rows
    int64_t lds;        // row pitch (elements)
    int32_t n2;         // interior columns
    int32_t pad;        // Dirichlet pad (= radius), 0 if periodic
    int32_t periodic;
    int32_t S;          // output columns per strip (128 - 2 * depth * radius)
    int32_t H;          // output rows per segment
    int32_t nstrips, nsegs;
    int32_t nblocks;    // ceil(steps / depth)
    int32_t depth_last; // steps done by the last block (<= depth)
    int32_t tile_base;  // index of this problem's first tile counter
    uint32_t sr_key;    // stochastic-rounding plan key (BF16-SR storage only)
    int32_t reserved_;
    double coef[kMaxPoints];
    float coef_f[kMaxPoints];  // the same rounded to FP32 (FP32/BF16 storage)
};

// Kernel parameters of a register-streaming launch.
struct RSParams {
    RSGrid g;                // the problem, when `grids` is null
    const RSGrid* grids;     // batched: per-problem descriptors (device)
    const int32_t* items;    // batched: (grid, block, tile) triples (device)
    int64_t nitems;          // single: nblocks * nstrips * nsegs
    Control* ctl;
    int64_t timeout_ns;      // bound on every dependency wait
    int32_t debug_stall;     // test hook: the first wait targets a count never reached
};

// Kernel parameters of a 3D register-streaming launch.
struct RS3Params {
    const void* src0;    // input of the first temporal block
    void* out;           // final destination
    void* ws;            // ping-pong buffer
    int64_t n[3];        // interior extents (z, y, x)
    int64_t lds, ld1;    // element strides of z and y
    int64_t nitems;      // nblocks * nstrips * nbands * nsegs (nbands: patches along y)
    Control* ctl;
    int64_t timeout_ns;
    int32_t pad;         // Dirichlet pad (= radius), 0 if periodic
    int32_t periodic;
    int32_t S;           // output columns per strip (64 - 2 * depth * radius)
    int32_t H;           // output planes per z segment
    int32_t nstrips, nbands, nsegs;
    int32_t nblocks;     // ceil(steps / depth)
    int32_t depth_last;  // steps done by the last block (<= depth)
    int32_t debug_stall;
    uint32_t sr_key;     // stochastic-rounding plan key (BF16-SR storage only)
    int32_t reserved_;
    double coef[kMaxPoints];
    float coef_f[kMaxPoints];
};

}  // namespace ebisu
