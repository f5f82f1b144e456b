// plan.cpp -- plans, runs and the core of the C ABI (include/ebisu.h).
#include "plan.h"
#include "stencil.cuh"  // the stochastic-rounding keys (host side)

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

using namespace ebisu;

namespace ebisu {

static thread_local char g_err[512] = "no CUDA error";

void set_cuda_error(cudaError_t e)
{
    snprintf(g_err, sizeof(g_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

int fail_cuda_at(cudaError_t e, const char* file, int line)
{
    const char* base = strrchr(file, '/');
    snprintf(g_err, sizeof(g_err), "%s:%d: %s: %s", base ? base + 1 : file, line, cudaGetErrorName(e),
             cudaGetErrorString(e));
    cudaGetLastError();
    return EBISU_ERR_CUDA;
}

static std::mutex g_dev_mu;
static DeviceInfo g_dev[16];

const DeviceInfo& device_info()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) dev = 0;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceInfo& d = g_dev[dev];
    if (d.device < 0) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
            d.sms = prop.multiProcessorCount;
            d.smem_optin = prop.sharedMemPerBlockOptin;
            d.smem_per_sm = prop.sharedMemPerMultiprocessor;
            strncpy(d.name, prop.name, sizeof(d.name) - 1);
        } else {
            cudaGetLastError();
            // no device: GB300 figures, so that plans can be built on a host
            d.sms = 152;
            d.smem_optin = 232448;
            d.smem_per_sm = 233472;
            strncpy(d.name, "no device", sizeof(d.name) - 1);
        }
        d.device = dev;
    }
    return d;
}

int64_t wait_timeout_ns()
{
    const char* e = getenv("EBISU_WAIT_TIMEOUT_MS");
    if (e && *e) {
        const long long ms = atoll(e);
        if (ms > 0) return (int64_t)ms * 1000000LL;
    }
    return 60LL * 1000000000LL;
}

int ring_q(int radius) { return 2 * radius + 2; }
int ring_q0(int radius, int ndim, int variant, size_t esize)
{
    return 2 * radius + 1 + prefetch_planes(ndim, variant, esize);
}

// largest level-0 region of any tile: (E1, E2), unpadded
static void max_plane(const ebisu_plan_s* p, const ebisu_params& q, int64_t* e1, int64_t* e2)
{
    const int r = p->radius;
    const bool per = p->boundary == EBISU_PERIODIC;
    const int64_t tx = std::min<int64_t>(q.tile_x, p->n[2]);
    *e2 = tx + 2LL * r * q.depth;
    if (!per) *e2 = std::min<int64_t>(*e2, p->n[2] + 2LL * p->pad);
    *e1 = 1;
    if (p->ndim == 3) {
        const int64_t ty = std::min<int64_t>(q.tile_y, p->n[1]);
        *e1 = ty + 2LL * r * q.depth;
        if (!per) *e1 = std::min<int64_t>(*e1, p->n[1] + 2LL * p->pad);
    }
}

int64_t plane_capacity(const ebisu_plan_s* p, const ebisu_params& q)
{
    int64_t e1, e2;
    max_plane(p, q, &e1, &e2);
    // row pitch as the kernel lays rows out: a 4-column margin, the row, one
    // column of pair-load shift and room for the 4-wide reads, rounded to 4
    const int64_t pitch = (e2 + 4 + 7 + 3) & ~(int64_t)3;
    return e1 * pitch;
}

size_t tb_smem_bytes(const ebisu_plan_s* p, const ebisu_params& q)
{
    const size_t slots = (size_t)ring_q0(p->radius, p->ndim, kernel_variant(p->dtype, q.ctas_per_sm), p->esize) +
                         (size_t)(q.depth - 1) * ring_q(p->radius);
    return slots * (size_t)plane_capacity(p, q) * p->esize;
}

// 3D register-streaming build: 64-column strips (S = 64 - 2r), bands of TY
// rows, z segments of H planes; depth 1 only.
static int rs3_layout(const ebisu_plan_s* p, const ebisu_params& q, RSLayout* L)
{
    const int r = p->radius, es = (int)p->esize;
    if (!rs3_built(es, p->shape, r)) return EBISU_ERR_UNSUPPORTED;
    if (q.depth != rs3_depth(es, p->shape, r, 0) && q.depth != rs3_depth(es, p->shape, r, 1))
        return EBISU_ERR_UNSUPPORTED;
    const int64_t n0 = p->n[0], n1 = p->n[1], n2 = p->n[2];
    if (n0 + 2 * p->pad > (1LL << 30) || n1 + 2 * p->pad > (1LL << 30) || n2 + 2 * p->pad > (1LL << 30))
        return EBISU_ERR_UNSUPPORTED;
    const bool per = p->boundary == EBISU_PERIODIC;
    // the kernel wraps a periodic index at most once
    if (per && (n0 < 16 || n1 < 16 || n2 < 72)) return EBISU_ERR_UNSUPPORTED;
    const int dr = q.depth * r;
    const int S = rs3_strip(es, q.depth, r), TY = rs3_rows(es);
    const int64_t H = (q.tile_s <= 0) ? n0 : std::min<int64_t>(q.tile_s, n0);
    const int64_t ns = (n2 + S - 1) / S, nb = (n1 + TY - 1) / TY, ng = (n0 + H - 1) / H;
    // a tile's inputs reach depth*r cells into its neighbours and no further
    if ((ng > 1 && H < dr) || TY < dr || S < dr) return EBISU_ERR_UNSUPPORTED;
    if (per && ((ns > 1 && n2 - (ns - 1) * S < dr) || (nb > 1 && n1 - (nb - 1) * TY < dr) ||
                (ng > 1 && n0 - (ng - 1) * H < dr)))
        return EBISU_ERR_UNSUPPORTED;
    if (ns * nb * ng > kRSMaxTiles) return EBISU_ERR_UNSUPPORTED;
    // the FP32/BF16 build addresses within a plane with 32-bit offsets
    if ((n1 + 2 * p->pad) * (n2 + 2 * p->pad) >= (1LL << 31)) return EBISU_ERR_UNSUPPORTED;
    if (L) {
        L->S = S;
        L->H = (int)H;
        L->nstrips = (int)ns;
        L->nsegs = (int)ng;
        L->TY = TY;
        L->nbands = (int)nb;
    }
    return EBISU_OK;
}

int rs_layout(const ebisu_plan_s* p, const ebisu_params& q, RSLayout* L)
{
    if (p->ndim == 3) return rs3_layout(p, q, L);
    if (p->ndim != 2) return EBISU_ERR_UNSUPPORTED;
    const int r = p->radius, es = (int)p->esize;
    if (q.depth != rs_depth(es, p->shape, r, 0) && q.depth != rs_depth(es, p->shape, r, 1))
        return EBISU_ERR_UNSUPPORTED;
    const int64_t n0 = p->n[0], n2 = p->n[2];
    if (n0 + 2 * p->pad > (1LL << 30) || n2 + 2 * p->pad > (1LL << 30)) return EBISU_ERR_UNSUPPORTED;
    const bool per = p->boundary == EBISU_PERIODIC;
    // the kernel wraps a periodic index at most once
    if (per && (n0 < 64 || n2 < 136)) return EBISU_ERR_UNSUPPORTED;
    const int dr = q.depth * r;
    const int S = kRSCols - 2 * dr;
    const int64_t H = (q.tile_s <= 0) ? n0 : std::min<int64_t>(q.tile_s, n0);
    const int64_t ns = (n2 + S - 1) / S, ng = (n0 + H - 1) / H;
    // a tile's inputs reach dr cells into its neighbours and no further
    if (ng > 1 && H < dr) return EBISU_ERR_UNSUPPORTED;
    if (per && ns > 1 && n2 - (ns - 1) * S < dr) return EBISU_ERR_UNSUPPORTED;
    if (per && ng > 1 && n0 - (ng - 1) * H < dr) return EBISU_ERR_UNSUPPORTED;
    if (ns * ng > kRSMaxTiles) return EBISU_ERR_UNSUPPORTED;
    if (L) {
        L->S = S;
        L->H = (int)H;
        L->nstrips = (int)ns;
        L->nsegs = (int)ng;
    }
    return EBISU_OK;
}

int check_params(const ebisu_plan_s* p, const ebisu_params& q)
{
    if (q.variant < 0 || q.variant > 2) return EBISU_ERR_INVALID_ARG;
    if (q.variant == 1) return EBISU_OK;
    // stochastic rounding is built into the register-streaming and one-step kernels only
    if (plan_sr(p) && q.variant == 0) return EBISU_ERR_UNSUPPORTED;
    if (q.variant == 2) {
        if (q.ctas_per_sm < 1 || q.ctas_per_sm > 16 || q.tile_s < 0) return EBISU_ERR_INVALID_ARG;
        return rs_layout(p, q, nullptr);
    }
    if (q.depth < 1 || q.depth > 64 || q.tile_x < 1 || (p->ndim == 3 && q.tile_y < 1) || q.tile_s < 0 ||
        q.ctas_per_sm < 1 || q.ctas_per_sm > 8)
        return EBISU_ERR_INVALID_ARG;
    int64_t e1, e2;
    max_plane(p, q, &e1, &e2);
    if (e1 * e2 > (int64_t)kStagePerThread * kThreads) return EBISU_ERR_UNSUPPORTED;
    const DeviceInfo& d = device_info();
    if (tb_smem_bytes(p, q) + 4096 > d.smem_optin) return EBISU_ERR_UNSUPPORTED;
    return EBISU_OK;
}

int64_t fill_grid_desc(const ebisu_plan_s* p, const void* in, void* out, void* wsgrid, int64_t steps,
                       bool in_copied_to_ws, GridDesc* g)
{
    memset(g, 0, sizeof(*g));
    const ebisu_params& q = p->prm;
    const int d = (int)std::min<int64_t>(q.depth, std::max<int64_t>(steps, 1));
    const int64_t nb = (steps + d - 1) / d;
    g->src0 = in_copied_to_ws ? wsgrid : in;
    g->out = out;
    g->ws = wsgrid;
    for (int i = 0; i < 3; ++i) g->n[i] = p->n[i];
    g->lds = p->lds;
    g->ld1 = p->ld1;
    g->pad = p->pad;
    g->periodic = p->boundary == EBISU_PERIODIC;
    g->tile[2] = (int32_t)std::min<int64_t>(q.tile_x, p->n[2]);
    g->tile[1] = (p->ndim == 3) ? (int32_t)std::min<int64_t>(q.tile_y, p->n[1]) : 1;
    g->tile[0] = (q.tile_s <= 0) ? (int32_t)p->n[0] : (int32_t)std::min<int64_t>(q.tile_s, p->n[0]);
    for (int i = 0; i < 3; ++i) g->nt[i] = (int32_t)((p->n[i] + g->tile[i] - 1) / g->tile[i]);
    g->ntiles = g->nt[0] * g->nt[1] * g->nt[2];
    g->depth = d;
    g->nblocks = (int32_t)nb;
    g->last_depth = (int32_t)(steps - (nb - 1) * d);
    g->grid_id = 0;
    g->total_elems = p->elems;
    if (p->esize >= 4) {
        g->load_mode = 0;  // one cp.async per element
    } else {
        // 2-byte elements: aligned 4-byte pairs when every row of a plane
        // starts on the same parity and no row wraps, else staged loads
        const bool rows_agree = (p->ndim == 2) || ((p->ld1 % 2 == 0) && (p->lds % 2 == 0));
        const bool aligned = ((uintptr_t)in % 4 == 0) && ((uintptr_t)out % 4 == 0) &&
                             ((uintptr_t)wsgrid % 4 == 0);
        g->load_mode = (!g->periodic && rows_agree && aligned) ? 1 : 2;
    }
    for (int k = 0; k < p->npts; ++k) g->coef[k] = p->coef[k];
    // Buffers whose Dirichlet pad must be filled during the first block.
    void* dst0 = ((nb - 1) % 2 == 0) ? out : wsgrid;
    void* dst1 = (nb >= 2) ? (((nb - 2) % 2 == 0) ? out : wsgrid) : nullptr;
    if (!g->periodic) {
        if (dst0 && dst0 != g->src0 && dst0 != in) g->halo_dst0 = dst0;
        if (dst1 && dst1 != g->src0 && dst1 != in) g->halo_dst1 = dst1;
    }
    return nb * (int64_t)g->ntiles;
}

cudaError_t tb_launch(const ebisu_plan_s* p, int v, const TBParams& prm, int grid, size_t smem, cudaStream_t st)
{
    switch (p->dtype) {
    case EBISU_F64: return tb_launch_f64(p->ndim, p->shape, p->radius, v, prm, grid, smem, st);
    case EBISU_F32: return tb_launch_f32(p->ndim, p->shape, p->radius, v, prm, grid, smem, st);
    default: return tb_launch_bf16(p->ndim, p->shape, p->radius, v, prm, grid, smem, st);
    }
}

cudaError_t tb_occupancy(const ebisu_plan_s* p, int v, size_t smem, int* blocks)
{
    switch (p->dtype) {
    case EBISU_F64: return tb_occupancy_f64(p->ndim, p->shape, p->radius, v, smem, blocks);
    case EBISU_F32: return tb_occupancy_f32(p->ndim, p->shape, p->radius, v, smem, blocks);
    default: return tb_occupancy_bf16(p->ndim, p->shape, p->radius, v, smem, blocks);
    }
}

static NaiveParams naive_params(const ebisu_plan_s* p)
{
    NaiveParams a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < 3; ++i) a.n[i] = p->n[i];
    a.lds = p->lds;
    a.ld1 = p->ld1;
    a.pad = p->pad;
    a.periodic = p->boundary == EBISU_PERIODIC;
    for (int k = 0; k < p->npts; ++k) {
        a.coef[k] = p->coef[k];
        a.coef_f[k] = (float)p->coef[k];  // round to nearest, as the device conversion does
    }
    return a;
}

cudaError_t naive_vc_launch(const ebisu_plan_s* p, const void* src, void* dst, cudaStream_t st)
{
    const NaiveParams a = naive_params(p);
    switch (p->dtype) {
    case EBISU_F64: return naive_vc_launch_f64(p->ndim, p->shape, p->radius, src, dst, p->field, p->elems, a, st);
    case EBISU_F32: return naive_vc_launch_f32(p->ndim, p->shape, p->radius, src, dst, p->field, p->elems, a, st);
    default: return naive_vc_launch_bf16(p->ndim, p->shape, p->radius, src, dst, p->field, p->elems, a, st);
    }
}

cudaError_t naive_launch(const ebisu_plan_s* p, const void* src, void* dst, int64_t t, cudaStream_t st)
{
    NaiveParams a = naive_params(p);
    if (plan_sr(p)) {
        a.sr_k = sr_step_key(p->sr_key, (uint32_t)t);
        return naive_launch_bf16sr(p->ndim, p->shape, p->radius, src, dst, a, st);
    }
    switch (p->dtype) {
    case EBISU_F64: return naive_launch_f64(p->ndim, p->shape, p->radius, src, dst, a, st);
    case EBISU_F32: return naive_launch_f32(p->ndim, p->shape, p->radius, src, dst, a, st);
    default: return naive_launch_bf16(p->ndim, p->shape, p->radius, src, dst, a, st);
    }
}

static PadParams pad_params(const ebisu_plan_s* p)
{
    PadParams a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < 3; ++i) a.n[i] = p->n[i];
    a.lds = p->lds;
    a.ld1 = p->ld1;
    a.pad = p->pad;
    a.pad1 = p->pad1;
    return a;
}

cudaError_t pad_copy(const ebisu_plan_s* p, const void* src, void* d0, void* d1, cudaStream_t st)
{
    if (p->boundary == EBISU_PERIODIC || (!d0 && !d1)) return cudaSuccess;
    const PadParams a = pad_params(p);
    switch (p->dtype) {
    case EBISU_F64: return pad_copy_f64(src, d0, d1, a, st);
    case EBISU_F32: return pad_copy_f32(src, d0, d1, a, st);
    default: return pad_copy_bf16(src, d0, d1, a, st);
    }
}

}  // namespace ebisu

// ===========================================================================
// C ABI

namespace ebisu {

cudaError_t rs_launch(const ebisu_plan_s* p, int depth, const RSParams& prm, int grid, cudaStream_t st)
{
    if (plan_sr(p)) return rs_launch_bf16sr(p->shape, p->radius, depth, prm, grid, st);
    switch (p->dtype) {
    case EBISU_F64: return rs_launch_f64(p->shape, p->radius, depth, prm, grid, st);
    case EBISU_F32: return rs_launch_f32(p->shape, p->radius, depth, prm, grid, st);
    default: return rs_launch_bf16(p->shape, p->radius, depth, prm, grid, st);
    }
}

cudaError_t rs3_launch(const ebisu_plan_s* p, int depth, const RS3Params& prm, int grid, cudaStream_t st)
{
    if (plan_sr(p)) return rs3_launch_bf16sr(p->shape, p->radius, depth, prm, grid, st);
    switch (p->dtype) {
    case EBISU_F64: return rs3_launch_f64(p->shape, p->radius, depth, prm, grid, st);
    case EBISU_F32: return rs3_launch_f32(p->shape, p->radius, depth, prm, grid, st);
    case EBISU_BF16: return rs3_launch_bf16(p->shape, p->radius, depth, prm, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t rs3_occupancy(const ebisu_plan_s* p, int depth, int* blocks)
{
    if (plan_sr(p)) return rs3_occupancy_bf16sr(p->shape, p->radius, depth, blocks);
    switch (p->dtype) {
    case EBISU_F64: return rs3_occupancy_f64(p->shape, p->radius, depth, blocks);
    case EBISU_F32: return rs3_occupancy_f32(p->shape, p->radius, depth, blocks);
    case EBISU_BF16: return rs3_occupancy_bf16(p->shape, p->radius, depth, blocks);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t rs_occupancy(const ebisu_plan_s* p, int depth, bool batch, int* blocks)
{
    if (plan_sr(p)) return rs_occupancy_bf16sr(p->shape, p->radius, depth, batch, blocks);
    switch (p->dtype) {
    case EBISU_F64: return rs_occupancy_f64(p->shape, p->radius, depth, batch, blocks);
    case EBISU_F32: return rs_occupancy_f32(p->shape, p->radius, depth, batch, blocks);
    default: return rs_occupancy_bf16(p->shape, p->radius, depth, batch, blocks);
    }
}

int64_t fill_rs_grid(const ebisu_plan_s* p, const RSLayout& L, const void* in, void* out, void* wsgrid,
                     int64_t steps, bool in_copied_to_ws, RSGrid* g)
{
    memset(g, 0, sizeof(*g));
    const int D = p->prm.depth;
    const int64_t nb = (steps + D - 1) / D;
    g->src0 = in_copied_to_ws ? wsgrid : in;
    g->out = out;
    g->ws = wsgrid;
    g->n0 = p->n[0];
    g->lds = p->lds;
    g->n2 = (int32_t)p->n[2];
    g->pad = p->pad;
    g->periodic = p->boundary == EBISU_PERIODIC;
    g->S = L.S;
    g->H = L.H;
    g->nstrips = L.nstrips;
    g->nsegs = L.nsegs;
    g->nblocks = (int32_t)nb;
    g->depth_last = (int32_t)(steps - (nb - 1) * D);
    g->sr_key = p->sr_key;
    for (int k = 0; k < p->npts; ++k) {
        g->coef[k] = p->coef[k];
        g->coef_f[k] = (float)p->coef[k];
    }
    if (!g->periodic) {
        // the kernel never writes pad cells: the buffers blocks write get the
        // input's pad during the first block
        void* d0 = ((nb - 1) % 2 == 0) ? out : wsgrid;
        void* d1 = (nb >= 2) ? (((nb - 2) % 2 == 0) ? out : wsgrid) : nullptr;
        if (d0 && d0 != g->src0 && d0 != in) g->pad_dst0 = d0;
        if (d1 && d1 != g->src0 && d1 != in) g->pad_dst1 = d1;
    }
    return nb;
}

// A run of the 3D register-streaming build (FP64: depth 1; FP32/BF16: depth 2 or
// 3).  The kernel never writes pad cells: the buffers it writes first get the
// input's pad from a copy kernel.
static int run_rs3(ebisu_plan_t p, const void* in, void* out, int64_t steps, void* ws, cudaStream_t st,
                   int debug_stall)
{
    const ebisu_params& q = p->prm;
    RSLayout L;
    int rc = rs_layout(p, q, &L);
    if (rc != EBISU_OK) return rc;
    const int D = q.depth;
    const int64_t nb = (steps + D - 1) / D;
    const int64_t ntiles = (int64_t)L.nstrips * L.nbands * L.nsegs;
    const DeviceInfo& dv = device_info();
    if (nb * ntiles + 64LL * 16 * dv.sms * kRSWarps >= (1LL << 32)) return EBISU_ERR_UNSUPPORTED;
    const size_t bytes = (size_t)p->elems * p->esize;
    void* wsgrid = (char*)ws + kControlBytes;
    cudaError_t e = cudaSuccess;
    const bool copy_in = (in == out) && (nb % 2 == 1);
    if (copy_in) {
        e = cudaMemcpyAsync(wsgrid, in, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail_cuda(e);
    }
    const void* src0 = copy_in ? wsgrid : in;
    const bool per = p->boundary == EBISU_PERIODIC;
    if (!per) {
        void* d0 = ((nb - 1) % 2 == 0) ? out : wsgrid;
        void* d1 = (nb >= 2) ? (((nb - 2) % 2 == 0) ? out : wsgrid) : nullptr;
        void* h0 = (d0 != src0 && d0 != in) ? d0 : nullptr;
        void* h1 = (d1 && d1 != src0 && d1 != in) ? d1 : nullptr;
        if (h0 || h1) {
            e = pad_copy(p, src0, h0, h1, st);
            if (e != cudaSuccess) return fail_cuda(e);
        }
    }
    RS3Params prm;
    memset(&prm, 0, sizeof(prm));
    prm.src0 = src0;
    prm.out = out;
    prm.ws = wsgrid;
    for (int i = 0; i < 3; ++i) prm.n[i] = p->n[i];
    prm.lds = p->lds;
    prm.ld1 = p->ld1;
    prm.nitems = nb * ntiles;
    prm.ctl = (Control*)ws;
    prm.timeout_ns = wait_timeout_ns();
    prm.pad = p->pad;
    prm.periodic = per ? 1 : 0;
    prm.S = L.S;
    prm.H = L.H;
    prm.nstrips = L.nstrips;
    prm.nbands = L.nbands;
    prm.nsegs = L.nsegs;
    prm.nblocks = (int32_t)nb;
    prm.depth_last = (int32_t)(steps - (nb - 1) * D);
    prm.debug_stall = debug_stall;
    prm.sr_key = p->sr_key;
    for (int k = 0; k < p->npts; ++k) {
        prm.coef[k] = p->coef[k];
        prm.coef_f[k] = (float)p->coef[k];
    }
    int occ = 0;
    e = rs3_occupancy(p, D, &occ);
    if (e != cudaSuccess) return fail_cuda(e);
    if (occ < 1) return EBISU_ERR_UNSUPPORTED;
    int64_t grid = (int64_t)std::min(occ, q.ctas_per_sm) * dv.sms;
    grid = std::min<int64_t>(grid, (prm.nitems + kRSWarps - 1) / kRSWarps);
    e = rs3_launch(p, D, prm, (int)grid, st);
    if (e != cudaSuccess) return fail_cuda(e);
    return EBISU_OK;
}

static int run_rs(ebisu_plan_t p, const void* in, void* out, int64_t steps, void* ws, cudaStream_t st,
                  int debug_stall)
{
    if (p->ndim == 3) return run_rs3(p, in, out, steps, ws, st, debug_stall);
    const ebisu_params& q = p->prm;
    RSLayout L;
    int rc = rs_layout(p, q, &L);
    if (rc != EBISU_OK) return rc;
    const int D = q.depth;
    const int64_t nb = (steps + D - 1) / D;
    const int64_t ntiles = (int64_t)L.nstrips * L.nsegs;
    const DeviceInfo& dv = device_info();
    // the queue head is a 32-bit counter that every warp overshoots once
    if (nb * ntiles + 64LL * 16 * dv.sms * kRSWarps >= (1LL << 32)) return EBISU_ERR_UNSUPPORTED;
    const size_t bytes = (size_t)p->elems * p->esize;
    void* wsgrid = (char*)ws + kControlBytes;
    cudaError_t e = cudaSuccess;
    const bool copy_in = (in == out) && (nb % 2 == 1);
    if (copy_in) {
        e = cudaMemcpyAsync(wsgrid, in, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail_cuda(e);
    }
    RSParams prm;
    memset(&prm, 0, sizeof(prm));
    fill_rs_grid(p, L, in, out, wsgrid, steps, copy_in, &prm.g);
    prm.nitems = nb * ntiles;
    prm.ctl = (Control*)ws;
    prm.timeout_ns = wait_timeout_ns();
    prm.debug_stall = debug_stall;
    int occ = 0;
    e = rs_occupancy(p, D, false, &occ);
    if (e != cudaSuccess) return fail_cuda(e);
    if (occ < 1) return EBISU_ERR_UNSUPPORTED;
    int64_t grid = (int64_t)std::min(occ, q.ctas_per_sm) * dv.sms;
    grid = std::min<int64_t>(grid, (prm.nitems + kRSWarps - 1) / kRSWarps);
    e = rs_launch(p, D, prm, (int)grid, st);
    if (e != cudaSuccess) return fail_cuda(e);
    return EBISU_OK;
}

}  // namespace ebisu

extern "C" {

const char* ebisu_status_string(int s)
{
    switch (s) {
    case EBISU_OK: return "ok";
    case EBISU_ERR_INVALID_ARG: return "invalid argument";
    case EBISU_ERR_UNSUPPORTED: return "unsupported stencil, size or parameters";
    case EBISU_ERR_CUDA: return "CUDA error";
    case EBISU_ERR_OOM: return "out of host memory";
    case EBISU_ERR_BUDGET: return "request exceeds the HBM budget";
    case EBISU_ERR_TIMEOUT: return "a device-side wait timed out";
    case EBISU_ERR_DEVICE_FAULT: return "kernel reported an inconsistent state";
    case EBISU_ERR_NOT_READY: return "not ready";
    default: return "unknown status";
    }
}

int ebisu_version(void) { return 10000; }

const char* ebisu_last_cuda_error(void) { return g_err; }

int ebisu_plan_create(int ndim, const int64_t* dims, int shape, int radius, const double* coeffs, int dtype,
                      int boundary, ebisu_plan_t* out)
{
    if (!out || !dims || !coeffs) return EBISU_ERR_INVALID_ARG;
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return EBISU_ERR_INVALID_ARG;
    if (shape < EBISU_STAR || shape > EBISU_J3D17PT) return EBISU_ERR_INVALID_ARG;
    if (dtype != EBISU_F64 && dtype != EBISU_F32 && dtype != EBISU_BF16) return EBISU_ERR_INVALID_ARG;
    if (boundary != EBISU_DIRICHLET && boundary != EBISU_PERIODIC) return EBISU_ERR_INVALID_ARG;
    if (radius < 1) return EBISU_ERR_INVALID_ARG;
    if ((shape == EBISU_STAR && radius > 3) || (shape == EBISU_BOX && radius > 2)) return EBISU_ERR_UNSUPPORTED;
    if ((shape == EBISU_POISSON || shape == EBISU_J3D17PT) && (ndim != 3 || radius != 1))
        return EBISU_ERR_UNSUPPORTED;
    for (int i = 0; i < ndim; ++i) {
        if (dims[i] < 1) return EBISU_ERR_INVALID_ARG;
        if (boundary == EBISU_PERIODIC && dims[i] < 2 * radius + 1) return EBISU_ERR_UNSUPPORTED;
        if (dims[i] > (int64_t)1 << 31) return EBISU_ERR_UNSUPPORTED;
    }
    ebisu_plan_s* p = new (std::nothrow) ebisu_plan_s();
    if (!p) return EBISU_ERR_OOM;
    p->ndim = ndim;
    p->shape = shape;
    p->radius = radius;
    p->dtype = dtype;
    p->boundary = boundary;
    for (int i = 0; i < ndim; ++i) p->dims[i] = dims[i];
    p->npts = (shape == EBISU_STAR)      ? 2 * ndim * radius + 1
              : (shape == EBISU_POISSON) ? 19
              : (shape == EBISU_J3D17PT) ? 17
              : (ndim == 3 ? (2 * radius + 1) * (2 * radius + 1) * (2 * radius + 1) : (2 * radius + 1) * (2 * radius + 1));
    for (int k = 0; k < p->npts; ++k) p->coef[k] = coeffs[k];
    p->esize = (dtype == EBISU_F64) ? 8 : (dtype == EBISU_F32 ? 4 : 2);
    p->pad = (boundary == EBISU_DIRICHLET) ? radius : 0;
    if (ndim == 2) {
        p->n[0] = dims[0];
        p->n[1] = 1;
        p->n[2] = dims[1];
        p->pad1 = 0;
        p->ext[0] = dims[0] + 2 * p->pad;
        p->ext[1] = 1;
        p->ext[2] = dims[1] + 2 * p->pad;
        p->lds = p->ext[2];
        p->ld1 = 0;
    } else {
        for (int i = 0; i < 3; ++i) p->n[i] = dims[i];
        p->pad1 = p->pad;
        for (int i = 0; i < 3; ++i) p->ext[i] = dims[i] + 2 * p->pad;
        p->lds = p->ext[1] * p->ext[2];
        p->ld1 = p->ext[2];
    }
    p->elems = p->ext[0] * p->ext[1] * p->ext[2];
    ebisu_params best;
    double pred = 0;
    if (rank_candidates(p, 1000, &best, &pred, 1) < 1) {
        // fall back to the smallest legal blocked configuration
        memset(&best, 0, sizeof(best));
        best.tile_x = 64;
        best.tile_y = 8;
        best.depth = 1;
        best.ctas_per_sm = 1;
        best.threads = kThreads;
    }
    p->prm = best;
    p->tb_prm = best;
    // 2D FP32/BF16: the register-streaming build is 2-5x faster than the
    // shared-memory one at every measured stencil; default to it (the
    // tuner still times both).  Segments of 128 rows (64 for BF16) give
    // every resident warp several tiles on large grids.
    if (p->ndim == 2 && p->dtype != EBISU_F64) {
        ebisu_params v{};
        v.variant = 2;
        v.fused_variant = 2;
        v.depth = rs_preferred_depth((int)p->esize, p->shape, p->radius);
        v.tile_s = (int32_t)std::max<int64_t>((int64_t)v.depth * p->radius,
                                              std::min<int64_t>(p->n[0], p->dtype == EBISU_BF16 ? 64 : 128));
        v.ctas_per_sm = 8;
        v.threads = kRSThreads;
        RSLayout L;
        if (rs_layout(p, v, &L) == EBISU_OK) {
            v.tile_x = L.S;
            v.tile_y = 1;
            v.tile_s = L.H;
            p->prm = v;
        }
    }
    *out = p;
    return EBISU_OK;
}

// Offsets of a named shape in canonical order (the kernels' tables, host side).
static int shape_offsets(int ndim, int shape, int r, int* oz, int* oy, int* ox)
{
    int n = 0;
    const int zr = ndim == 3 ? r : 0;
    for (int a = -zr; a <= zr; ++a)
        for (int b = -r; b <= r; ++b)
            for (int c = -r; c <= r; ++c) {
                const int nz = (a != 0) + (b != 0) + (c != 0);
                if (shape == EBISU_STAR && nz > 1) continue;
                if ((shape == EBISU_POISSON || shape == EBISU_J3D17PT) && nz > 2) continue;
                if (shape == EBISU_J3D17PT && a != 0 && b == 0 && c == 0) continue;
                oz[n] = a;
                oy[n] = b;
                ox[n] = c;
                ++n;
            }
    return n;
}

int ebisu_plan_create_offsets(int ndim, const int64_t* dims, int npts, const int32_t* offsets, const double* coeffs,
                              int dtype, int boundary, ebisu_plan_t* out)
{
    if (!out || !dims || !offsets || !coeffs || npts < 1 || npts > kMaxPoints) return EBISU_ERR_INVALID_ARG;
    if (ndim != 2 && ndim != 3) return EBISU_ERR_INVALID_ARG;
    *out = nullptr;
    int r = 0;
    for (int k = 0; k < npts; ++k) {
        const int32_t* o = offsets + 3 * k;
        if (ndim == 2 && o[0] != 0) return EBISU_ERR_INVALID_ARG;
        for (int i = 0; i < 3; ++i) r = std::max(r, std::abs(o[i]));
        for (int j = 0; j < k; ++j)
            if (o[0] == offsets[3 * j] && o[1] == offsets[3 * j + 1] && o[2] == offsets[3 * j + 2])
                return EBISU_ERR_INVALID_ARG;  // repeated offset
    }
    if (r < 1) r = 1;
    if (r > 3) return EBISU_ERR_UNSUPPORTED;
    // the coefficient of offset (a, b, c), 0 where the list has none
    auto coef_of = [&](int a, int b, int c, bool* found) {
        for (int k = 0; k < npts; ++k)
            if (offsets[3 * k] == a && offsets[3 * k + 1] == b && offsets[3 * k + 2] == c) {
                *found = true;
                return coeffs[k];
            }
        *found = false;
        return 0.0;
    };
    // a named shape whose set is exactly the list runs its own kernels;
    // any other list runs on the box of its radius with zero weights on the
    // offsets it lacks (x + 0*u = x for finite u, so the sum is unchanged)
    int oz[kMaxPoints], oy[kMaxPoints], ox[kMaxPoints];
    double c[kMaxPoints];
    for (int shape : {EBISU_STAR, EBISU_POISSON, EBISU_J3D17PT, EBISU_BOX}) {
        if ((shape == EBISU_POISSON || shape == EBISU_J3D17PT) && (ndim != 3 || r != 1)) continue;
        if (shape == EBISU_BOX && r > 2) continue;
        const int n = shape_offsets(ndim, shape, r, oz, oy, ox);
        bool covers = true;
        int matched = 0;
        for (int k = 0; k < n; ++k) {
            bool f = false;
            c[k] = coef_of(oz[k], oy[k], ox[k], &f);
            matched += f ? 1 : 0;
        }
        if (matched != npts) covers = false;  // some offset lies outside this shape
        if (!covers || (shape != EBISU_BOX && n != npts)) continue;
        return ebisu_plan_create(ndim, dims, shape, r, c, dtype, boundary, out);
    }
    return EBISU_ERR_UNSUPPORTED;  // radius 3 and not a star: no box of that radius is built
}

int ebisu_plan_destroy(ebisu_plan_t plan)
{
    delete plan;
    return EBISU_OK;
}

int ebisu_plan_npoints(ebisu_plan_t plan, int* npts)
{
    if (!plan || !npts) return EBISU_ERR_INVALID_ARG;
    *npts = plan->npts;
    return EBISU_OK;
}

int ebisu_plan_grid_elems(ebisu_plan_t plan, int64_t* elems)
{
    if (!plan || !elems) return EBISU_ERR_INVALID_ARG;
    *elems = plan->elems;
    return EBISU_OK;
}

int ebisu_plan_get_params(ebisu_plan_t plan, ebisu_params* q)
{
    if (!plan || !q) return EBISU_ERR_INVALID_ARG;
    *q = plan->prm;
    return EBISU_OK;
}

int ebisu_plan_set_params(ebisu_plan_t plan, const ebisu_params* q)
{
    if (!plan || !q) return EBISU_ERR_INVALID_ARG;
    ebisu_params v = *q;
    if (v.fused_variant != 0 && v.fused_variant != 2) return EBISU_ERR_INVALID_ARG;
    // the build whose parameters the tile and depth fields hold
    const int build = (v.variant == 1) ? v.fused_variant : v.variant;
    v.threads = (build == 2) ? kRSThreads : kThreads;
    if (v.ctas_per_sm == 0) v.ctas_per_sm = 1;
    const int rc = check_params(plan, v);
    if (rc != EBISU_OK) return rc;
    if (v.variant == 2) {
        RSLayout L;
        rs_layout(plan, v, &L);
        v.tile_x = L.S;  // derived: 128 - 2 * depth * radius (3D: 64 - 2 * radius)
        v.tile_y = L.TY;
        v.tile_s = L.H;
        v.fused_variant = 2;
    } else if (build == 0) {
        plan->tb_prm = v;
        plan->tb_prm.variant = 0;
        plan->tb_prm.fused_variant = 0;
        if (v.variant == 0) v.fused_variant = 0;
    }
    plan->prm = v;
    return EBISU_OK;
}

int ebisu_plan_set_rounding(ebisu_plan_t plan, int rounding, uint64_t seed)
{
    if (!plan) return EBISU_ERR_INVALID_ARG;
    if (rounding != EBISU_ROUND_NEAREST && rounding != EBISU_ROUND_STOCHASTIC) return EBISU_ERR_INVALID_ARG;
    if (rounding == EBISU_ROUND_STOCHASTIC && (plan->dtype != EBISU_BF16 || plan->field)) return EBISU_ERR_UNSUPPORTED;
    plan->rounding = rounding;
    plan->sr_seed = seed;
    plan->sr_key = sr_plan_key(seed);
    if (!plan_sr(plan)) return EBISU_OK;
    // the shared-memory build has no stochastic-rounding form: move the plan
    // to the register-streaming build where one exists, else to the
    // one-step kernel
    const ebisu_params& q = plan->prm;
    if (q.variant == 2 || (q.variant == 1 && q.fused_variant == 2)) return EBISU_OK;
    ebisu_params v{};
    v.variant = 2;
    v.fused_variant = 2;
    v.ctas_per_sm = 8;
    v.threads = kRSThreads;
    const int es = (int)plan->esize;
    if (plan->ndim == 2) {
        v.depth = rs_preferred_depth(es, plan->shape, plan->radius);
        v.tile_s = (int32_t)std::max<int64_t>((int64_t)v.depth * plan->radius, std::min<int64_t>(plan->n[0], 64));
    } else {
        v.depth = rs3_built(es, plan->shape, plan->radius) ? rs3_depth(es, plan->shape, plan->radius, 1) : 1;
        v.tile_s = (int32_t)std::min<int64_t>(plan->n[0], 64);
    }
    RSLayout L;
    if (rs_layout(plan, v, &L) == EBISU_OK) {
        v.tile_x = L.S;
        v.tile_y = L.TY;
        v.tile_s = L.H;
        plan->prm = v;
    } else {
        plan->prm.variant = 1;  // no fused build of this stencil: the one-step kernel
        plan->prm.fused_variant = 0;
    }
    return EBISU_OK;
}

int ebisu_plan_set_ablation(ebisu_plan_t plan, int mask)
{
    if (!plan) return EBISU_ERR_INVALID_ARG;
    const int steps[] = {0, EBISU_ABLATE_REGISTER_REUSE, EBISU_ABLATE_REGISTER_REUSE | EBISU_ABLATE_LAZY,
                         EBISU_ABLATE_REGISTER_REUSE | EBISU_ABLATE_LAZY | EBISU_ABLATE_PREFETCH,
                         EBISU_ABLATE_REGISTER_REUSE | EBISU_ABLATE_LAZY | EBISU_ABLATE_PREFETCH |
                             EBISU_ABLATE_CIRCULAR};
    bool known = false;
    for (int m : steps) known = known || (m == mask);
    if (!known) return EBISU_ERR_INVALID_ARG;
    if (mask != 0 && (plan->shape != EBISU_STAR || plan->radius != 1 || plan->dtype == EBISU_BF16 ||
                      plan_sr(plan)))
        return EBISU_ERR_UNSUPPORTED;
    plan->ablate = mask;
    return EBISU_OK;
}

int ebisu_plan_set_coefficient_field(ebisu_plan_t plan, const void* field)
{
    if (!plan) return EBISU_ERR_INVALID_ARG;
    if (field && (plan_sr(plan) || plan->ablate)) return EBISU_ERR_UNSUPPORTED;
    const size_t align = plan->dtype == EBISU_F64 ? 8 : 4;
    if (((uintptr_t)field) % align != 0) return EBISU_ERR_INVALID_ARG;
    plan->field = field;
    return EBISU_OK;
}

int ebisu_plan_get_rounding(ebisu_plan_t plan, int* rounding, uint64_t* seed)
{
    if (!plan || !rounding) return EBISU_ERR_INVALID_ARG;
    *rounding = plan->rounding;
    if (seed) *seed = plan->sr_seed;
    return EBISU_OK;
}

int ebisu_plan_rs_depths(ebisu_plan_t plan, int* shallow, int* deep)
{
    if (!plan || !shallow || !deep) return EBISU_ERR_INVALID_ARG;
    if (plan->ndim != 2) {
        const int es = (int)plan->esize;
        const bool b = rs3_built(es, plan->shape, plan->radius);
        *shallow = b ? rs3_depth(es, plan->shape, plan->radius, 0) : 0;
        *deep = b ? rs3_depth(es, plan->shape, plan->radius, 1) : 0;
        return EBISU_OK;
    }
    *shallow = rs_depth((int)plan->esize, plan->shape, plan->radius, 0);
    *deep = rs_depth((int)plan->esize, plan->shape, plan->radius, 1);
    return EBISU_OK;
}

int ebisu_plan_workspace_bytes(ebisu_plan_t plan, size_t* bytes)
{
    if (!plan || !bytes) return EBISU_ERR_INVALID_ARG;
    *bytes = kControlBytes + align_up((size_t)plan->elems * plan->esize, kAlign);
    return EBISU_OK;
}

static int run_common(ebisu_plan_t p, const void* in, void* out, int64_t steps, void* ws, void* stream,
                      bool naive, int debug_stall)
{
    if (!p || !in || !out || !ws) return EBISU_ERR_INVALID_ARG;
    if (steps < 0) return EBISU_ERR_INVALID_ARG;
    if (((uintptr_t)ws) % kAlign != 0) return EBISU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)p->elems * p->esize;
    void* wsgrid = (char*)ws + kControlBytes;
    cudaError_t e = cudaMemsetAsync(ws, 0, kControlBytes, st);
    if (e != cudaSuccess) return fail_cuda(e);
    if (steps == 0) {
        if (in != out) {
            e = cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return fail_cuda(e);
        }
        return EBISU_OK;
    }
    if (!naive && !p->field && p->prm.variant == 2) return run_rs(p, in, out, steps, ws, st, debug_stall);
    if (naive || p->prm.variant == 1 || p->field) {
        // one launch per step; buffers alternate so that the last lands in out
        const void* src = in;
        if (in == out && (steps % 2 == 1)) {
            e = cudaMemcpyAsync(wsgrid, in, bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return fail_cuda(e);
            src = wsgrid;
        }
        void* d0 = ((steps - 1) % 2 == 0) ? out : wsgrid;
        void* d1 = (steps >= 2) ? (((steps - 2) % 2 == 0) ? out : wsgrid) : nullptr;
        void* h0 = (d0 != src && d0 != in) ? d0 : nullptr;
        void* h1 = (d1 && d1 != src && d1 != in) ? d1 : nullptr;
        e = pad_copy(p, src, h0, h1, st);
        if (e != cudaSuccess) return fail_cuda(e);
        for (int64_t s = 0; s < steps; ++s) {
            void* dst = ((steps - 1 - s) % 2 == 0) ? out : wsgrid;
            e = p->field ? naive_vc_launch(p, src, dst, st) : naive_launch(p, src, dst, s + 1, st);
            if (e != cudaSuccess) return fail_cuda(e);
            src = dst;
        }
        return EBISU_OK;
    }
    const ebisu_params& q = p->prm;
    const int d = (int)std::min<int64_t>(q.depth, steps);
    const int64_t nb = (steps + d - 1) / d;
    const bool copy_in = (in == out) && (nb % 2 == 1);
    if (copy_in) {
        e = cudaMemcpyAsync(wsgrid, in, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail_cuda(e);
    }
    TBParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.nitems = fill_grid_desc(p, in, out, wsgrid, steps, copy_in, &prm.g);
    prm.grids = nullptr;
    prm.items = nullptr;
    prm.ctl = (Control*)ws;
    prm.timeout_ns = wait_timeout_ns();
    prm.debug_stall = debug_stall;
    ebisu_params qd = q;
    qd.depth = d;
    prm.smem_plane = (int32_t)plane_capacity(p, qd);
    prm.g.plane_cap = prm.smem_plane;
    const size_t smem = tb_smem_bytes(p, qd);
    const int variant = kernel_variant(p->dtype, q.ctas_per_sm);
    int occ = 0;
    e = p->ablate ? tb_ablate_occupancy(p->esize, p->ndim, p->ablate, smem, &occ)
                  : tb_occupancy(p, variant, smem, &occ);
    if (e != cudaSuccess) return fail_cuda(e);
    if (occ < 1) return EBISU_ERR_UNSUPPORTED;
    const DeviceInfo& dv = device_info();
    int64_t grid = (int64_t)std::min(occ, q.ctas_per_sm) * dv.sms;
    grid = std::min<int64_t>(grid, prm.nitems);
    e = p->ablate ? tb_ablate_launch(p->esize, p->ndim, p->ablate, prm, (int)grid, smem, st)
                  : tb_launch(p, variant, prm, (int)grid, smem, st);
    if (e != cudaSuccess) return fail_cuda(e);
    return EBISU_OK;
}

int ebisu_run(ebisu_plan_t plan, const void* in, void* out, int64_t steps, void* workspace, void* stream)
{
    return run_common(plan, in, out, steps, workspace, stream, false, 0);
}

int ebisu_run_naive(ebisu_plan_t plan, const void* in, void* out, int64_t steps, void* workspace, void* stream)
{
    return run_common(plan, in, out, steps, workspace, stream, true, 0);
}

// Test hook (not in the public header): a blocked run whose first dependency
// wait targets a count nothing reaches, so the bounded wait must give up and
// report EBISU_ERR_TIMEOUT.
int ebisu_debug_run_stalled(ebisu_plan_t plan, const void* in, void* out, int64_t steps, void* workspace,
                            void* stream)
{
    return run_common(plan, in, out, steps, workspace, stream, false, 1);
}

int ebisu_sync(void* workspace, void* stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e);
    if (!workspace) return EBISU_OK;
    int st = 0;
    e = cudaMemcpy(&st, workspace, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(e);
    if (st != 0) {
        cudaMemset(workspace, 0, sizeof(int));
        return st;
    }
    return EBISU_OK;
}

int ebisu_reduce(ebisu_plan_t p, const void* a, const void* b, double* result, void* ws, void* stream)
{
    if (!p || !a || !result || !ws) return EBISU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    PadParams g = pad_params(p);
    double* part = (double*)((char*)ws + kControlBytes);
    double* fin = (double*)((char*)ws + 2048);
    int64_t nparts = 0;
    cudaError_t e;
    switch (p->dtype) {
    case EBISU_F64: e = reduce_partial_f64(a, b, part, g, &nparts, st); break;
    case EBISU_F32: e = reduce_partial_f32(a, b, part, g, &nparts, st); break;
    default: e = reduce_partial_bf16(a, b, part, g, &nparts, st); break;
    }
    if (e != cudaSuccess) return fail_cuda(e);
    e = reduce_final(part, nparts, fin, st);
    if (e != cudaSuccess) return fail_cuda(e);
    e = cudaMemcpyAsync(result, fin, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return fail_cuda(e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e);
    return EBISU_OK;
}

int ebisu_probe_device(double* out)
{
    if (!out) return EBISU_ERR_INVALID_ARG;
    cudaError_t e = probe_device(out);
    if (e != cudaSuccess) return fail_cuda(e);
    record_device_rates(out);  // the cost model uses the same figures from now on
    return EBISU_OK;
}

}  // extern "C"
