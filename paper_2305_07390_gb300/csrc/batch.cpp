// batch.cpp -- many independent problems in one persistent launch per kernel
// type (ebisu_batch_*).
//
// Problems that share (ndim, shape, radius, dtype) and kernel build form a
// group and run in one launch of that temporally blocked kernel: the
// register-streaming build (2D plans whose tuner chose it, grouped by depth)
// or the shared-memory build (every other plan, with its shared-memory
// parameters).  The group's work table lists
// (problem, temporal block, tile) items in "waves": every tile of block 0 of
// every problem, then block 1 of every problem, and so on, so that while one
// problem's tiles of block b finish, the CTAs work on other problems instead
// of waiting (the dependency counters of Section 4.3.2's one-wait-per-block
// scheme are per problem, or per tile in the register-streaming build).
// Each problem keeps its own plan parameters (tile, depth), so results are
// bit-identical to running it alone.
//
// Workspace layout (all offsets 256-byte aligned):
//   per group: Control block with one completion counter per problem
//     (shared-memory build) or per tile of every member (register streaming)
//   GridDesc table and RSGrid table (all problems), work tables (per group),
//   one ping-pong grid buffer per problem.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "plan.h"

using namespace ebisu;

struct BatchGroup {
    const ebisu_plan_s* kind = nullptr;  // representative plan (kernel type)
    int variant = 0;                     // kernel build (same for all members)
    bool rs = false;                     // register-streaming build (variant = depth)
    std::vector<int> members;            // problem indices
    size_t ctl_off = 0, items_off = 0;
    int64_t nitems = 0;
    size_t smem = 0;
    int plane_cap = 0;
    int grid = 0;
};

struct ebisu_batch_s {
    int n = 0;
    std::vector<ebisu_plan_s> plans;
    std::vector<BatchGroup> groups;
    std::vector<GridDesc> descs;
    std::vector<RSGrid> rsdescs;
    std::vector<int32_t> tile_base;  // register streaming: first tile counter of a problem
    std::vector<RSLayout> rsl;
    std::vector<std::vector<int32_t>> items;
    std::vector<const void*> in;
    std::vector<void*> out;
    std::vector<int64_t> steps;
    std::vector<size_t> grid_off;
    std::vector<bool> copy_in;
    size_t desc_off = 0, rsdesc_off = 0, total = 0;
    void* ws = nullptr;
    bool uploaded = false;
    // several kernel groups run concurrently: each on a stream of its own,
    // forked from and joined back into the caller's stream by events
    std::vector<cudaStream_t> gstreams;
    std::vector<cudaEvent_t> gdone;
    cudaEvent_t fork = nullptr;
    ~ebisu_batch_s()
    {
        // (destruction with work in flight is allowed: the runtime releases
        // streams and events once their work completes)
        for (cudaStream_t s : gstreams) cudaStreamDestroy(s);
        for (cudaEvent_t e : gdone) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
    }
};

namespace {

struct Key {
    int ndim, shape, radius, dtype, rounding, rs, variant;
    bool operator<(const Key& o) const
    {
        return std::tie(ndim, shape, radius, dtype, rounding, rs, variant) <
               std::tie(o.ndim, o.shape, o.radius, o.dtype, o.rounding, o.rs, o.variant);
    }
};

// Does a plan run the register-streaming build (its tuner chose it)?
bool uses_rs(const ebisu_plan_s* p)
{
    const ebisu_params& q = p->prm;
    if (p->ndim != 2) return false;
    if (!(q.variant == 2 || (q.variant == 1 && q.fused_variant == 2))) return false;
    ebisu_params v = q;
    v.variant = 2;
    return rs_layout(p, v, nullptr) == EBISU_OK;
}

int64_t nblocks_of(const ebisu_plan_s* p, int64_t steps)
{
    if (steps <= 0) return 0;
    const int d = (int)std::min<int64_t>(p->prm.depth, steps);
    return (steps + d - 1) / d;
}

int64_t ntiles_of(const ebisu_plan_s* p)
{
    if (p->prm.variant == 2) {
        RSLayout L;
        rs_layout(p, p->prm, &L);
        return (int64_t)L.nstrips * L.nsegs;
    }
    GridDesc g;
    fill_grid_desc(p, nullptr, nullptr, nullptr, 1, false, &g);
    return g.ntiles;
}

// Lay out the workspace and the work tables (host only).
int layout(ebisu_batch_s* b)
{
    const int n = b->n;
    std::map<Key, int> gid;
    for (int i = 0; i < n; ++i) {
        // batches always run a fused kernel with the plan's tile and depth
        // (a plan whose tuner preferred the one-step kernel keeps the best
        // fused parameters too)
        const bool rs = uses_rs(&b->plans[i]);
        // stochastic rounding exists in the register-streaming build only;
        // per-cell weights in the one-step kernel only
        if (!rs && plan_sr(&b->plans[i]) && b->steps[i] > 0) return EBISU_ERR_UNSUPPORTED;
        if (b->plans[i].field && b->steps[i] > 0) return EBISU_ERR_UNSUPPORTED;
        if (rs) {
            b->plans[i].prm.variant = 2;
        } else {
            b->plans[i].prm = b->plans[i].tb_prm;
            b->plans[i].prm.variant = 0;
        }
        const ebisu_plan_s* p = &b->plans[i];
        if (b->steps[i] <= 0) continue;  // zero steps: plain copy, no kernel
        Key k{p->ndim, p->shape, p->radius, p->dtype, plan_sr(p) ? 1 : 0, rs ? 1 : 0,
              rs ? p->prm.depth : kernel_variant(p->dtype, p->prm.ctas_per_sm)};
        auto it = gid.find(k);
        if (it == gid.end()) {
            it = gid.emplace(k, (int)b->groups.size()).first;
            b->groups.emplace_back();
            b->groups.back().kind = p;
            b->groups.back().variant = k.variant;
            b->groups.back().rs = rs;
        }
        b->groups[it->second].members.push_back(i);
    }
    size_t off = 0;
    b->tile_base.assign(n, 0);
    b->rsl.assign(n, RSLayout{});
    for (auto& g : b->groups) {
        g.ctl_off = off;
        size_t counters = g.members.size();
        if (g.rs) {
            counters = 0;
            for (int m : g.members) {
                rs_layout(&b->plans[m], b->plans[m].prm, &b->rsl[m]);
                b->tile_base[m] = (int32_t)counters;
                counters += (size_t)b->rsl[m].nstrips * b->rsl[m].nsegs;
            }
            if (counters >= (1u << 31)) return EBISU_ERR_UNSUPPORTED;
        }
        off += align_up(offsetof(Control, done) + sizeof(unsigned) * counters, kAlign);
    }
    b->desc_off = off;
    off += align_up(sizeof(GridDesc) * (size_t)std::max(n, 1), kAlign);
    b->rsdesc_off = off;
    off += align_up(sizeof(RSGrid) * (size_t)std::max(n, 1), kAlign);
    b->items.resize(b->groups.size());
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        BatchGroup& g = b->groups[gi];
        int64_t maxnb = 0;
        for (int m : g.members) maxnb = std::max(maxnb, nblocks_of(&b->plans[m], b->steps[m]));
        std::vector<int32_t>& it = b->items[gi];
        for (int64_t blk = 0; blk < maxnb; ++blk)
            for (size_t k = 0; k < g.members.size(); ++k) {
                const int m = g.members[k];
                if (blk >= nblocks_of(&b->plans[m], b->steps[m])) continue;
                const int64_t nt = ntiles_of(&b->plans[m]);
                for (int64_t t = 0; t < nt; ++t) {
                    it.push_back(m);
                    it.push_back((int32_t)blk);
                    it.push_back((int32_t)t);
                }
            }
        g.nitems = (int64_t)it.size() / 3;
        g.items_off = off;
        off += align_up(sizeof(int32_t) * std::max<size_t>(it.size(), 1), kAlign);
        if (g.rs) continue;  // no shared memory
        for (int m : g.members) {
            ebisu_params q = b->plans[m].prm;
            q.depth = (int)std::min<int64_t>(q.depth, b->steps[m]);
            g.smem = std::max(g.smem, tb_smem_bytes(&b->plans[m], q));
            g.plane_cap = std::max<int>(g.plane_cap, (int)plane_capacity(&b->plans[m], q));
        }
        // every member lays its rings out with its own plane stride (its
        // descriptor carries it), so the launch needs the largest member's
        // footprint, which fits because each member's parameters were checked
        if (g.smem + 4096 > device_info().smem_optin) return EBISU_ERR_UNSUPPORTED;
    }
    b->grid_off.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        b->grid_off[i] = off;
        off += align_up((size_t)b->plans[i].elems * b->plans[i].esize, kAlign);
    }
    b->total = off;
    return EBISU_OK;
}

int build(int n, const ebisu_plan_t* plans, const void* const* in, void* const* out, const int64_t* steps,
          ebisu_batch_s** res)
{
    if (n < 1 || !plans || !steps) return EBISU_ERR_INVALID_ARG;
    ebisu_batch_s* b = new (std::nothrow) ebisu_batch_s();
    if (!b) return EBISU_ERR_OOM;
    b->n = n;
    b->plans.reserve(n);
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || steps[i] < 0) {
            delete b;
            return EBISU_ERR_INVALID_ARG;
        }
        b->plans.push_back(*plans[i]);
        b->steps.push_back(steps[i]);
        b->in.push_back(in ? in[i] : nullptr);
        b->out.push_back(out ? out[i] : nullptr);
    }
    const int rc = layout(b);
    if (rc != EBISU_OK) {
        delete b;
        return rc;
    }
    *res = b;
    return EBISU_OK;
}

}  // namespace

extern "C" {

int ebisu_batch_workspace_bytes(int n, const ebisu_plan_t* plans, const int64_t* steps, size_t* bytes)
{
    if (!bytes) return EBISU_ERR_INVALID_ARG;
    ebisu_batch_s* b = nullptr;
    const int rc = build(n, plans, nullptr, nullptr, steps, &b);
    if (rc != EBISU_OK) return rc;
    *bytes = b->total;
    delete b;
    return EBISU_OK;
}

int ebisu_batch_create(int n, const ebisu_plan_t* plans, const void* const* in, void* const* out,
                       const int64_t* steps, void* workspace, void* stream, ebisu_batch_t* res)
{
    if (!res || !in || !out || !workspace) return EBISU_ERR_INVALID_ARG;
    if (((uintptr_t)workspace) % kAlign != 0) return EBISU_ERR_INVALID_ARG;
    *res = nullptr;
    for (int i = 0; i < n; ++i)
        if (!in[i] || !out[i]) return EBISU_ERR_INVALID_ARG;
    ebisu_batch_s* b = nullptr;
    int rc = build(n, plans, in, out, steps, &b);
    if (rc != EBISU_OK) return rc;
    b->ws = workspace;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    b->descs.assign(n, GridDesc{});
    b->rsdescs.assign(n, RSGrid{});
    b->copy_in.assign(n, false);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const BatchGroup& g = b->groups[gi];
        for (size_t k = 0; k < g.members.size(); ++k) {
            const int m = g.members[k];
            const ebisu_plan_s* p = &b->plans[m];
            void* wsg = ws + b->grid_off[m];
            const int64_t nb = nblocks_of(p, b->steps[m]);
            b->copy_in[m] = (b->in[m] == b->out[m]) && (nb % 2 == 1);
            if (g.rs) {
                fill_rs_grid(p, b->rsl[m], b->in[m], b->out[m], wsg, b->steps[m], b->copy_in[m], &b->rsdescs[m]);
                b->rsdescs[m].tile_base = b->tile_base[m];
            } else {
                fill_grid_desc(p, b->in[m], b->out[m], wsg, b->steps[m], b->copy_in[m], &b->descs[m]);
                b->descs[m].grid_id = (int32_t)k;
                ebisu_params q = p->prm;
                q.depth = (int)std::min<int64_t>(q.depth, b->steps[m]);
                b->descs[m].plane_cap = (int32_t)plane_capacity(p, q);
            }
        }
    }
    cudaError_t e = cudaMemcpyAsync(ws + b->desc_off, b->descs.data(), sizeof(GridDesc) * n,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + b->rsdesc_off, b->rsdescs.data(), sizeof(RSGrid) * n, cudaMemcpyHostToDevice, st);
    for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
        const auto& it = b->items[gi];
        if (!it.empty())
            e = cudaMemcpyAsync(ws + b->groups[gi].items_off, it.data(), sizeof(int32_t) * it.size(),
                                cudaMemcpyHostToDevice, st);
    }
    // (copies from pageable memory return once the host data is staged, so
    // the host tables may be released after this point)
    for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
        BatchGroup& g = b->groups[gi];
        int occ = 0;
        e = g.rs ? rs_occupancy(g.kind, g.variant, true, &occ) : tb_occupancy(g.kind, g.variant, g.smem, &occ);
        if (e != cudaSuccess) break;
        if (occ < 1) {
            delete b;
            return EBISU_ERR_UNSUPPORTED;
        }
        int cps = 1;
        for (int m : g.members) cps = std::max(cps, b->plans[m].prm.ctas_per_sm);
        const int64_t per_cta = g.rs ? kRSWarps : 1;  // work items one CTA takes at a time
        g.grid = (int)std::min<int64_t>((int64_t)std::min(occ, cps) * device_info().sms,
                                        (g.nitems + per_cta - 1) / per_cta);
    }
    if (e != cudaSuccess) {
        delete b;
        return fail_cuda(e);
    }
    b->items.clear();
    b->items.shrink_to_fit();
    int launched = 0;
    for (const BatchGroup& g : b->groups) launched += (g.nitems > 0) ? 1 : 0;
    if (launched > 1) {
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
            cudaStream_t gs = nullptr;
            cudaEvent_t ge = nullptr;
            e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
            if (e == cudaSuccess) b->gstreams.push_back(gs);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ge, cudaEventDisableTiming);
            if (e == cudaSuccess) b->gdone.push_back(ge);
        }
        if (e != cudaSuccess) {
            delete b;
            return fail_cuda(e);
        }
    }
    b->uploaded = true;
    *res = b;
    return EBISU_OK;
}

// Enqueue the batch: counter reset, in-place copies, one launch per group.
// Only stream operations: can be captured into a CUDA graph and replayed.
int ebisu_batch_launch(ebisu_batch_t b, void* stream)
{
    if (!b || !b->uploaded) return EBISU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)b->ws;
    cudaError_t e = cudaSuccess;
    if (b->desc_off > 0) e = cudaMemsetAsync(ws, 0, b->desc_off, st);  // every group's Control
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        const ebisu_plan_s* p = &b->plans[i];
        const size_t bytes = (size_t)p->elems * p->esize;
        if (b->steps[i] == 0) {
            if (b->in[i] != b->out[i]) e = cudaMemcpyAsync(b->out[i], b->in[i], bytes, cudaMemcpyDeviceToDevice, st);
        } else if (b->copy_in[i]) {
            e = cudaMemcpyAsync(ws + b->grid_off[i], b->in[i], bytes, cudaMemcpyDeviceToDevice, st);
        }
    }
    const bool forked = !b->gstreams.empty();
    if (forked && e == cudaSuccess) e = cudaEventRecord(b->fork, st);
    for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
        const BatchGroup& g = b->groups[gi];
        if (g.nitems == 0) continue;
        cudaStream_t gst = st;
        if (forked) {
            gst = b->gstreams[gi];
            e = cudaStreamWaitEvent(gst, b->fork, 0);
            if (e != cudaSuccess) break;
        }
        if (g.rs) {
            RSParams prm;
            memset(&prm, 0, sizeof(prm));
            prm.grids = (const RSGrid*)(ws + b->rsdesc_off);
            prm.items = (const int32_t*)(ws + g.items_off);
            prm.nitems = g.nitems;
            prm.ctl = (Control*)(ws + g.ctl_off);
            prm.timeout_ns = wait_timeout_ns();
            e = rs_launch(g.kind, g.variant, prm, g.grid, gst);
        } else {
            TBParams prm;
            memset(&prm, 0, sizeof(prm));
            prm.grids = (const GridDesc*)(ws + b->desc_off);
            prm.items = (const int32_t*)(ws + g.items_off);
            prm.nitems = g.nitems;
            prm.ctl = (Control*)(ws + g.ctl_off);
            prm.timeout_ns = wait_timeout_ns();
            prm.smem_plane = g.plane_cap;
            e = tb_launch(g.kind, g.variant, prm, g.grid, g.smem, gst);
        }
        if (forked && e == cudaSuccess) {
            e = cudaEventRecord(b->gdone[gi], gst);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->gdone[gi], 0);
        }
    }
    if (e != cudaSuccess) return fail_cuda(e);
    return EBISU_OK;
}

// Status word of every group of a finished batch (after the stream is done).
int ebisu_batch_sync(ebisu_batch_t b, void* stream)
{
    if (!b) return EBISU_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e);
    for (const BatchGroup& g : b->groups) {
        int st = 0;
        e = cudaMemcpy(&st, (char*)b->ws + g.ctl_off, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(e);
        if (st != 0) return st;
    }
    return EBISU_OK;
}

int ebisu_batch_destroy(ebisu_batch_t b)
{
    delete b;
    return EBISU_OK;
}

int ebisu_batch_run(int n, const ebisu_plan_t* plans, const void* const* in, void* const* out, const int64_t* steps,
                    void* workspace, void* stream)
{
    ebisu_batch_t b = nullptr;
    int rc = ebisu_batch_create(n, plans, in, out, steps, workspace, stream, &b);
    if (rc != EBISU_OK) return rc;
    rc = ebisu_batch_launch(b, stream);
    ebisu_batch_destroy(b);
    return rc;
}

}  // extern "C"
