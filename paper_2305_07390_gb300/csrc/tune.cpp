// tune.cpp -- the cost model of Section 5 and the autotuner of Section 6.
//
// Practical attainable performance (Section 5, Eq. 1-12):
//   T_gm  = a_gm  * D_gm * S / B_gm          (global memory, per temporal block)
//   T_sm  = a_sm  * D_sm * t * S / B_sm      (shared memory)
//   T_cmp = a_cmp * D_cmp * t / THR_cmp      (FP pipe)
//   P     = D * t / max(T_gm, T_sm, T_cmp)
//   PP    = P * V,  V = V_SMtile (useful / computed cells of the overlapped
//           trapezoid) * V_sync (Eq. 11 with one wait per temporal block,
//           Section 4.3.2) * V_wave (tiles / (waves * resident CTAs)).
// D_gm counts every cell a tile loads (its input region, halo included) and
// stores; D_sm counts every computed cell with a_sm = P reads + 1 write (the
// kernel keeps every neighbour in the shared-memory ring); a_cmp = 2P flops.
//
// The tuner ranks candidate (tile, depth) pairs by PP ("deeper or wider",
// Section 6.4) and, on request, times the best few and keeps the fastest
// (Section 6.4.1's fine-tuning of depth).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "plan.h"

namespace ebisu {

static std::mutex g_rate_mu;
static bool g_rates_done[16] = {false};
static DeviceInfo g_rates[16];

const DeviceInfo& device_rates()
{
    const DeviceInfo& base = device_info();
    std::lock_guard<std::mutex> lk(g_rate_mu);
    const int dev = base.device < 0 ? 0 : base.device;
    DeviceInfo& r = g_rates[dev];
    if (!g_rates_done[dev]) {
        r = base;
        // GB300 figures measured with ebisu_probe_device (FMA rates at the
        // 2070 MHz boost clock, 16-byte shared loads, one wait round trip)
        // serve until a probe in this process replaces them
        // (ebisu_probe_device records its results here; EBISU_PROBE=1 runs
        // it on first use).
        r.f64 = 1.255e12;
        r.f32 = 74.7e12;
        r.lds = 38.0e12;
        r.barrier_s = 2.5e-6;
        const char* e = getenv("EBISU_PROBE");
        if (e && e[0] == '1') {
            double out[6];
            if (probe_device(out) == cudaSuccess) {
                r.f64 = out[0];
                r.f32 = out[1];
                r.lds = out[2];
                r.barrier_s = out[3];
            } else {
                cudaGetLastError();
            }
        }
        g_rates_done[dev] = true;
    }
    return r;
}

void record_device_rates(const double* out)
{
    const DeviceInfo& base = device_info();
    device_rates();  // initialise the entry first
    std::lock_guard<std::mutex> lk(g_rate_mu);
    DeviceInfo& r = g_rates[base.device < 0 ? 0 : base.device];
    if (out[0] > 0) r.f64 = out[0];
    if (out[1] > 0) r.f32 = out[1];
    if (out[2] > 0) r.lds = out[2];
    if (out[3] > 0) r.barrier_s = out[3];
}

static double hbm_bytes_per_s()
{
    const char* e = getenv("EBISU_HBM_GBS");
    if (e && *e) return atof(e) * 1e9;
    return 6704.5e9;  // measured copy bandwidth of the GB300s this was built on
}

// Sum over the levels of a trapezoid: cells computed at level s, s = 1..t.
static double trapezoid_cells(const ebisu_plan_s* p, const GridDesc& g, int t, double* useful, double* loaded)
{
    const int r = p->radius;
    const bool per = p->boundary == EBISU_PERIODIC;
    double comp = 0, use = 0, load = 0;
    // sum over all tiles (rows of tiles are identical up to clipping: use the
    // average tile by summing per axis)
    auto axis_sum = [&](int ax, int rr, int s, bool for_load) {
        // total extent of level-s regions over all tiles along axis `ax`
        double tot = 0;
        const int64_t n = g.n[ax];
        const int64_t padax = (ax == 1) ? (p->ndim == 3 ? p->pad : 0) : p->pad;
        for (int i = 0; i < g.nt[ax]; ++i) {
            const int64_t a = (int64_t)i * g.tile[ax];
            const int64_t b = std::min<int64_t>(a + g.tile[ax], n);
            int64_t lo = a - (int64_t)rr * (t - s), hi = b + (int64_t)rr * (t - s);
            if (!per) {
                lo = std::max<int64_t>(lo, for_load ? -padax : 0);
                hi = std::min<int64_t>(hi, for_load ? n + padax : n);
            }
            tot += (double)(hi - lo);
        }
        return tot;
    };
    const int rp1 = (p->ndim == 3) ? r : 0;
    for (int s = 1; s <= t; ++s)
        comp += axis_sum(0, r, s, false) * axis_sum(1, rp1, s, false) * axis_sum(2, r, s, false);
    use = (double)g.n[0] * g.n[1] * g.n[2] * t;
    load = axis_sum(0, r, 0, true) * axis_sum(1, rp1, 0, true) * axis_sum(2, r, 0, true);
    *useful = use;
    *loaded = load;
    return comp;
}

double model_pp(const ebisu_plan_s* p, const ebisu_params& q, int64_t steps, int* bound, double* valid)
{
    const DeviceInfo& dv = device_rates();
    GridDesc g;
    const int t = (int)std::max<int64_t>(1, std::min<int64_t>(q.depth, std::max<int64_t>(steps, 1)));
    ebisu_plan_s tmp = *p;
    tmp.prm = q;
    tmp.prm.depth = t;
    fill_grid_desc(&tmp, nullptr, nullptr, nullptr, std::max<int64_t>(steps, 1), false, &g);
    double useful = 0, loaded = 0;
    double computed = trapezoid_cells(p, g, t, &useful, &loaded);
    const double vsm = useful / computed;
    // Partial passes.  The barrier after every streamed plane makes each
    // level cost as much as its busiest thread: for 2-byte and 4-byte storage
    // (four cells per thread) a level of width w costs ceil(quads / threads)
    // full passes; for FP64 (one cell per slot) about half a warp of the last
    // slot is empty.
    if (p->esize <= 4 && p->ndim == 2) {
        double eff_cells = 0, real_cells = 0;
        for (int s = 1; s <= t; ++s) {
            const double w = (double)g.tile[2] + 2.0 * p->radius * (t - s);
            const double quads = std::ceil((w + 3.0) / 4.0);
            eff_cells += std::ceil(quads / kThreads) * 4.0 * kThreads;
            real_cells += w;
        }
        computed *= eff_cells / real_cells;
    } else {
        const double region = (double)g.tile[1] * g.tile[2];
        computed *= 1.0 + 16.0 / std::max(region, 32.0);
    }
    const double S = (double)p->esize;
    const double cells = (double)g.n[0] * g.n[1] * g.n[2];
    const double thr = (p->dtype == EBISU_F64) ? dv.f64 : dv.f32;
    const double Tgm = (loaded + cells) * S / hbm_bytes_per_s();
    const double Tsm = computed * (p->npts + 1) * S / dv.lds;
    const double Tcmp = computed * 2.0 * p->npts / thr;
    double T = std::max(Tgm, std::max(Tsm, Tcmp));
    int b = 0;
    if (T == Tsm) b = 1;
    if (T == Tcmp) b = 2;
    // Resident CTAs per SM: shared memory and the build's register cap.
    const size_t smem = tb_smem_bytes(p, tmp.prm) + 4096;
    const int variant = kernel_variant(p->dtype, q.ctas_per_sm);
    const int reg_cap = (variant == 1) ? 4 : 2;
    const int fit = (int)std::max<size_t>(1, dv.smem_per_sm / std::max<size_t>(smem, 1));
    const int res = std::max(1, std::min(std::min(q.ctas_per_sm, fit), reg_cap));
    // The one barrier per streamed plane idles the FP pipe unless other
    // warps are resident; measured on this part: 8 warps/SM keep it ~60%
    // busy, 16 ~85%, 32 ~95% (2D FP64 sweeps).
    const double warps = 8.0 * res;
    const double eff = 1.0 - 0.4 * std::exp(-(warps - 8.0) / 8.0);
    T /= eff;
    // wave quantisation of one temporal block over the resident CTAs
    const double ctas = (double)dv.sms * res;
    const double waves = std::ceil((double)g.ntiles / ctas);
    const double vwave = (double)g.ntiles / (waves * ctas);
    // one temporal block (stretched by the wave quantisation) plus one
    // dependency wait between blocks: Eq. 11 with n = 1 (lazy streaming)
    const double Tblock = T / vwave;
    const double vsync = Tblock / (Tblock + dv.barrier_s);
    if (bound) *bound = b;
    if (valid) *valid = vsm;
    const double P = useful / T;  // cell updates per second at the bound
    return P * vwave * vsync;
}

static void push_unique(std::vector<int>& v, int x)
{
    if (x >= 1 && std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
}

int rank_candidates(const ebisu_plan_s* p, int64_t steps, ebisu_params* out, double* pred, int cap, double share)
{
    const DeviceInfo& dv = device_info();
    std::vector<std::pair<double, ebisu_params>> cand;
    std::vector<int> depths = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
    std::vector<int> txs, tys;
    if (p->ndim == 2) {
        for (int x : {512, 1024, 1536, 2048, 3072, 4000}) push_unique(txs, (int)std::min<int64_t>(x, p->n[2]));
        tys.push_back(1);
    } else {
        for (int x : {32, 64, 128}) push_unique(txs, (int)std::min<int64_t>(x, p->n[2]));
        for (int y : {8, 16, 32, 64}) push_unique(tys, (int)std::min<int64_t>(y, p->n[1]));
    }
    for (int d : depths) {
        if (d > std::max<int64_t>(steps, 1) && d != 1) continue;
        std::vector<int> txd = txs;
        if (p->ndim == 2 && p->esize <= 4) {
            // widths whose widest level (w + r(2d-1) + alignment) fills whole
            // passes of four cells per thread
            for (int k : {1, 2, 3}) {
                const int w = (4 * kThreads * k - p->radius * (2 * d - 1) - 4) & ~3;
                if (w >= 64) push_unique(txd, (int)std::min<int64_t>(w, p->n[2]));
            }
        }
        for (int tx : txd)
            for (int ty : tys)
                for (int cps : {1, 2, 4}) {
                    if (cps == 4 && p->dtype != EBISU_F64) continue;
                    ebisu_params q;
                    memset(&q, 0, sizeof(q));
                    q.tile_x = tx;
                    q.tile_y = ty;
                    q.depth = d;
                    q.ctas_per_sm = cps;
                    q.threads = kThreads;
                    if (check_params(p, q) != EBISU_OK) continue;
                    if (cps > 1 && (tb_smem_bytes(p, q) + 4096) * cps > dv.smem_per_sm) continue;
                    (void)0;
                    // band length along the streamed axis: enough tiles for
                    // one or two waves of resident CTAs
                    const int64_t nt2 = (p->n[2] + tx - 1) / tx;
                    const int64_t nt1 = (p->ndim == 3) ? (p->n[1] + ty - 1) / ty : 1;
                    const int64_t ctas = std::max<int64_t>(1, (int64_t)((double)dv.sms * cps * share));
                    for (int waves : {1, 2, 4}) {
                        int64_t nts = std::max<int64_t>(1, (ctas * waves + nt2 * nt1 - 1) / (nt2 * nt1));
                        nts = std::min<int64_t>(nts, p->n[0]);
                        // grids smaller than a wave: fewer, taller tiles (a
                        // band shorter than 2rt rows is all overlap)
                        const int64_t smin = std::max(4, 2 * p->radius * d);
                        if ((p->n[0] + nts - 1) / nts < smin) nts = std::max<int64_t>(1, p->n[0] / smin);
                        q.tile_s = (int)((p->n[0] + nts - 1) / nts);
                        bool dup = false;  // several wave counts can give the same band
                        for (const auto& c : cand)
                            dup = dup || (c.second.tile_x == q.tile_x && c.second.tile_y == q.tile_y &&
                                          c.second.tile_s == q.tile_s && c.second.depth == q.depth &&
                                          c.second.ctas_per_sm == q.ctas_per_sm);
                        if (dup) continue;
                        const double pp = model_pp(p, q, steps, nullptr, nullptr);
                        cand.push_back({pp, q});
                    }
                }
    }
    std::stable_sort(cand.begin(), cand.end(),
                     [](const auto& a, const auto& b) { return a.first > b.first; });
    int n = 0;
    for (auto& c : cand) {
        if (n >= cap) break;
        out[n] = c.second;
        if (pred) pred[n] = c.first;
        ++n;
    }
    return n;
}

}  // namespace ebisu

using namespace ebisu;

extern "C" {

int ebisu_cost_model(const ebisu_model_in* in, ebisu_model_out* out)
{
    if (!in || !out) return EBISU_ERR_INVALID_ARG;
    if (in->b_gm <= 0 || in->b_sm <= 0 || in->thr_cmp <= 0 || in->t <= 0 || (in->ndim != 2 && in->ndim != 3))
        return EBISU_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->t_gm = in->a_gm * in->d_gm * in->s_cell / in->b_gm;
    out->t_sm = in->a_sm * in->d_sm * in->t * in->s_cell / in->b_sm;
    out->t_cmp = in->a_cmp * in->d_cmp * in->t / in->thr_cmp;
    out->t_stencil = std::max(out->t_gm, std::max(out->t_sm, out->t_cmp));
    out->bound = (out->t_stencil == out->t_cmp) ? 2 : (out->t_stencil == out->t_sm ? 1 : 0);
    out->p = out->t_stencil > 0 ? in->d_cmp * in->t / out->t_stencil : 0.0;
    double v = 1.0;
    if (in->tile_x > 0) {
        v = std::max(0.0, (in->tile_x - 2.0 * in->rad * (in->t - 1.0)) / in->tile_x);
        if (in->ndim == 3 && in->tile_y > 0)
            v *= std::max(0.0, (in->tile_y - 2.0 * in->rad * (in->t - 1.0)) / in->tile_y);
    }
    out->v_smtile = v;
    out->v_dtile = out->t_stencil / (out->t_stencil + in->t_dsync * in->n_sync);
    out->pp = out->p * (in->tiling == 1 ? out->v_dtile : out->v_smtile);
    if (in->a_sm > 0 && in->d_sm > 0)
        out->depth_sm = in->a_gm * in->d_gm * in->b_sm / (in->a_sm * in->d_sm * in->b_gm);
    const double txy = in->tile_x * (in->tile_y > 0 ? in->tile_y : 1.0);
    const double lhs = in->a_sm * txy / in->b_sm - in->a_gm * (in->tile_x + in->tile_y) * 2.0 * in->rad / in->b_gm;
    out->depth_device = lhs > 0 ? (in->a_gm * txy / in->b_gm) / lhs : INFINITY;
    if (in->a_sm > 0) out->min_device_tile = 4.0 * in->a_gm * in->b_sm / (in->a_sm * in->b_gm) * in->rad;
    return EBISU_OK;
}

int ebisu_plan_model(ebisu_plan_t plan, double* pred, int* bound, double* valid)
{
    if (!plan) return EBISU_ERR_INVALID_ARG;
    const double pp = model_pp(plan, plan->prm, 1000, bound, valid);
    if (pred) *pred = pp;
    return EBISU_OK;
}

int ebisu_plan_tune(ebisu_plan_t plan, const void* in, void* out, int64_t steps, void* workspace,
                    int max_candidates, double* best_ms, void* stream)
{
    return ebisu_plan_tune_share(plan, in, out, steps, workspace, max_candidates, 1.0, best_ms, stream);
}

int ebisu_plan_tune_share(ebisu_plan_t plan, const void* in, void* out, int64_t steps, void* workspace,
                          int max_candidates, double share, double* best_ms, void* stream)
{
    if (!plan || !in || !out || !workspace || steps < 1 || max_candidates < 1) return EBISU_ERR_INVALID_ARG;
    if (!(share > 0.0 && share <= 1.0)) return EBISU_ERR_INVALID_ARG;
    if (plan->field) return EBISU_ERR_UNSUPPORTED;  // one kernel only: nothing to choose
    if (in == out) return EBISU_ERR_INVALID_ARG;
    std::vector<ebisu_params> cand(max_candidates);
    std::vector<double> pred(max_candidates);
    const bool sr = plan_sr(plan);
    int n = sr ? 0 : rank_candidates(plan, steps, cand.data(), pred.data(), max_candidates, share);
    if (n < 1 && !sr) return EBISU_ERR_UNSUPPORTED;
    cand.resize(n);  // the ranking may return fewer than max_candidates
    // (stochastic rounding: no shared-memory build; the one-step kernel keeps
    // the plan's current fused parameters)
    ebisu_params naive = sr ? plan->prm : cand[0];
    naive.variant = 1;
    // The one-step-per-launch kernel is timed too: where the fused kernel
    // cannot beat it (measured: 3D low-order FP64 stars), the plan runs it.
    cand.push_back(naive);
    ++n;
    // The 3D register-streaming build (FP64 depth 1, FP32/BF16 depths 2-3): z segments sized so
    // that one step has about 1, 2 or 4 tiles per resident warp.
    if (plan->ndim == 3 && rs3_built((int)plan->esize, plan->shape, plan->radius)) {
        const DeviceInfo& dv = device_info();
        const int es = (int)plan->esize;
        for (int which = 0; which < 2; ++which) {
        const int D = rs3_depth(es, plan->shape, plan->radius, which);
        if (which == 1 && D == rs3_depth(es, plan->shape, plan->radius, 0)) break;
        int occ = 0;
        if (rs3_occupancy(plan, D, &occ) != cudaSuccess || occ < 1) {
            cudaGetLastError();
        } else {
            const int64_t warps = std::max<int64_t>(1, (int64_t)((double)occ * dv.sms * kRSWarps * share));
            const int64_t S = rs3_strip(es, D, plan->radius), TY = rs3_rows(es);
            const int64_t xy = ((plan->n[2] + S - 1) / S) * ((plan->n[1] + TY - 1) / TY);
            int64_t lastH = -1;
            for (int k : {1, 2, 3, 4, 6}) {
                const int64_t ng = std::max<int64_t>(1, (k * warps + xy - 1) / xy);
                const int64_t H = (plan->n[0] + ng - 1) / ng;
                if (H == lastH) continue;
                lastH = H;
                ebisu_params q{};
                q.variant = 2;
                q.depth = D;
                q.tile_s = (int32_t)H;
                q.ctas_per_sm = occ;
                q.threads = kRSThreads;
                RSLayout L;
                if (rs_layout(plan, q, &L) != EBISU_OK) continue;
                q.tile_x = L.S;
                q.tile_y = L.TY;
                cand.push_back(q);
                ++n;
            }
        }
        }
    }
    // The register-streaming build (2D): both built depths, segments sized so
    // that one temporal block has about 1, 2 or 4 tiles per resident warp.
    if (plan->ndim == 2) {
        const DeviceInfo& dv = device_info();
        for (int which = 0; which < 2; ++which) {
            const int D = rs_depth((int)plan->esize, plan->shape, plan->radius, which);
            if (which == 1 && D == rs_depth((int)plan->esize, plan->shape, plan->radius, 0)) break;
            int occ = 0;
            if (rs_occupancy(plan, D, false, &occ) != cudaSuccess || occ < 1) {
                cudaGetLastError();
                continue;
            }
            const int64_t warps = std::max<int64_t>(1, (int64_t)((double)occ * dv.sms * kRSWarps * share));
            const int64_t S = kRSCols - 2LL * D * plan->radius;
            const int64_t ns = (plan->n[2] + S - 1) / S;
            int64_t lastH = -1;
            for (int k : {1, 2, 3, 4, 6}) {
                const int64_t ng = std::max<int64_t>(1, (k * warps + ns - 1) / ns);
                const int64_t H = (plan->n[0] + ng - 1) / ng;
                if (H == lastH) continue;
                lastH = H;
                ebisu_params q{};
                q.variant = 2;
                q.depth = D;
                q.tile_s = (int32_t)H;
                q.ctas_per_sm = occ;
                q.threads = kRSThreads;
                RSLayout L;
                if (rs_layout(plan, q, &L) != EBISU_OK) continue;
                q.tile_x = L.S;
                q.tile_y = 1;
                cand.push_back(q);
                ++n;
            }
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail_cuda(cudaGetLastError());
    const ebisu_params saved = plan->prm;
    const ebisu_params saved_tb = plan->tb_prm;
    double best = 1e300;
    ebisu_params bestp = saved;
    ebisu_params best_blocked = cand[0];  // shared-memory build (variant 0)
    double best_blocked_ms = 1e300;
    ebisu_params best_fused = cand[0];    // variant 0 or 2
    double best_fused_ms = 1e300;
    int rc = EBISU_OK;
    for (int i = 0; i < n; ++i) {
        plan->prm = cand[i];
        rc = ebisu_run(plan, in, out, steps, workspace, stream);  // warm-up
        if (rc != EBISU_OK) break;
        cudaEventRecord(e0, st);
        rc = ebisu_run(plan, in, out, steps, workspace, stream);
        if (rc != EBISU_OK) break;
        cudaEventRecord(e1, st);
        rc = ebisu_sync(workspace, stream);
        if (rc != EBISU_OK) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bestp = cand[i];
        }
        if (cand[i].variant == 0 && ms < best_blocked_ms) {
            best_blocked_ms = ms;
            best_blocked = cand[i];
        }
        if (cand[i].variant != 1 && ms < best_fused_ms) {
            best_fused_ms = ms;
            best_fused = cand[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == EBISU_OK && sr) {
        // no shared-memory build to keep; the fused build, if any, is the
        // register-streaming one
        if (best_fused_ms < 1e300) {
            plan->prm = best_fused;
            plan->prm.fused_variant = 2;
            if (bestp.variant == 1) plan->prm.variant = 1;
        } else {
            plan->prm = naive;
        }
    } else if (rc == EBISU_OK) {
        // keep the best shared-memory-kernel parameters (batches and the
        // server use them) and the best temporally blocked build's
        // parameters; `variant` says which kernel won (1: the one-step
        // kernel, whose runs ignore the other fields)
        plan->tb_prm = best_blocked;
        plan->tb_prm.fused_variant = 0;
        plan->prm = best_fused;
        plan->prm.fused_variant = best_fused.variant;
        if (bestp.variant == 1) plan->prm.variant = 1;
    } else {
        plan->prm = saved;
        plan->tb_prm = saved_tb;
    }
    if (best_ms) *best_ms = best;
    return rc;
}

}  // extern "C"
