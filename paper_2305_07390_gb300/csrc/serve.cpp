// serve.cpp -- continuous-batching serving loop (ebisu_serve_*).
//
// A host scheduler thread owns a few CUDA streams ("lanes").  Requests are
// queued at submit time; on every tick the scheduler
//   1. retires finished launches (event query), frees their device memory and
//      returns their bytes to the HBM budget;
//   2. admits queued requests while the budget allows and a lane is free (a
//      request that can never fit is refused at submit), in arrival order or
//      -- ebisu_serve_set_policy -- least estimated work first, where a
//      request's priority is its estimated run time minus the time it has
//      waited (so a large request is not passed over forever);
//   3. groups the newly admitted requests by kernel type and starts each group
//      as ONE batched persistent launch (ebisu_batch_*) on a free lane: the
//      request's grid is copied into server memory (kept resident until the
//      request finishes), stepped there, and the result written to the
//      caller's output buffer.
// Requests that arrive while others run are admitted as memory and lanes free
// up, and their launches overlap on the device with those already running.
// Latency is measured from submit to the moment the scheduler sees the
// launch's completion event.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan.h"

using namespace ebisu;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    ebisu_plan_s plan;
    const void* in = nullptr;
    void* out = nullptr;
    int64_t steps = 0;
    size_t need = 0;
    double est_s = 0;  // estimated run time alone on the GPU
    double t_submit = 0, t_done = 0;
    int state = 0;  // 0 queued, 1 running, 2 done, 3 cancelled, 4 failed
    int status = EBISU_OK;
};

struct Launch {
    std::vector<Request*> reqs;
    double t_start = 0, est_s = 0;  // when it was enqueued; its requests' estimated work
    int lane = -1;
    void* mem = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
    ebisu_batch_t batch = nullptr;
    void* ws = nullptr;
};

constexpr size_t kDefaultMaxQueue = 1024;

// Estimated run time of a request alone on the GPU: cell updates over half
// the roofline of its stencil and storage type at its temporal depth (the
// lower of HBM bandwidth over 2S/t bytes per update and the FMA rate over 2P
// flops).  Only used to order requests and to predict queue waits.
double estimate_s(const ebisu_plan_s* p, int64_t steps)
{
    const DeviceInfo& dv = device_rates();
    const double t = std::max(1, p->prm.variant == 1 ? 1 : p->prm.depth);
    const double hbm = 6.7e12 / (2.0 * (double)p->esize / t);
    const double fp = (p->dtype == EBISU_F64 ? dv.f64 : dv.f32) / (2.0 * p->npts);
    const double rate = 0.5 * std::min(hbm, fp);
    const double cells = (double)p->n[0] * p->n[1] * p->n[2];
    return cells * (double)steps / rate;
}

}  // namespace

struct ebisu_server_s {
    size_t budget = 0;
    int max_slots = 1;
    size_t max_queue = kDefaultMaxQueue;
    int order = EBISU_SERVE_FIFO;
    double max_wait_s = 0;  // admission control: refuse when the predicted wait exceeds it (0 = off)
    double queued_est = 0;  // estimated work of the queued requests (s)
    // measured over estimated run time of finished launches (running mean),
    // applied to the queued work when predicting a new request's wait
    double est_scale = 1.0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> reqs;
    std::vector<cudaStream_t> lanes;
    std::vector<int> lane_busy;
    std::vector<Launch*> running;
    size_t held = 0, peak = 0;
    int64_t submitted = 0, completed = 0, rejected = 0, nrunning = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread th;

    // Device bytes a request holds while admitted: its resident copy plus
    // its share of a batch workspace (ping-pong buffer, control, tables).
    static size_t need_of(ebisu_plan_t p, int64_t steps)
    {
        const size_t g = align_up((size_t)p->elems * p->esize, kAlign);
        size_t ws = 0;
        if (ebisu_batch_workspace_bytes(1, &p, &steps, &ws) != EBISU_OK) ws = g + 64 * 1024;
        return g + ws;
    }

    void retire_locked()
    {
        for (size_t i = 0; i < running.size();) {
            Launch* L = running[i];
            const cudaError_t q = cudaEventQuery(L->ev);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            int st = EBISU_OK;
            if (q != cudaSuccess) {
                set_cuda_error(q);
                st = EBISU_ERR_CUDA;
            } else if (L->batch) {
                st = ebisu_batch_sync(L->batch, lanes[L->lane]);
            }
            const double t = now_s();
            if (st == EBISU_OK && L->est_s > 1e-4) {
                const double ratio = std::min(10.0, std::max(0.1, (t - L->t_start) / L->est_s));
                est_scale = 0.8 * est_scale + 0.2 * ratio;
            }
            for (Request* r : L->reqs) {
                r->t_done = t;
                r->status = st;
                r->state = (st == EBISU_OK) ? 2 : 4;
                held -= r->need;
                ++completed;
                --nrunning;
            }
            if (L->batch) ebisu_batch_destroy(L->batch);
            cudaFreeAsync(L->mem, lanes[L->lane]);
            cudaEventDestroy(L->ev);
            lane_busy[L->lane] = 0;
            delete L;
            running.erase(running.begin() + i);
            cv_done.notify_all();
        }
    }

    // Start one group (same kernel type) on a free lane.  Called unlocked.
    int start_group(std::vector<Request*>& grp, int lane)
    {
        cudaStream_t st = lanes[lane];
        Launch* L = new Launch();
        L->reqs = grp;
        L->lane = lane;
        L->t_start = now_s();
        for (Request* r : grp) L->est_s += r->est_s;
        const int n = (int)grp.size();
        std::vector<ebisu_plan_t> plans(n);
        std::vector<int64_t> steps(n);
        for (int i = 0; i < n; ++i) {
            plans[i] = &grp[i]->plan;
            steps[i] = grp[i]->steps;
        }
        size_t wsb = 0;
        int rc = ebisu_batch_workspace_bytes(n, plans.data(), steps.data(), &wsb);
        size_t grids = 0;
        std::vector<size_t> goff(n);
        for (int i = 0; i < n; ++i) {
            goff[i] = grids;
            grids += align_up((size_t)grp[i]->plan.elems * grp[i]->plan.esize, kAlign);
        }
        cudaError_t e = cudaSuccess;
        if (rc == EBISU_OK) {
            L->bytes = grids + wsb;
            e = cudaMallocAsync(&L->mem, L->bytes, st);
            if (e != cudaSuccess) rc = fail_cuda(e);
        }
        std::vector<const void*> ins(n);
        std::vector<void*> outs(n);
        if (rc == EBISU_OK) {
            for (int i = 0; i < n && e == cudaSuccess; ++i) {
                void* res = (char*)L->mem + goff[i];
                e = cudaMemcpyAsync(res, grp[i]->in, (size_t)grp[i]->plan.elems * grp[i]->plan.esize,
                                    cudaMemcpyDeviceToDevice, st);
                ins[i] = res;
                outs[i] = grp[i]->out;
            }
            if (e != cudaSuccess) rc = fail_cuda(e);
        }
        if (rc == EBISU_OK) {
            L->ws = (char*)L->mem + grids;
            rc = ebisu_batch_create(n, plans.data(), ins.data(), outs.data(), steps.data(), L->ws, st, &L->batch);
        }
        if (rc == EBISU_OK) rc = ebisu_batch_launch(L->batch, st);
        if (rc == EBISU_OK) {
            e = cudaEventCreateWithFlags(&L->ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(L->ev, st);
            if (e != cudaSuccess) rc = fail_cuda(e);
        }
        std::lock_guard<std::mutex> lk(mu);
        if (rc != EBISU_OK) {
            for (Request* r : grp) {
                r->state = 4;
                r->status = rc;
                r->t_done = now_s();
                held -= r->need;
                ++completed;
                --nrunning;
            }
            if (L->batch) ebisu_batch_destroy(L->batch);
            if (L->mem) cudaFreeAsync(L->mem, st);
            if (L->ev) cudaEventDestroy(L->ev);
            lane_busy[lane] = 0;
            delete L;
            cv_done.notify_all();
            return rc;
        }
        running.push_back(L);
        return EBISU_OK;
    }

    void loop()
    {
        cudaSetDevice(device);
        for (;;) {
            std::vector<std::pair<std::vector<Request*>, int>> todo;
            {
                std::unique_lock<std::mutex> lk(mu);
                retire_locked();
                if (stop && queue.empty() && running.empty()) break;
                // admission in arrival order: budget and free lanes
                std::vector<Request*> admitted;
                int free_lanes = 0;
                for (int b : lane_busy) free_lanes += (b == 0);
                const double tnow = now_s();
                while (!queue.empty() && free_lanes > 0) {
                    // the next request: the queue's head, or the one with the
                    // least estimated run time net of its wait so far
                    auto pick = queue.begin();
                    if (order == EBISU_SERVE_SHORTEST) {
                        double best = 1e300;
                        for (auto q = queue.begin(); q != queue.end(); ++q) {
                            if ((*q)->state == 3) {  // cancelled: remove it first
                                pick = q;
                                break;
                            }
                            const double key = (*q)->est_s - (tnow - (*q)->t_submit);
                            if (key < best) {
                                best = key;
                                pick = q;
                            }
                        }
                    }
                    Request* r = *pick;
                    if (r->state == 3) {  // cancelled while queued
                        queued_est -= r->est_s;
                        queue.erase(pick);
                        continue;
                    }
                    if (held + r->need > budget) break;
                    queue.erase(pick);
                    queued_est -= r->est_s;
                    r->state = 1;
                    held += r->need;
                    peak = std::max(peak, held);
                    ++nrunning;
                    admitted.push_back(r);
                    // one lane per kernel type in this tick
                    bool new_kind = true;
                    for (Request* o : admitted)
                        if (o != r && o->plan.ndim == r->plan.ndim && o->plan.shape == r->plan.shape &&
                            o->plan.radius == r->plan.radius && o->plan.dtype == r->plan.dtype)
                            new_kind = false;
                    if (new_kind) --free_lanes;
                }
                // group by kernel type, give each group a free lane
                std::map<std::tuple<int, int, int, int>, std::vector<Request*>> groups;
                for (Request* r : admitted)
                    groups[{r->plan.ndim, r->plan.shape, r->plan.radius, r->plan.dtype}].push_back(r);
                for (auto& kv : groups) {
                    int lane = -1;
                    for (size_t i = 0; i < lane_busy.size(); ++i)
                        if (!lane_busy[i]) {
                            lane = (int)i;
                            break;
                        }
                    if (lane < 0) {  // no lane: back to the head of the queue
                        for (auto it = kv.second.rbegin(); it != kv.second.rend(); ++it) {
                            (*it)->state = 0;
                            held -= (*it)->need;
                            --nrunning;
                            queued_est += (*it)->est_s;
                            queue.push_front(*it);
                        }
                        continue;
                    }
                    lane_busy[lane] = 1;
                    todo.push_back({kv.second, lane});
                }
                if (todo.empty()) {
                    if (running.empty() && queue.empty() && !stop)
                        cv_sched.wait(lk);
                    else
                        cv_sched.wait_for(lk, std::chrono::microseconds(50));
                    continue;
                }
            }
            for (auto& t : todo) start_group(t.first, t.second);
        }
    }
};

extern "C" {

int ebisu_serve_create(size_t hbm_budget, int max_slots, ebisu_server_t* out)
{
    if (!out || hbm_budget == 0 || max_slots < 0 || max_slots > 64) return EBISU_ERR_INVALID_ARG;
    *out = nullptr;
    // 0: lanes scale with the budget, one per 4 GiB, 4 to 32
    if (max_slots == 0) max_slots = (int)std::min<size_t>(32, std::max<size_t>(4, hbm_budget >> 32));
    ebisu_server_s* s = new (std::nothrow) ebisu_server_s();
    if (!s) return EBISU_ERR_OOM;
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    cudaError_t e = cudaGetDevice(&s->device);
    for (int i = 0; i < max_slots && e == cudaSuccess; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->lanes.push_back(st);
    }
    if (e != cudaSuccess) {
        for (auto st : s->lanes) cudaStreamDestroy(st);
        delete s;
        return fail_cuda(e);
    }
    s->lane_busy.assign(max_slots, 0);
    s->th = std::thread([s] { s->loop(); });
    *out = s;
    return EBISU_OK;
}

int ebisu_serve_submit(ebisu_server_t s, ebisu_plan_t plan, const void* in_dev, void* out_dev, int64_t steps,
                       uint64_t* ticket)
{
    if (!s || !plan || !in_dev || !out_dev || !ticket || steps < 0) return EBISU_ERR_INVALID_ARG;
    if (plan->field) return EBISU_ERR_UNSUPPORTED;  // the server runs batches, which take fixed weights
    Request* r = new (std::nothrow) Request();
    if (!r) return EBISU_ERR_OOM;
    r->plan = *plan;
    r->in = in_dev;
    r->out = out_dev;
    r->steps = steps;
    r->need = ebisu_server_s::need_of(plan, steps);
    r->est_s = estimate_s(plan, steps);
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    ++s->submitted;
    if (r->need > s->budget) {
        ++s->rejected;
        delete r;
        return EBISU_ERR_BUDGET;
    }
    // admission control: the queue's length limit, and (if set) the predicted
    // wait -- the estimated work already queued -- against the wait limit
    const bool late = s->max_wait_s > 0 && s->queued_est * s->est_scale > s->max_wait_s;
    if (s->queue.size() >= s->max_queue || s->stop || late) {
        ++s->rejected;
        delete r;
        return EBISU_ERR_BUSY;
    }
    s->queued_est += r->est_s;
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *ticket = r->id;
    s->cv_sched.notify_all();
    return EBISU_OK;
}

int ebisu_serve_poll(ebisu_server_t s, uint64_t ticket, int* done, double* latency_s)
{
    if (!s || !done) return EBISU_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return EBISU_ERR_INVALID_ARG;
    Request* r = it->second;
    *done = (r->state >= 2) ? 1 : 0;
    if (latency_s) *latency_s = (r->state >= 2 ? r->t_done : now_s()) - r->t_submit;
    return (r->state == 4) ? r->status : EBISU_OK;
}

int ebisu_serve_wait(ebisu_server_t s, uint64_t ticket, double timeout_s, double* latency_s)
{
    if (!s) return EBISU_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return EBISU_ERR_INVALID_ARG;
    Request* r = it->second;
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (r->state < 2) {
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && r->state < 2) return EBISU_ERR_NOT_READY;
    }
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    return (r->state == 4) ? r->status : EBISU_OK;
}

int ebisu_serve_stats(ebisu_server_t s, int64_t* stats)
{
    if (!s || !stats) return EBISU_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    stats[0] = s->submitted;
    stats[1] = s->completed;
    stats[2] = s->rejected;
    stats[3] = (int64_t)s->queue.size();
    stats[4] = s->nrunning;
    stats[5] = (int64_t)s->peak;
    stats[6] = (int64_t)s->held;
    return EBISU_OK;
}

int ebisu_serve_set_max_queue(ebisu_server_t s, int max_queue)
{
    if (!s || max_queue < 1) return EBISU_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->max_queue = (size_t)max_queue;
    return EBISU_OK;
}

int ebisu_serve_set_policy(ebisu_server_t s, int order, double max_wait_s)
{
    if (!s || (order != EBISU_SERVE_FIFO && order != EBISU_SERVE_SHORTEST) || !(max_wait_s >= 0))
        return EBISU_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->order = order;
    s->max_wait_s = max_wait_s;
    s->cv_sched.notify_all();
    return EBISU_OK;
}

int ebisu_serve_cancel(ebisu_server_t s, uint64_t ticket)
{
    if (!s) return EBISU_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return EBISU_ERR_INVALID_ARG;
    Request* r = it->second;
    if (r->state != 0) return EBISU_ERR_NOT_READY;
    r->state = 3;
    s->queued_est -= r->est_s;  // it no longer delays later requests
    r->est_s = 0;
    r->t_done = now_s();
    s->cv_done.notify_all();
    return EBISU_OK;
}

int ebisu_serve_destroy(ebisu_server_t s)
{
    if (!s) return EBISU_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_sched.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    for (auto st : s->lanes) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return EBISU_OK;
}

}  // extern "C"
