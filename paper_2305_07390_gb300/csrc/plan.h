// plan.h -- host-side plan object and helpers shared by the C-ABI files.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/ebisu.h"
#include "common.h"
#include "dispatch.h"

struct ebisu_plan_s {
    int ndim = 0, shape = 0, radius = 0, dtype = 0, boundary = 0;
    int64_t dims[3] = {0, 0, 0};  // interior extents, slowest first (as given)
    int npts = 0;
    double coef[ebisu::kMaxPoints] = {};
    ebisu_params prm{};
    ebisu_params tb_prm{};  // shared-memory kernel parameters (batches and the server use them)
    // streaming coordinates (s, p1, p2); p1 is a dummy axis in 2D
    int64_t n[3] = {1, 1, 1};
    int64_t ext[3] = {1, 1, 1};  // stored extents
    int64_t lds = 0, ld1 = 0;
    int pad = 0, pad1 = 0;
    size_t esize = 8;
    int64_t elems = 0;
    // storage rounding (EBISU_ROUND_*): stochastic for BF16 storage only;
    // sr_key = sr_plan_key(sr_seed), the kernels' plan key
    int rounding = 0;
    uint64_t sr_seed = 0;
    uint32_t sr_key = 0;
    int ablate = 0;  // shared-memory build with elements switched off (EBISU_ABLATE_* mask)
    const void* field = nullptr;  // per-cell weights (device; P arrays like the grid), or null
};

namespace ebisu {

constexpr int kThreads = 256;      // threads per CTA of the blocked kernel
constexpr int kStagePerThread = 16; // register-staged plane elements per thread
// Build of the blocked kernel a parameter set runs (see kernels_impl.cuh):
// FP64 with 3 or more CTAs per SM uses the 64-register, 2-plane-prefetch build.
inline int kernel_variant(int dtype, int ctas_per_sm) { return (dtype == EBISU_F64 && ctas_per_sm >= 3) ? 1 : 0; }
// Input planes in flight (cp.async) of a build.
inline int prefetch_planes(int ndim, int variant, size_t esize)
{
    return (variant == 1 || ndim == 3) ? 2 : (esize == 8 ? 3 : 4);
}

struct DeviceInfo {
    int device = -1;
    int sms = 0;
    size_t smem_optin = 0;
    size_t smem_per_sm = 0;
    char name[256] = {0};
    // measured rates (filled lazily by the tuner)
    double f64 = 0, f32 = 0, lds = 0, barrier_s = 0;
};

// Cached properties of the current device (queried once per device).
const DeviceInfo& device_info();
// Measured throughputs for the cost model; runs the microbenchmarks once per
// process (or uses defaults from a host without a GPU).
const DeviceInfo& device_rates();
// Replace the current device's rates with a probe's results (ebisu_probe_device
// output layout), so the cost model and the caller's roofline use one figure.
void record_device_rates(const double* probe_out);

void set_cuda_error(cudaError_t e);
// Record a failed CUDA call (its error and the source line that saw it, for
// ebisu_last_cuda_error), clear the runtime's last-error state so the
// caller's next CUDA call does not report it again, and return EBISU_ERR_CUDA.
int fail_cuda_at(cudaError_t e, const char* file, int line);
#define fail_cuda(e) ::ebisu::fail_cuda_at((e), __FILE__, __LINE__)

int ring_q(int radius);   // slots of a level-1.. ring (2r+2)
int ring_q0(int radius, int ndim, int variant, size_t esize);  // input ring slots (2r+1+prefetch)
// Elements per ring plane and dynamic shared memory of a parameter set.
int64_t plane_capacity(const ebisu_plan_s* p, const ebisu_params& q);
size_t tb_smem_bytes(const ebisu_plan_s* p, const ebisu_params& q);
// Validate a parameter set against the plan and the device.
int check_params(const ebisu_plan_s* p, const ebisu_params& q);
// Cost-model ranking (tune.cpp): writes up to `cap` candidates, best first.
// `share` is the fraction of the GPU the plan will have (1 = alone; a batch
// member gets less), which sizes the streamed bands.
int rank_candidates(const ebisu_plan_s* p, int64_t steps, ebisu_params* out, double* pred, int cap,
                    double share = 1.0);
// Cost model of one parameter set (tune.cpp).
double model_pp(const ebisu_plan_s* p, const ebisu_params& q, int64_t steps, int* bound, double* valid);

// Fill a GridDesc for one run of `steps` steps; returns the number of items.
int64_t fill_grid_desc(const ebisu_plan_s* p, const void* in, void* out, void* wsgrid, int64_t steps,
                       bool in_copied_to_ws, GridDesc* g);

cudaError_t tb_launch(const ebisu_plan_s* p, int variant, const TBParams& prm, int grid, size_t smem,
                      cudaStream_t st);
cudaError_t tb_occupancy(const ebisu_plan_s* p, int variant, size_t smem, int* blocks);
// one step (t = 1 .. steps: the step whose result is written; stochastic
// rounding keys its random bits on it)
cudaError_t naive_launch(const ebisu_plan_s* p, const void* src, void* dst, int64_t t, cudaStream_t st);
// one step with the plan's per-cell weights (variable coefficients)
cudaError_t naive_vc_launch(const ebisu_plan_s* p, const void* src, void* dst, cudaStream_t st);
// does the plan store BF16 with stochastic rounding (its own kernel builds)?
inline bool plan_sr(const ebisu_plan_s* p) { return p->dtype == EBISU_BF16 && p->rounding == EBISU_ROUND_STOCHASTIC; }
cudaError_t pad_copy(const ebisu_plan_s* p, const void* src, void* d0, void* d1, cudaStream_t st);

int64_t wait_timeout_ns();

// Register-streaming build (variant 2, 2D): strips of S columns, segments of H rows.
struct RSLayout {
    int S, H, nstrips, nsegs;
    int TY = 1, nbands = 1;  // 3D: rows per patch, patches along y
};
int rs_layout(const ebisu_plan_s* p, const ebisu_params& q, RSLayout* L);
cudaError_t rs_launch(const ebisu_plan_s* p, int depth, const RSParams& prm, int grid, cudaStream_t st);
cudaError_t rs_occupancy(const ebisu_plan_s* p, int depth, bool batch, int* blocks);
cudaError_t rs3_launch(const ebisu_plan_s* p, int depth, const RS3Params& prm, int grid, cudaStream_t st);
cudaError_t rs3_occupancy(const ebisu_plan_s* p, int depth, int* blocks);
// Fill the descriptor of one register-streaming run of `steps` >= 1 steps
// (src0: the first block's input; pads of the other written buffers are
// filled by the kernel).  Returns the number of temporal blocks.
int64_t fill_rs_grid(const ebisu_plan_s* p, const RSLayout& L, const void* in, void* out, void* wsgrid,
                     int64_t steps, bool in_copied_to_ws, RSGrid* g);

}  // namespace ebisu
