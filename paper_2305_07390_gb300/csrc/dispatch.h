// dispatch.h -- host-callable launchers of the CUDA kernels, one set per
// storage type (defined in kern_f64.cu, kern_f32.cu, kern_bf16.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.h"

namespace ebisu {

// Arguments of the naive one-step kernel (streaming coordinates, see GridDesc).
struct NaiveParams {
    int64_t n[3];
    int64_t lds, ld1;
    int32_t pad;
    int32_t periodic;
    uint32_t sr_k;             // stochastic rounding: this step's key K_t (BF16-SR storage only)
    int32_t reserved_;
    double coef[kMaxPoints];
    float coef_f[kMaxPoints];  // the same rounded to FP32 on the host (FP32/BF16 storage)
};

// Geometry of a stored grid for pad copies and reductions.
struct PadParams {
    int64_t n[3];     // interior extents (s, p1, p2)
    int64_t lds, ld1; // element strides
    int32_t pad;      // pad along s and p2
    int32_t pad1;     // pad along p1 (0 in 2D)
};

#define EBISU_DECLARE_DTYPE_ENTRY(NAME)                                                          \
    cudaError_t tb_launch_##NAME(int d, int s, int r, int v, const TBParams& p, int g, size_t sm, \
                                 cudaStream_t st);                                               \
    cudaError_t tb_occupancy_##NAME(int d, int s, int r, int v, size_t sm, int* b);              \
    cudaError_t naive_launch_##NAME(int d, int s, int r, const void* a, void* b,                 \
                                    const NaiveParams& p, cudaStream_t st);                      \
    cudaError_t pad_copy_##NAME(const void* s, void* d0, void* d1, const PadParams& p,           \
                                cudaStream_t st);                                                \
    cudaError_t naive_vc_launch_##NAME(int d, int s, int r, const void* a, void* b, const void* f, \
                                       int64_t fs, const NaiveParams& p, cudaStream_t st);       \
    cudaError_t reduce_partial_##NAME(const void* a, const void* b, double* part,                \
                                      const PadParams& p, int64_t* n, cudaStream_t st);

// kernel lookups of the register-streaming builds (see rs_impl.cuh)
#define EBISU_DECLARE_RS_PTRS(NAME)                                \
    const void* rs_ptr_##NAME##_0(int shape, int r, int depth);    \
    const void* rs_ptr_##NAME##_1(int shape, int r, int depth);    \
    const void* rs3_ptr_##NAME##_0(int shape, int r, int depth);   \
    const void* rs3_ptr_##NAME##_1(int shape, int r, int depth);

EBISU_DECLARE_RS_PTRS(f64)
EBISU_DECLARE_RS_PTRS(f32)
EBISU_DECLARE_RS_PTRS(bf16)
EBISU_DECLARE_RS_PTRS(bf16sr)

#define EBISU_DECLARE_RS_ENTRY(NAME)                                                               \
    cudaError_t rs_launch_##NAME(int s, int r, int d, const RSParams& p, int g, cudaStream_t st);   \
    cudaError_t rs_occupancy_##NAME(int s, int r, int d, bool batch, int* b);                      \
    cudaError_t rs3_launch_##NAME(int s, int r, int d, const RS3Params& p, int g, cudaStream_t st); \
    cudaError_t rs3_occupancy_##NAME(int s, int r, int d, int* b);

EBISU_DECLARE_RS_ENTRY(f64)
EBISU_DECLARE_RS_ENTRY(f32)
EBISU_DECLARE_RS_ENTRY(bf16)
EBISU_DECLARE_RS_ENTRY(bf16sr)

// BF16 storage with stochastic rounding: the one-step kernel (kern_bf16sr.cu;
// pad copies and reductions use the BF16 ones, the storage is the same)
cudaError_t naive_launch_bf16sr(int d, int s, int r, const void* a, void* b, const NaiveParams& p, cudaStream_t st);

EBISU_DECLARE_DTYPE_ENTRY(f64)
EBISU_DECLARE_DTYPE_ENTRY(f32)
EBISU_DECLARE_DTYPE_ENTRY(bf16)

// kern_ablate.cu: ablation builds of the shared-memory kernel (2D 5-point
// and 3D 7-point star, FP32/FP64; mask = the tb_kernel.cuh kAbl* bits)
cudaError_t tb_ablate_launch(size_t esize, int dim, int mask, const TBParams& p, int grid, size_t smem,
                             cudaStream_t st);
cudaError_t tb_ablate_occupancy(size_t esize, int dim, int mask, size_t smem, int* blocks);

// util.cu
cudaError_t reduce_final(const double* part, int64_t nparts, double* out3_dev, cudaStream_t st);
cudaError_t probe_device(double* out6);

}  // namespace ebisu
