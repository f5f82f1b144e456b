// rs_impl.cuh -- instantiation and launch glue of the register-streaming
// kernel (rs_kernel.cuh), included once per storage type.
#pragma once
#include <cuda_runtime.h>

#include "dispatch.h"
#include "rs3_kernel.cuh"
#include "rs3t_kernel.cuh"
#include "rs_kernel.cuh"

namespace ebisu {

template <class T>
static const void* rs_kernel_ptr(int shape, int r, int depth, bool batch)
{
#define X(S_, R_)                                                                                    \
    if (shape == S_ && r == R_) {                                                                    \
        constexpr int d0 = rs_depth((int)sizeof(T), S_, R_, 0);                                      \
        constexpr int d1 = rs_depth((int)sizeof(T), S_, R_, 1);                                      \
        if (depth == d0)                                                                             \
            return batch ? (const void*)&rs_kernel<T, S_, R_, d0, true>                              \
                         : (const void*)&rs_kernel<T, S_, R_, d0, false>;                            \
        if (d1 != d0 && depth == d1)                                                                 \
            return batch ? (const void*)&rs_kernel<T, S_, R_, d1, true>                              \
                         : (const void*)&rs_kernel<T, S_, R_, d1, false>;                            \
        return nullptr;                                                                              \
    }
    X(kStar, 1) X(kStar, 2) X(kStar, 3) X(kBox, 1) X(kBox, 2)
#undef X
    return nullptr;
}

template <class T>
static cudaError_t rs_launch_t(int shape, int r, int depth, const RSParams& p, int grid, cudaStream_t st)
{
    const void* k = rs_kernel_ptr<T>(shape, r, depth, p.grids != nullptr);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(k, dim3(grid), dim3(kRSThreads), args, 0, st);
}

template <class T>
static cudaError_t rs_occupancy_t(int shape, int r, int depth, bool batch, int* blocks)
{
    const void* k = rs_kernel_ptr<T>(shape, r, depth, batch);
    if (!k) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kRSThreads, 0);
}

// 3D: FP64 at depth 1 (the 7- and 13-point stars and the 27-point box);
// FP32: the 7-point star at depth 2 or 3, the 27-point box at depth 2 (rs3t_kernel.cuh).
template <class T>
static const void* rs3_kernel_ptr(int shape, int r, int depth)
{
    if constexpr (sizeof(T) == 8) {
        if (depth != 1) return nullptr;
        if (shape == kStar && r == 1) return (const void*)&rs3_kernel<T, kStar, 1>;
        if (shape == kStar && r == 2) return (const void*)&rs3_kernel<T, kStar, 2>;
        if (shape == kBox && r == 1) return (const void*)&rs3_kernel<T, kBox, 1>;
    } else if constexpr (std::is_same<T, float>::value) {
        if (r == 1 && shape == kStar && depth == 2) return (const void*)&rs3t_kernel<T, kStar, 2>;
        if (r == 1 && shape == kStar && depth == 3) return (const void*)&rs3t_kernel<T, kStar, 3>;
        if (r == 1 && shape == kBox && depth == 2) return (const void*)&rs3t_kernel<T, kBox, 2>;
    }
    return nullptr;
}

template <class T>
static cudaError_t rs3_launch_t(int shape, int r, int depth, const RS3Params& p, int grid, cudaStream_t st)
{
    const void* k = rs3_kernel_ptr<T>(shape, r, depth);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(k, dim3(grid), dim3(kRSThreads), args, 0, st);
}

template <class T>
static cudaError_t rs3_occupancy_t(int shape, int r, int depth, int* blocks)
{
    const void* k = rs3_kernel_ptr<T>(shape, r, depth);
    if (!k) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kRSThreads, 0);
}

}  // namespace ebisu

#define EBISU_DEFINE_RS_ENTRY(T, NAME)                                                              \
    namespace ebisu {                                                                               \
    cudaError_t rs_launch_##NAME(int s, int r, int d, const RSParams& p, int g, cudaStream_t st)    \
    {                                                                                               \
        return rs_launch_t<T>(s, r, d, p, g, st);                                                   \
    }                                                                                               \
    cudaError_t rs_occupancy_##NAME(int s, int r, int d, bool bt, int* b) { return rs_occupancy_t<T>(s, r, d, bt, b); } \
    cudaError_t rs3_launch_##NAME(int s, int r, int d, const RS3Params& p, int g, cudaStream_t st) \
    {                                                                                               \
        return rs3_launch_t<T>(s, r, d, p, g, st);                                                  \
    }                                                                                               \
    cudaError_t rs3_occupancy_##NAME(int s, int r, int d, int* b) { return rs3_occupancy_t<T>(s, r, d, b); } \
    }
