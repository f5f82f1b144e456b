// rs_impl.cuh -- instantiation and launch glue of the register-streaming
// kernel (rs_kernel.cuh), included once per storage type.
#pragma once
#include <cuda_runtime.h>

#include "dispatch.h"
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

}  // namespace ebisu

#define EBISU_DEFINE_RS_ENTRY(T, NAME)                                                              \
    namespace ebisu {                                                                               \
    cudaError_t rs_launch_##NAME(int s, int r, int d, const RSParams& p, int g, cudaStream_t st)    \
    {                                                                                               \
        return rs_launch_t<T>(s, r, d, p, g, st);                                                   \
    }                                                                                               \
    cudaError_t rs_occupancy_##NAME(int s, int r, int d, bool bt, int* b) { return rs_occupancy_t<T>(s, r, d, bt, b); } \
    }
