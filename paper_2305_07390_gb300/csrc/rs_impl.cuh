// rs_impl.cuh -- instantiation and launch glue of the register-streaming
// kernels (rs_kernel.cuh, rs3_kernel.cuh, rs3t_kernel.cuh).
//
// The kernels of one storage type are instantiated in three translation
// units so that the build compiles them in parallel:
//   kern_rs_<t>_single.cu : 2D, one problem per launch   -> rs_ptr_<t>_0
//   kern_rs_<t>_batch.cu  : 2D, batched launches          -> rs_ptr_<t>_1
//   kern_rs3_<t>.cu       : 3D                            -> rs3_ptr_<t>
// and kern_rs_<t>.cu holds the launchers, which look the kernel up through
// those functions.
#pragma once
#include <cuda_runtime.h>

#include "dispatch.h"

namespace ebisu {

// The 2D kernel of (shape, radius, depth) for one storage type and batch
// mode, or null if that depth is not built.
#define EBISU_RS2D_PTR_BODY(T, BATCH)                                                  \
    {                                                                                  \
        if (shape == kStar && r == 1) return rs_ptr_pick<T, kStar, 1, BATCH>(depth);   \
        if (shape == kStar && r == 2) return rs_ptr_pick<T, kStar, 2, BATCH>(depth);   \
        if (shape == kStar && r == 3) return rs_ptr_pick<T, kStar, 3, BATCH>(depth);   \
        if (shape == kBox && r == 1) return rs_ptr_pick<T, kBox, 1, BATCH>(depth);     \
        if (shape == kBox && r == 2) return rs_ptr_pick<T, kBox, 2, BATCH>(depth);     \
        return nullptr;                                                                \
    }

}  // namespace ebisu

#ifdef EBISU_RS2D_KERNELS
#include "rs_kernel.cuh"
namespace ebisu {
template <class T, int S_, int R_, bool BATCH>
static const void* rs_ptr_pick(int depth)
{
    constexpr int d0 = rs_depth((int)sizeof(T), S_, R_, 0);
    constexpr int d1 = rs_depth((int)sizeof(T), S_, R_, 1);
    if (depth == d0) return (const void*)&rs_kernel<T, S_, R_, d0, BATCH>;
    if (d1 != d0 && depth == d1) return (const void*)&rs_kernel<T, S_, R_, d1, BATCH>;
    return nullptr;
}
}  // namespace ebisu
// defines rs_ptr_<NAME>_<B>(shape, r, depth)
#define EBISU_DEFINE_RS2D_PTRS(T, NAME, B)                                                 \
    namespace ebisu {                                                                      \
    const void* rs_ptr_##NAME##_##B(int shape, int r, int depth) EBISU_RS2D_PTR_BODY(T, (B != 0)) \
    }
#endif

#ifdef EBISU_RS3D_KERNELS
#include <type_traits>

#include "rs3_kernel.cuh"
#include "rs3t_kernel.cuh"
// defines rs3_ptr_<NAME>_<PART>(shape, r, depth), the 3D kernels of one
// storage type split over two translation units so that they compile in
// parallel: part 0 the stars and the 27-point box, part 1 poisson and
// j3d17pt.  FP64 at depth 1 (the 7- and 13-point stars, the three radius-1
// boxes); FP32 and BF16 radius 1: the 7-point star at depth 2 or 3, the
// others at depth 2.
#define EBISU_DEFINE_RS3D_PTRS(T, NAME, PART)                                                          \
    namespace ebisu {                                                                                  \
    const void* rs3_ptr_##NAME##_##PART(int shape, int r, int depth)                                   \
    {                                                                                                  \
        if constexpr (PART == 0) {                                                                     \
            if constexpr (sizeof(T) == 8) {                                                            \
                if (depth != 1) return nullptr;                                                        \
                if (shape == kStar && r == 1) return (const void*)&rs3_kernel<T, kStar, 1>;            \
                if (shape == kStar && r == 2) return (const void*)&rs3_kernel<T, kStar, 2>;            \
                if (shape == kBox && r == 1) return (const void*)&rs3_kernel<T, kBox, 1>;              \
            } else {                                                                                   \
                if (r == 1 && shape == kStar && depth == 2) return (const void*)&rs3t_kernel<T, kStar, 2>; \
                if (r == 1 && shape == kStar && depth == 3) return (const void*)&rs3t_kernel<T, kStar, 3>; \
                if (r == 1 && shape == kBox && depth == 2) return (const void*)&rs3t_kernel<T, kBox, 2>; \
            }                                                                                          \
        } else {                                                                                       \
            if constexpr (sizeof(T) == 8) {                                                            \
                if (depth != 1) return nullptr;                                                        \
                if (shape == kPoisson && r == 1) return (const void*)&rs3_kernel<T, kPoisson, 1>;      \
                if (shape == kJ3d17 && r == 1) return (const void*)&rs3_kernel<T, kJ3d17, 1>;          \
            } else {                                                                                   \
                if (r == 1 && shape == kPoisson && depth == 2)                                         \
                    return (const void*)&rs3t_kernel<T, kPoisson, 2>;                                  \
                if (r == 1 && shape == kJ3d17 && depth == 2) return (const void*)&rs3t_kernel<T, kJ3d17, 2>; \
            }                                                                                          \
        }                                                                                              \
        (void)shape; (void)r; (void)depth;                                                             \
        return nullptr;                                                                                \
    }                                                                                                  \
    }
#endif

// launchers and occupancy queries of one storage type
#define EBISU_DEFINE_RS_ENTRY(T, NAME)                                                                   \
    namespace ebisu {                                                                                    \
    static const void* rs_ptr_##NAME(int s, int r, int d, bool batch)                                    \
    {                                                                                                    \
        return batch ? rs_ptr_##NAME##_1(s, r, d) : rs_ptr_##NAME##_0(s, r, d);                          \
    }                                                                                                    \
    cudaError_t rs_launch_##NAME(int s, int r, int d, const RSParams& p, int g, cudaStream_t st)         \
    {                                                                                                    \
        const void* k = rs_ptr_##NAME(s, r, d, p.grids != nullptr);                                      \
        if (!k) return cudaErrorInvalidValue;                                                            \
        void* args[] = {(void*)&p};                                                                      \
        return cudaLaunchKernel(k, dim3(g), dim3(kRSThreads), args, 0, st);                              \
    }                                                                                                    \
    cudaError_t rs_occupancy_##NAME(int s, int r, int d, bool bt, int* b)                                \
    {                                                                                                    \
        const void* k = rs_ptr_##NAME(s, r, d, bt);                                                      \
        if (!k) return cudaErrorInvalidValue;                                                            \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, k, kRSThreads, 0);                       \
    }                                                                                                    \
    static const void* rs3_ptr_##NAME(int s, int r, int d)                                               \
    {                                                                                                    \
        const void* k = rs3_ptr_##NAME##_0(s, r, d);                                                     \
        return k ? k : rs3_ptr_##NAME##_1(s, r, d);                                                      \
    }                                                                                                    \
    cudaError_t rs3_launch_##NAME(int s, int r, int d, const RS3Params& p, int g, cudaStream_t st)       \
    {                                                                                                    \
        const void* k = rs3_ptr_##NAME(s, r, d);                                                         \
        if (!k) return cudaErrorInvalidValue;                                                            \
        void* args[] = {(void*)&p};                                                                      \
        return cudaLaunchKernel(k, dim3(g), dim3(kRSThreads), args, 0, st);                              \
    }                                                                                                    \
    cudaError_t rs3_occupancy_##NAME(int s, int r, int d, int* b)                                        \
    {                                                                                                    \
        const void* k = rs3_ptr_##NAME(s, r, d);                                                         \
        if (!k) return cudaErrorInvalidValue;                                                            \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, k, kRSThreads, 0);                       \
    }                                                                                                    \
    }
