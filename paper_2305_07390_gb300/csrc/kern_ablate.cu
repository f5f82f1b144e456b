// Ablation builds of the shared-memory temporally blocked kernel for the
// paper's two breakdown case studies (Section 7.4: the 2D 5-point and the 3D
// 7-point star), FP32 and FP64 storage.  Each build switches off one more
// element of the method (see tb_kernel.cuh): the cumulative steps BASE (no
// circular queue: shifting queues, no prefetch, no lazy streaming, no
// register reuse), +CMQ, +PRE, +LST; the last step, +RST, is the production
// build itself.
#include "kernels_impl.cuh"

namespace ebisu {

template <class T, int DIM, int ABL>
static const void* abl_kernel()
{
    using I = TBInst<T, DIM, kStar, 1, 0>;
    return (const void*)&tb_kernel<T, DIM, kStar, 1, kTBThreads, I::ILP, I::PF, kTBStage, I::MINB, I::VEC, ABL>;
}

template <class T, int DIM>
static const void* abl_pick(int mask)
{
    switch (mask) {
    case kAblNoCircular | kAblNoPrefetch | kAblNoLazy | kAblNoRegReuse: return abl_kernel<T, DIM, 15>();
    case kAblNoPrefetch | kAblNoLazy | kAblNoRegReuse: return abl_kernel<T, DIM, 7>();
    case kAblNoLazy | kAblNoRegReuse: return abl_kernel<T, DIM, 6>();
    case kAblNoRegReuse: return abl_kernel<T, DIM, 4>();
    default: return nullptr;
    }
}

static const void* abl_ptr(size_t esize, int dim, int mask)
{
    if (esize == 8) return dim == 2 ? abl_pick<double, 2>(mask) : abl_pick<double, 3>(mask);
    if (esize == 4) return dim == 2 ? abl_pick<float, 2>(mask) : abl_pick<float, 3>(mask);
    return nullptr;
}

cudaError_t tb_ablate_launch(size_t esize, int dim, int mask, const TBParams& p, int grid, size_t smem,
                             cudaStream_t st)
{
    const void* k = abl_ptr(esize, dim, mask);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(k, dim3(grid), dim3(kTBThreads), args, smem, st);
}

cudaError_t tb_ablate_occupancy(size_t esize, int dim, int mask, size_t smem, int* blocks)
{
    const void* k = abl_ptr(esize, dim, mask);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kTBThreads, smem);
}

}  // namespace ebisu
