// One-step kernel for BF16 storage with stochastic rounding (FP32
// arithmetic, every step's result rounded to BF16 with the random bits of
// its cell and step).  Pad copies and reductions use the BF16 kernels.
#include "kernels_impl.cuh"
namespace ebisu {
cudaError_t naive_launch_bf16sr(int d, int s, int r, const void* a, void* b, const NaiveParams& p, cudaStream_t st)
{
    return naive_launch_t<bf16sr>(d, s, r, a, b, p, st);
}
}  // namespace ebisu
