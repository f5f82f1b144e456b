// Register-streaming 2D kernels for BF16 storage with stochastic rounding, batched launches.
#define EBISU_RS2D_KERNELS
#include "rs_impl.cuh"
EBISU_DEFINE_RS2D_PTRS(bf16sr, bf16sr, 1)
