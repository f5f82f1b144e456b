// Register-streaming 3D kernels for BF16 storage with stochastic rounding.
#define EBISU_RS3D_KERNELS
#include "rs_impl.cuh"
EBISU_DEFINE_RS3D_PTRS(bf16sr, bf16sr, 0)
