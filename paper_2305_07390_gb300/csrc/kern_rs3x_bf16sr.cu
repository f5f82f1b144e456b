// Register-streaming 3D kernels for BF16 with stochastic rounding storage: poisson and j3d17pt.
#define EBISU_RS3D_KERNELS
#include "rs_impl.cuh"
EBISU_DEFINE_RS3D_PTRS(bf16sr, bf16sr, 1)
