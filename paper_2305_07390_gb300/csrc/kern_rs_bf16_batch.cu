// Register-streaming 2D kernels for BF16 storage, batched launches.
#define EBISU_RS2D_KERNELS
#include "rs_impl.cuh"
EBISU_DEFINE_RS2D_PTRS(__nv_bfloat16, bf16, 1)
