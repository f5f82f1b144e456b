// Register-streaming 2D kernels for FP32 storage, one problem per launch.
#define EBISU_RS2D_KERNELS
#include "rs_impl.cuh"
EBISU_DEFINE_RS2D_PTRS(float, f32, 0)
