// Register-streaming 3D kernels for FP32 storage: poisson and j3d17pt.
#define EBISU_RS3D_KERNELS
#include "rs_impl.cuh"
EBISU_DEFINE_RS3D_PTRS(float, f32, 1)
