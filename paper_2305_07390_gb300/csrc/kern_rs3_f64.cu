// Register-streaming 3D kernels for FP64 storage.
#define EBISU_RS3D_KERNELS
#include "rs_impl.cuh"
EBISU_DEFINE_RS3D_PTRS(double, f64, 0)
