// Kernel instantiations for FP32 storage (FP32 arithmetic).
#include "kernels_impl.cuh"
EBISU_DEFINE_DTYPE_ENTRY(float, f32)
