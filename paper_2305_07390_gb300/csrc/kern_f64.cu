// Kernel instantiations for FP64 storage (FP64 arithmetic).
#include "kernels_impl.cuh"
EBISU_DEFINE_DTYPE_ENTRY(double, f64)
