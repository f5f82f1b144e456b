// Register-streaming kernels for FP32 storage: launchers.
#include "rs_impl.cuh"
EBISU_DEFINE_RS_ENTRY(float, f32)
