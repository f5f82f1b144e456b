// Register-streaming kernel instantiations (2D) for FP32 storage.
#include "rs_impl.cuh"
EBISU_DEFINE_RS_ENTRY(float, f32)
