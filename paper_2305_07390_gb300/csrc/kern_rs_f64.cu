// Register-streaming kernel instantiations (2D) for FP64 storage.
#include "rs_impl.cuh"
EBISU_DEFINE_RS_ENTRY(double, f64)
