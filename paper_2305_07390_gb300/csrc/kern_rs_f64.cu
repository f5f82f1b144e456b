// Register-streaming kernels for FP64 storage: launchers.
#include "rs_impl.cuh"
EBISU_DEFINE_RS_ENTRY(double, f64)
