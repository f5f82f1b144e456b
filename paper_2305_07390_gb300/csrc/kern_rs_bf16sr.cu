// Register-streaming kernels for BF16 storage with stochastic rounding: launchers.
#include "rs_impl.cuh"
EBISU_DEFINE_RS_ENTRY(bf16sr, bf16sr)
