// Register-streaming kernels for BF16 storage (FP32 arithmetic): launchers.
#include "rs_impl.cuh"
EBISU_DEFINE_RS_ENTRY(__nv_bfloat16, bf16)
