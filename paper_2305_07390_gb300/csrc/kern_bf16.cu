// Kernel instantiations for BF16 storage (FP32 arithmetic, every step
// rounded to BF16, nearest even).
#include "kernels_impl.cuh"
EBISU_DEFINE_DTYPE_ENTRY(__nv_bfloat16, bf16)
