// Kernel variants of the 2D lattices with __nv_bfloat16 population storage.
#include "dispatch.cuh"
LBM_DEFINE_KERNEL_SET(kernels_2d_bf16, 2, __nv_bfloat16)
