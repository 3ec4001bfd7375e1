// Kernel variants of the 3D lattices with __nv_bfloat16 population storage.
#include "dispatch.cuh"
LBM_DEFINE_KERNEL_SET(kernels_3d_bf16, 3, __nv_bfloat16)
