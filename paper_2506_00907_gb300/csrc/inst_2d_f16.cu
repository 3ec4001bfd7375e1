// Kernel variants of the 2D lattices with __half population storage.
#include "dispatch.cuh"
LBM_DEFINE_KERNEL_SET(kernels_2d_f16, 2, __half)
