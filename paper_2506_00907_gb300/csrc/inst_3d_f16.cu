// Kernel variants of the 3D lattices with __half population storage.
#include "dispatch.cuh"
LBM_DEFINE_KERNEL_SET(kernels_3d_f16, 3, __half)
