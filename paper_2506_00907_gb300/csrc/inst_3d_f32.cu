// Kernel variants of the 3D lattices with float population storage.
#include "dispatch.cuh"
LBM_DEFINE_KERNEL_SET(kernels_3d_f32, 3, float)
