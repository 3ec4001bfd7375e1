// Kernel variants of the 2D lattices with float population storage.
#include "dispatch.cuh"
LBM_DEFINE_KERNEL_SET(kernels_2d_f32, 2, float)
