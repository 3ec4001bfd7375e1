// Kernel variants of the 2D lattices with double population storage.
#include "dispatch.cuh"
LBM_DEFINE_KERNEL_SET(kernels_2d_f64, 2, double)
