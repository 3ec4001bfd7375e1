// Kernel variants of the 3D lattices with double population storage.
#include "dispatch.cuh"
LBM_DEFINE_KERNEL_SET(kernels_3d_f64, 3, double)
