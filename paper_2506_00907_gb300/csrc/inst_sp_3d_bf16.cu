// Kernel variants of the 3D lattices with several concentration species, __nv_bfloat16 storage.
#include "dispatch.cuh"
LBM_DEFINE_SPECIES_SET(species_3d_bf16, 3, __nv_bfloat16)
