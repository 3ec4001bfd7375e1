// Kernel variants of the 2D lattices with several concentration species, __nv_bfloat16 storage.
#include "dispatch.cuh"
LBM_DEFINE_SPECIES_SET(species_2d_bf16, 2, __nv_bfloat16)
