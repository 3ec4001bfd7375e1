// Kernel variants of the 3D lattices with several concentration species, __half storage.
#include "dispatch.cuh"
LBM_DEFINE_SPECIES_SET(species_3d_f16, 3, __half)
