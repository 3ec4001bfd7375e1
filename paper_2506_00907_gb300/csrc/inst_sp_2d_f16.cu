// Kernel variants of the 2D lattices with several concentration species, __half storage.
#include "dispatch.cuh"
LBM_DEFINE_SPECIES_SET(species_2d_f16, 2, __half)
