// Kernel variants of the 2D lattices with several concentration species, float storage.
#include "dispatch.cuh"
LBM_DEFINE_SPECIES_SET(species_2d_f32, 2, float)
