// Kernel variants of the 2D lattices with several concentration species, double storage.
#include "dispatch.cuh"
LBM_DEFINE_SPECIES_SET(species_2d_f64, 2, double)
