// Kernel variants of the 3D lattices with several concentration species, double storage.
#include "dispatch.cuh"
LBM_DEFINE_SPECIES_SET(species_3d_f64, 3, double)
