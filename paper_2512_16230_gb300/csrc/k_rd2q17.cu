// Time-step and initialisation kernels of the rD2Q17 lattice (instantiation unit).
#include "mrt_kernels.cuh"

LBM_INSTANTIATE_LATTICE(LBM_RD2Q17)
