// Time-step and initialisation kernels of the rD3Q53 lattice (instantiation unit).
#include "mrt_kernels.cuh"

LBM_INSTANTIATE_LATTICE(LBM_RD3Q53)
