// Time-step and initialisation kernels of the single-speed rD3Q27 lattice (instantiation unit).
#include "mrt_kernels.cuh"

LBM_INSTANTIATE_LATTICE(LBM_RD3Q27)
