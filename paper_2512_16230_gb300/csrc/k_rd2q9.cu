// Time-step and initialisation kernels of the single-speed rD2Q9 lattice (instantiation unit).
#include "mrt_kernels.cuh"

LBM_INSTANTIATE_LATTICE(LBM_RD2Q9)
