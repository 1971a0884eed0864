// Row-staged collide-stream kernels of the rD2Q25 lattice (instantiation unit).
#include "mrt_kernels.cuh"
#include "row_kernels.cuh"

LBM_INSTANTIATE_ROWS(LBM_RD2Q25)
