// Row-staged collide-stream kernels of the rD2Q9 lattice (instantiation unit).
#include "mrt_kernels.cuh"
#include "row_kernels.cuh"

LBM_INSTANTIATE_ROWS(LBM_RD2Q9)
