// Row-staged collide-stream kernels of the rD3Q33 lattice (instantiation unit).
#include "mrt_kernels.cuh"
#include "row_kernels.cuh"

LBM_INSTANTIATE_ROWS(LBM_RD3Q33)
