// Instantiations of the particle kernels at the wide bound K = 64 (float
// paths): the time-dependent and Dirichlet maps on the FP32 pipes with the
// table in shared memory, and the time-dependent, Dirichlet and batched maps
// on the tensor cores with the coefficient tiles from global memory.
#include "pm_dirichlet_tc.cuh"
#include "pm_batched_tc.cuh"

PM_INSTANTIATE_WIDE(64)
PM_INSTANTIATE_TC(64)
PM_INSTANTIATE_DIR_TC(64)
PM_INSTANTIATE_BATCHED_TC(64)
