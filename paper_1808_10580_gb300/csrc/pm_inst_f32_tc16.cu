// Instantiations of the tensor-core particle kernels at K = 16 (float paths).
#include "pm_batched.cuh"
#include "pm_dirichlet_tc.cuh"
#include "pm_batched_tc.cuh"

PM_INSTANTIATE_TC(16)
PM_INSTANTIATE_DIR_TC(16)
PM_INSTANTIATE_BATCHED_TC(16)
