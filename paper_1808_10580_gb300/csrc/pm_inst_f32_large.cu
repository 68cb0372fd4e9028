// Instantiations of the particle kernels: float paths, K in {12 16}.
#include "pm_batched.cuh"
#include "pm_dirichlet_tc.cuh"
#include "pm_batched_tc.cuh"

PM_INSTANTIATE(float, 12)
PM_INSTANTIATE(float, 16)
PM_INSTANTIATE_BATCHED(12)
PM_INSTANTIATE_BATCHED(16)
PM_INSTANTIATE_TC(12)
PM_INSTANTIATE_DIR_TC(12)
PM_INSTANTIATE_BATCHED_TC(12)
