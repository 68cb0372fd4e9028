// Instantiations of the particle kernels: float paths, K in {10}.
#include "pm_batched.cuh"
#include "pm_dirichlet_tc.cuh"
#include "pm_batched_tc.cuh"

PM_INSTANTIATE(float, 10)
PM_INSTANTIATE_BATCHED(10)
PM_INSTANTIATE_TC(10)
PM_INSTANTIATE_DIR_TC(10)
PM_INSTANTIATE_BATCHED_TC(10)
