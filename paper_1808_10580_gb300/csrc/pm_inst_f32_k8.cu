// Instantiations of the particle kernels: float paths, K in {8}.
#include "pm_batched.cuh"

PM_INSTANTIATE(float, 8)
PM_INSTANTIATE_BATCHED(8)
