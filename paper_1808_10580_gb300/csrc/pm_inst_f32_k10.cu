// Instantiations of the particle kernels: float paths, K in {10}.
#include "pm_batched.cuh"

PM_INSTANTIATE(float, 10)
PM_INSTANTIATE_BATCHED(10)
