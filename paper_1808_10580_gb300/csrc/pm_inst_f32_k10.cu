// Instantiations of the particle kernels: float paths, K in {10}.
#include "pm_kernels.cuh"

PM_INSTANTIATE(float, 10)
