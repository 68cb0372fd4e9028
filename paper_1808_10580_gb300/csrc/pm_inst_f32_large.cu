// Instantiations of the particle kernels: float paths, K in {12 16}.
#include "pm_kernels.cuh"

PM_INSTANTIATE(float, 12)
PM_INSTANTIATE(float, 16)
