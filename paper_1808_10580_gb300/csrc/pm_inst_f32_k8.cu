// Instantiations of the particle kernels: float paths, K in {8}.
#include "pm_kernels.cuh"

PM_INSTANTIATE(float, 8)
