// Instantiations of the particle kernels: double paths, K in {8 10 12 16}.
#include "pm_kernels.cuh"

PM_INSTANTIATE(double, 8)
PM_INSTANTIATE(double, 10)
PM_INSTANTIATE(double, 12)
PM_INSTANTIATE(double, 16)
