// Instantiations of the particle kernels: double paths, K in {0 1 2 3 4 5 6}.
#include "pm_kernels.cuh"

PM_INSTANTIATE(double, 0)
PM_INSTANTIATE(double, 1)
PM_INSTANTIATE(double, 2)
PM_INSTANTIATE(double, 3)
PM_INSTANTIATE(double, 4)
PM_INSTANTIATE(double, 5)
PM_INSTANTIATE(double, 6)
