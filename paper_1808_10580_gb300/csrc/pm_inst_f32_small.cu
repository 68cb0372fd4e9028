// Instantiations of the particle kernels: float paths, K in {0 1 2 3 4 5 6}.
#include "pm_kernels.cuh"

PM_INSTANTIATE(float, 0)
PM_INSTANTIATE(float, 1)
PM_INSTANTIATE(float, 2)
PM_INSTANTIATE(float, 3)
PM_INSTANTIATE(float, 4)
PM_INSTANTIATE(float, 5)
PM_INSTANTIATE(float, 6)
