// Instantiations of the time-dependent particle kernels at the wide bound
// K = 48 (float paths): FP32 pipes with the table in shared memory, and the
// tensor-core kernel with its coefficient tiles loaded from global memory.
#include "pm_timedep_tc.cuh"

PM_INSTANTIATE_WIDE(48)
PM_INSTANTIATE_TC(48)
