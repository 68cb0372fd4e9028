// Instantiation of the time-dependent map at the widest bound K = 80 (float
// paths on the FP32 pipes, the velocity table staged in each CTA's shared
// memory); no tensor-core or Dirichlet kernel exists at this bound.
#include "pm_kernels.cuh"

template cudaError_t pm::launch_timedep<float, 80>(const pm::TimedepLaunch&, cudaStream_t);
