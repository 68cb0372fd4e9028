// Test helper (not part of the library): raw draws of cuRAND's Philox4_32_10
// device generator, to cross-check the library's Philox4x32-10 against an
// independent implementation.  Built and loaded by tests/test_gpu_curand.py.
#include <cstdint>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(unsigned long long seed, unsigned long long subsequence,
                                     unsigned long long offset, int n, uint4* out)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subsequence, offset, &st);
    for (int k = 0; k < n; ++k) out[k] = curand4(&st);
}

// n consecutive curand4() results after curand_init(seed, subsequence, offset)
// into host[4 n]; 0 on success.
extern "C" int curand_philox_draws(unsigned long long seed, unsigned long long subsequence, unsigned long long offset,
                                   int n, unsigned* host)
{
    if (n < 1 || n > (1 << 16) || !host) return 1;
    uint4* d = nullptr;
    if (cudaMalloc(&d, sizeof(uint4) * (size_t)n) != cudaSuccess) return 2;
    curand_philox_kernel<<<1, 1>>>(seed, subsequence, offset, n, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(host, d, sizeof(uint4) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 3;
}
