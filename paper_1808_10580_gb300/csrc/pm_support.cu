// pm_support.cu -- small kernels around the particle kernels: per-observation
// preparation, deterministic double-precision reductions, and the RNG
// diagnostics.
#include <cmath>

#include "pm_device.cuh"
#include "pm_launch.h"

namespace pm {

// ---------------------------------------------------------------------------
// Per-observation records: N_j = ceil(t_j/dt - 1e-9) steps of dt, the last
// one shortened to t_j - (N_j - 1) dt.  Flags non-finite inputs, negative
// times and step counts beyond int32 in *err.
// ---------------------------------------------------------------------------
__global__ void prep_timedep_kernel(const double* __restrict__ x, const double* __restrict__ t, int64_t n_obs,
                                    double dt, double kappa, ObsRec* __restrict__ rec, unsigned int* err,
                                    unsigned long long* step_count, int64_t M)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_obs) return;
    const double x1 = x[2 * j], x2 = x[2 * j + 1], tj = t[j];
    ObsRec r;
    r.x1 = x1;
    r.x2 = x2;
    r.pad = 0;
    bool bad = !isfinite(x1) || !isfinite(x2) || !isfinite(tj) || tj < 0.0;
    double steps = 0.0;
    if (!bad && tj > 0.0) steps = ceil(tj / dt - 1e-9);
    if (steps > 2147483646.0) bad = true;
    if (bad) {
        atomicOr(err, 1u);
        r.nsteps = 0;
        r.h_last = 0.0;
        r.s_last = 0.0;
    } else {
        const int32_t N = (int32_t)steps;
        r.nsteps = N;
        r.h_last = N > 0 ? __dsub_rn(tj, __dmul_rn((double)(N - 1), dt)) : 0.0;
        r.s_last = sqrt(__dmul_rn(__dmul_rn(2.0, kappa), r.h_last));
        if (step_count) atomicAdd(step_count, (unsigned long long)N * (unsigned long long)M);
    }
    rec[j] = r;
}

// Longest-first processing order (stable): rank of j = #{k : N_k > N_j} +
// #{k < j : N_k = N_j}.  Quadratic in n_obs; the host uses it for n_obs <= 8192.

__global__ void order_kernel(const ObsRec* __restrict__ rec, int64_t n_obs, int32_t* __restrict__ order)
{
    __shared__ int32_t tile[256];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t Nj = j < n_obs ? rec[j].nsteps : 0;
    int64_t rank = 0;
    for (int64_t base = 0; base < n_obs; base += 256) {
        const int64_t k = base + threadIdx.x;
        tile[threadIdx.x] = k < n_obs ? rec[k].nsteps : -1;
        __syncthreads();
        const int64_t lim = (n_obs - base) < 256 ? (n_obs - base) : 256;
        for (int q = 0; q < lim; ++q) {
            const int32_t Nk = tile[q];
            rank += (Nk > Nj) || (Nk == Nj && base + q < j);
        }
        __syncthreads();
    }
    if (j < n_obs) order[rank] = (int32_t)j;
}

cudaError_t launch_prep_timedep(const double* x, const double* t, int64_t n_obs, double dt, double kappa,
                                ObsRec* rec, int32_t* order, unsigned int* err, cudaStream_t s,
                                unsigned long long* steps, int64_t M)
{
    const unsigned grid = (unsigned)((n_obs + 255) / 256);
    prep_timedep_kernel<<<grid, 256, 0, s>>>(x, t, n_obs, dt, kappa, rec, err, steps, M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || order == nullptr) return e;
    order_kernel<<<grid, 256, 0, s>>>(rec, n_obs, order);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reductions.  Neumaier-compensated sums in a fixed order: lane l of the warp
// of observation j takes items l, l+32, ...; the 32 partial (sum, carry)
// pairs are then combined by a fixed shuffle tree.  mean = S/M,
// var = (S2 - S mean)/(M - 1).
// ---------------------------------------------------------------------------
struct Kahan {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double v)
    {
        const double t = s + v;
        c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    __device__ __forceinline__ double value() const { return s + c; }
};

__device__ __forceinline__ void warp_combine(Kahan& k)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s = __shfl_down_sync(0xffffffffu, k.s, off);
        const double c = __shfl_down_sync(0xffffffffu, k.c, off);
        k.add(s);
        k.c += c;
    }
}

__device__ __forceinline__ void finish_stats(double S, double S2, int64_t M, double* mean, double* var, int64_t j)
{
    const double m = S / (double)M;
    mean[j] = m;
    if (var) {
        double v = M > 1 ? (S2 - S * m) / (double)(M - 1) : 0.0;
        var[j] = v > 0.0 ? v : 0.0;
    }
}

__global__ void reduce_chunks_kernel(const double2* __restrict__ part, int64_t n_obs, int32_t chunks, int64_t M,
                                     double* __restrict__ mean, double* __restrict__ var)
{
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n_obs) return;
    Kahan a, b;
    for (int c = lane; c < chunks; c += 32) {
        const double2 p = part[j * chunks + c];
        a.add(p.x);
        b.add(p.y);
    }
    warp_combine(a);
    warp_combine(b);
    if (lane == 0) finish_stats(a.value(), b.value(), M, mean, var, j);
}

cudaError_t launch_reduce(const double2* part, int64_t n_obs, int32_t chunks, int64_t M, double* mean, double* var,
                          cudaStream_t s)
{
    const unsigned grid = (unsigned)((n_obs + 7) / 8);
    reduce_chunks_kernel<<<grid, 256, 0, s>>>(part, n_obs, chunks, M, mean, var);
    return cudaGetLastError();
}

// Per-path values g[j*M + i]: one CTA of 256 threads per observation; thread
// t takes i = t, t+256, ... (Neumaier), then a fixed tree over the warps.
__global__ void reduce_paths_kernel(const double* __restrict__ g, int64_t M, double* __restrict__ mean,
                                    double* __restrict__ var)
{
    const int64_t j = blockIdx.x;
    const double* gj = g + j * M;
    Kahan a, b;
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        const double v = gj[i];
        a.add(v);
        b.add(v * v);
    }
    warp_combine(a);
    warp_combine(b);
    __shared__ double sa[8], sca[8], sb[8], scb[8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sa[w] = a.s; sca[w] = a.c; sb[w] = b.s; scb[w] = b.c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        Kahan A, B;
        for (int k = 0; k < 8; ++k) { A.add(sa[k]); A.c += sca[k]; B.add(sb[k]); B.c += scb[k]; }
        finish_stats(A.value(), B.value(), M, mean, var, j);
    }
}

// Long rows (M > kReducePathChunk): first one CTA per (observation, chunk of
// kReducePathChunk paths) forms the chunk's compensated (sum, sum of squares)
// in the same fixed order, then reduce_chunks_kernel combines the chunks in
// chunk order.  Enough CTAs to stream the per-path array at HBM speed.
__global__ void reduce_path_chunks_kernel(const double* __restrict__ g, int64_t M, int32_t chunks,
                                          double2* __restrict__ part)
{
    const int64_t j = blockIdx.y;
    const int64_t i0 = (int64_t)blockIdx.x * kReducePathChunk;
    const int64_t i1 = (i0 + kReducePathChunk < M) ? i0 + kReducePathChunk : M;
    const double* gj = g + j * M;
    Kahan a, b;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double v = gj[i];
        a.add(v);
        b.add(v * v);
    }
    warp_combine(a);
    warp_combine(b);
    __shared__ double sa[8], sca[8], sb[8], scb[8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sa[w] = a.s; sca[w] = a.c; sb[w] = b.s; scb[w] = b.c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        Kahan A, B;
        for (int k = 0; k < 8; ++k) { A.add(sa[k]); A.c += sca[k]; B.add(sb[k]); B.c += scb[k]; }
        part[j * chunks + blockIdx.x] = make_double2(A.value(), B.value());
    }
}

int32_t reduce_path_chunks(int64_t M) { return M > kReducePathChunk ? (int32_t)((M + kReducePathChunk - 1) / kReducePathChunk) : 0; }

cudaError_t launch_reduce_paths(const double* g, int64_t n_obs, int64_t M, double* mean, double* var, cudaStream_t s,
                                double2* part)
{
    const int32_t chunks = reduce_path_chunks(M);
    if (chunks == 0 || part == nullptr) {
        reduce_paths_kernel<<<(unsigned)n_obs, 256, 0, s>>>(g, M, mean, var);
        return cudaGetLastError();
    }
    reduce_path_chunks_kernel<<<dim3((unsigned)chunks, (unsigned)n_obs), 256, 0, s>>>(g, M, chunks, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce(part, n_obs, chunks, M, mean, var, s);
}

// ---------------------------------------------------------------------------
// RNG diagnostics.
// ---------------------------------------------------------------------------
__global__ void philox_kernel(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1, int64_t n, uint4* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint4 c = ctr[q];
    const u32x4 r = philox4x32_10(u32x4{c.x, c.y, c.z, c.w}, k0, k1);
    out[q] = make_uint4(r.x, r.y, r.z, r.w);
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), k0, k1, n,
                                                              reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

// sin and cos of 2 pi x as the tensor-core kernels' harmonic recurrences form
// them (sincos_turns2), for points x[n] (float), two points per thread.
__global__ void sincos_turns_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ s, float* __restrict__ c)
{
    const int64_t q = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (q >= n) return;
    const bool two = q + 1 < n;
    float2 sv, cv;
    sincos_turns2(make_float2(x[q], two ? x[q + 1] : 0.f), sv, cv);
    s[q] = sv.x;
    c[q] = cv.x;
    if (two) {
        s[q + 1] = sv.y;
        c[q + 1] = cv.y;
    }
}

cudaError_t launch_sincos_turns(const float* x, int64_t n, float* s, float* c, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t pairs = (n + 1) / 2;
    sincos_turns_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(x, n, s, c);
    return cudaGetLastError();
}

template <typename Real>
__global__ void normals_kernel(uint32_t k0, uint32_t k1, uint32_t b, uint32_t j, uint32_t i, int64_t n0,
                               int64_t count, double* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const int64_t n = n0 + q;
    const u32x4 r = philox4x32_10(u32x4{(uint32_t)(n >> 1), i, j, b}, k0, k1);
    Real xi1, xi2;
    if ((n & 1) == 0) box_muller<Real>(r.x, r.y, xi1, xi2);
    else box_muller<Real>(r.z, r.w, xi1, xi2);
    out[2 * q] = (double)xi1;
    out[2 * q + 1] = (double)xi2;
}

// The tensor-core kernels' form: both steps of a Philox block from one packed
// Box-Muller pass (box_muller2), the step's half taken.
__global__ void normals_packed_kernel(uint32_t k0, uint32_t k1, uint32_t b, uint32_t j, uint32_t i, int64_t n0,
                                      int64_t count, double* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const int64_t n = n0 + q;
    const u32x4 r = philox4x32_10(u32x4{(uint32_t)(n >> 1), i, j, b}, k0, k1);
    float2 z1, z2;
    box_muller2(r.x, r.y, r.z, r.w, z1, z2);
    out[2 * q] = (double)((n & 1) ? z1.y : z1.x);
    out[2 * q + 1] = (double)((n & 1) ? z2.y : z2.x);
}

cudaError_t launch_normals(uint64_t seed, uint32_t b, uint32_t j, uint32_t i, int64_t n0, int64_t count, double* out,
                           bool fp64, bool packed, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    const unsigned grid = (unsigned)((count + 255) / 256);
    if (packed) {
        normals_packed_kernel<<<grid, 256, 0, s>>>(k0, k1, b, j, i, n0, count, out);
        return cudaGetLastError();
    }
    if (fp64) normals_kernel<double><<<grid, 256, 0, s>>>(k0, k1, b, j, i, n0, count, out);
    else normals_kernel<float><<<grid, 256, 0, s>>>(k0, k1, b, j, i, n0, count, out);
    return cudaGetLastError();
}

}  // namespace pm
