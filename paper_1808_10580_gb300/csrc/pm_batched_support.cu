// pm_batched_support.cu -- staging, per-row preparation and per-row reduction
// around the batched persistent kernel.
#include "pm_batched.cuh"

namespace pm {

namespace {
constexpr double kTwoPiD = 6.283185307179586476925286766559;

__device__ __forceinline__ int64_t half_idx(int K, int m, int n)
{
    return m == 0 ? (n - 1) : K + (int64_t)(m - 1) * (2 * K + 1) + (n + K);
}
}  // namespace

// One CTA per instance; thread t handles grid point (m, n) = (t / (K+1), t % (K+1)).
// For m, n >= 1 the modes (m, n) and (m, -n) fold into the product-basis
// coefficients A, B, G, D of C1 C2, C1 S2, S1 C2, S1 S2 (Eq. v_expand), then
// e = 2 pi n (A, -B, G, -D) and f = 2 pi m (G, D, -A, -B).
__global__ void stage_tables_kernel(const BatchInstDev* __restrict__ inst, int K, float* __restrict__ tables)
{
    const int b = blockIdx.x;
    const double* u = inst[b].u;
    const int TS = (K + 1) * (K + 1) * 8;
    for (int q = threadIdx.x; q < (K + 1) * (K + 1); q += blockDim.x) {
        const int m = q / (K + 1), n = q % (K + 1);
        double A = 0, B = 0, G = 0, D = 0;
        if (m == 0 && n > 0) { A = u[2 * half_idx(K, 0, n)]; B = u[2 * half_idx(K, 0, n) + 1]; }
        else if (m > 0 && n == 0) { A = u[2 * half_idx(K, m, 0)]; G = u[2 * half_idx(K, m, 0) + 1]; }
        else if (m > 0) {
            const double ap = u[2 * half_idx(K, m, n)], bp = u[2 * half_idx(K, m, n) + 1];
            const double am = u[2 * half_idx(K, m, -n)], bm = u[2 * half_idx(K, m, -n) + 1];
            A = ap + am; B = bp - bm; G = bp + bm; D = am - ap;
        }
        const double sn = kTwoPiD * n, sm = kTwoPiD * m;
        float* e = tables + (size_t)b * TS + (size_t)q * 8;
        e[0] = (float)(sn * A); e[1] = (float)(-sn * B); e[2] = (float)(sn * G); e[3] = (float)(-sn * D);
        e[4] = (float)(sm * G); e[5] = (float)(sm * D); e[6] = (float)(-sm * A); e[7] = (float)(-sm * B);
    }
}

cudaError_t launch_stage_tables(const BatchInstDev* inst, int B, int K, float* tables, cudaStream_t s)
{
    stage_tables_kernel<<<B, 128, 0, s>>>(inst, K, tables);
    return cudaGetLastError();
}

__global__ void prep_rows_kernel(const BatchInstDev* __restrict__ inst, const double* __restrict__ x,
                                 const double* __restrict__ t, RowRec* __restrict__ rows, unsigned* err)
{
    const BatchInstDev I = inst[blockIdx.y];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= I.n_obs) return;
    const int64_t r = I.row0 + j;
    RowRec rr;
    rr.x1 = x[2 * r];
    rr.x2 = x[2 * r + 1];
    rr.pad = 0;
    rr.nsteps = 0;
    rr.h_last = 0.0;
    rr.s_last = 0.0;
    bool bad = !isfinite(rr.x1) || !isfinite(rr.x2);
    if (I.kind == 0) {
        const double tj = t[r];
        bad = bad || !isfinite(tj) || tj < 0.0;
        double steps = (!bad && tj > 0.0) ? ceil(tj / I.dt - 1e-9) : 0.0;
        if (steps > 2147483646.0) { bad = true; steps = 0.0; }
        if (!bad) {
            const int32_t N = (int32_t)steps;
            rr.nsteps = N;
            rr.h_last = N > 0 ? __dsub_rn(tj, __dmul_rn((double)(N - 1), I.dt)) : 0.0;
            rr.s_last = sqrt(__dmul_rn(__dmul_rn(2.0, I.kappa), rr.h_last));
        }
    }
    if (bad) atomicOr(err, 1u);
    rows[r] = rr;
}

cudaError_t launch_prep_rows(const BatchInstDev* inst, int B, int max_obs, const double* x, const double* t,
                             RowRec* rows, unsigned* err, cudaStream_t s)
{
    dim3 grid((unsigned)((max_obs + 127) / 128), (unsigned)B);
    prep_rows_kernel<<<grid, 128, 0, s>>>(inst, x, t, rows, err);
    return cudaGetLastError();
}

namespace {
struct KahanB {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double v)
    {
        const double t = s + v;
        c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
};
__device__ __forceinline__ void warp_combine_b(KahanB& k)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s = __shfl_down_sync(0xffffffffu, k.s, off);
        const double c = __shfl_down_sync(0xffffffffu, k.c, off);
        k.add(s);
        k.c += c;
    }
}
}  // namespace

// One CTA of 256 threads per (instance, row): Neumaier sums in a fixed order.
__global__ void reduce_rows_kernel(const BatchInstDev* __restrict__ inst, const double* __restrict__ g,
                                   double* __restrict__ mean, double* __restrict__ var)
{
    const BatchInstDev I = inst[blockIdx.y];
    const int j = blockIdx.x;
    if (j >= I.n_obs) return;
    const double* gj = g + I.path_base + (int64_t)j * I.M;
    KahanB a, b;
    for (int64_t i = threadIdx.x; i < I.M; i += blockDim.x) {
        const double v = gj[i];
        a.add(v);
        b.add(v * v);
    }
    warp_combine_b(a);
    warp_combine_b(b);
    __shared__ double sa[8], sca[8], sb[8], scb[8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sa[w] = a.s; sca[w] = a.c; sb[w] = b.s; scb[w] = b.c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        KahanB A, Bs;
        for (int k = 0; k < 8; ++k) { A.add(sa[k]); A.c += sca[k]; Bs.add(sb[k]); Bs.c += scb[k]; }
        const double S = A.s + A.c, S2 = Bs.s + Bs.c;
        const double m = S / (double)I.M;
        const int64_t r = I.row0 + j;
        mean[r] = m;
        if (var) {
            const double v = I.M > 1 ? (S2 - S * m) / (double)(I.M - 1) : 0.0;
            var[r] = v > 0.0 ? v : 0.0;
        }
    }
}

cudaError_t launch_reduce_rows(const BatchInstDev* inst, int B, int max_obs, const double* g, double* mean,
                               double* var, cudaStream_t s)
{
    dim3 grid((unsigned)max_obs, (unsigned)B);
    reduce_rows_kernel<<<grid, 256, 0, s>>>(inst, g, mean, var);
    return cudaGetLastError();
}

}  // namespace pm
