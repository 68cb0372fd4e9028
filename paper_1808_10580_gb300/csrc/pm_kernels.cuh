// pm_kernels.cuh -- the particle kernels of Algorithms 1 and 2, templated on
// the path precision Real and the wave-number bound K.  Included by the
// per-precision translation units, which instantiate them for the supported K.
#pragma once
#include <vector>
#include "pm_device.cuh"
#include "pm_launch.h"

namespace pm {

// Launch parameters travel in the kernel-parameter constant bank: the
// velocity table is read as FMA operands at compile-time offsets, and every
// launch carries its own copy (no shared constant symbol, so concurrent calls
// on different streams cannot interfere).
// Velocity table of a launch: in the parameter bank, or (wide K, float paths)
// a device copy that every CTA stages into its shared memory.
template <typename Real, int K, bool Wide = (K > kMaxUnrolledK)>
struct FieldSource {
    FieldTable<Real, K> field;
};
template <int K>
struct FieldSource<float, K, true> {
    const float4* table;  // device [coef_count<K>() / 4]
};

template <typename Real, int K>
struct TimedepParams : FieldSource<Real, K> {
    Theta0Table<Real> th;
    const ObsRec* obs;
    const int32_t* order;
    double2* part;
    double* g_out;
    double* x_out;
    Real dt, s_dt;
    int64_t M, path_offset;
    int32_t n_obs, chunks;
    uint32_t inst, key0, key1;
    const int4* groups;       // shared paths: {m0, m1, stream, nmax} per grid row
    const int32_t* members;   // [n_obs] observation indices of the groups
};

template <typename Real>
__device__ __forceinline__ void em_update(Coord<Real>& X, Real v, Real h, Real s, Real xi);

// float: X += -v h + s xi, the increment formed with one FMA and added with compensation.
template <>
__device__ __forceinline__ void em_update<float>(Coord<float>& X, float v, float h, float s, float xi)
{
    X.add(fmaf(s, xi, -v * h));
}

// double: ((X - v h) + s xi) with each operation rounded once, the order the
// plain sequential statement of Eq. euler gives.
template <>
__device__ __forceinline__ void em_update<double>(Coord<double>& X, double v, double h, double s, double xi)
{
    X.hi = __dadd_rn(__dsub_rn(X.hi, __dmul_rn(v, h)), __dmul_rn(s, xi));
}

template <typename Real>
__device__ __forceinline__ double theta0_eval(const Theta0Table<Real>& th, const Coord<Real>& X1,
                                              const Coord<Real>& X2)
{
    Real acc = (Real)0;
    for (int q = 0; q < th.n; ++q) {
        const Real ph = phase_frac(th.k1[q], th.k2[q], X1, X2);
        Real s, c;
        sincos2pi(ph, &s, &c);
        acc = fma_(th.a[q], c, fma_(th.b[q], s, acc));
    }
    return (double)acc;
}

// Block-wide sum of (a, b) in double by warp shuffles and a fixed-order pass
// over the warps: deterministic for a given block size.
template <int BLOCK>
__device__ __forceinline__ double2 block_sum2(double a, double b)
{
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
    __shared__ double2 warp_part[BLOCK / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_part[w] = make_double2(a, b);
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < BLOCK / 32; ++k) { r.x += warp_part[k].x; r.y += warp_part[k].y; }
    }
    return r;
}

// The table a kernel reads: its parameter-bank copy, or for wide K the shared
// memory copy staged here (all threads of the CTA must call this).
template <typename Real, int K, typename Src>
__device__ __forceinline__ auto field_table(const Src& src)
{
    if constexpr (K > kMaxUnrolledK) {
        extern __shared__ float4 s_field[];
        constexpr int nq = coef_count<K>() / 4;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) s_field[q] = __ldg(src.table + q);
        __syncthreads();
        return SharedTable{s_field};
    } else {
        return ParamTable<Real, K>{src.field};
    }
}

// Dynamic shared memory of the kernels that read the table above.
template <typename Real, int K>
constexpr int field_smem() { return K > kMaxUnrolledK ? coef_count<K>() * (int)sizeof(float) : 0; }

// ---------------------------------------------------------------------------
// Algorithm 1.  One CTA = one chunk of BLOCK consecutive paths of one
// observation; all its paths take the same N_j steps, so the step loop is
// uniform.  Two Euler steps per Philox call.  Per-path g goes into a
// double-precision (sum, sum of squares) per CTA.
// ---------------------------------------------------------------------------
template <typename Real, int K, int BLOCK>
__global__ void __launch_bounds__(BLOCK) timedep_kernel(const __grid_constant__ TimedepParams<Real, K> p)
{
    const int slot = blockIdx.x / p.chunks;
    const int c = blockIdx.x - slot * p.chunks;
    const int j = p.order ? p.order[slot] : slot;
    const int64_t i = (int64_t)c * BLOCK + threadIdx.x;
    const bool active = i < p.M;
    const auto tab = field_table<Real, K>(p);
    double g = 0.0;
    if (active) {
        const ObsRec o = p.obs[j];
        Coord<Real> X1, X2;
        X1.set(o.x1);
        X2.set(o.x2);
        const uint32_t pid = (uint32_t)(p.path_offset + i);
        const int N = o.nsteps;
        const Real h_last = (Real)o.h_last, s_last = (Real)o.s_last;
        for (int n = 0; n < N; n += 2) {
            const u32x4 r = philox4x32_10(u32x4{(uint32_t)(n >> 1), pid, (uint32_t)j, p.inst}, p.key0, p.key1);
            // One copy of the step body (kept rolled): the unrolled velocity sum is
            // ~1000 instructions, and two copies overflow the instruction cache.
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
                const int nn = n + half;
                if (nn >= N) break;
                Real xi1, xi2;
                box_muller<Real>(half ? r.z : r.x, half ? r.w : r.y, xi1, xi2);
                const bool last = (nn == N - 1);
                const Real h = last ? h_last : p.dt;
                const Real s = last ? s_last : p.s_dt;
                Real x1[1] = {X1.val()}, x2[1] = {X2.val()}, v1[1], v2[1];
                velocity<Real, K, 1>(tab, x1, x2, v1, v2);
                em_update<Real>(X1, v1[0], h, s, xi1);
                em_update<Real>(X2, v2[0], h, s, xi2);
                X1.wrap();
                X2.wrap();
            }
        }
        g = theta0_eval(p.th, X1, X2);
        const int64_t w = (int64_t)j * p.M + i;
        if (p.g_out) p.g_out[w] = g;
        if (p.x_out) { p.x_out[2 * w] = X1.full(); p.x_out[2 * w + 1] = X2.full(); }
    }
    const double2 s = block_sum2<BLOCK>(g, g * g);
    if (threadIdx.x == 0) p.part[(int64_t)j * p.chunks + c] = s;
}

// Shared paths (PM_SHARE_PATHS) on the FP32 / FP64 pipes: one CTA = one chunk
// of BLOCK paths of a group of observations at one point; a path runs to the
// group's largest step count and every member takes its own last step from
// the path's position at its step N_j - 1 (same velocity and noise), so each
// member's values equal those of a single-observation call on the group's
// stream.  Members finish at steps every thread of the CTA shares, so the
// per-member CTA sums run inside the step loop.
template <typename Real, int K, int BLOCK>
__global__ void __launch_bounds__(BLOCK) timedep_shared_kernel(const __grid_constant__ TimedepParams<Real, K> p)
{
    const int slot = blockIdx.x / p.chunks;
    const int c = blockIdx.x - slot * p.chunks;
    const int4 G = p.groups[slot];
    const int m1 = G.y;
    const uint32_t stream = (uint32_t)G.z;
    const int64_t i = (int64_t)c * BLOCK + threadIdx.x;
    const bool active = i < p.M;
    const uint32_t pid = (uint32_t)(p.path_offset + (active ? i : 0));
    Coord<Real> X1, X2;
    {
        const ObsRec o = p.obs[p.members[G.x]];
        X1.set(o.x1);
        X2.set(o.x2);
    }
    const auto tab = field_table<Real, K>(p);
    auto finish = [&](int m, const Coord<Real>& Y1, const Coord<Real>& Y2) {
        const int jm = p.members[m];
        double g = 0.0;
        if (active) {
            g = theta0_eval(p.th, Y1, Y2);
            const int64_t w = (int64_t)jm * p.M + i;
            if (p.g_out) p.g_out[w] = g;
            if (p.x_out) { p.x_out[2 * w] = Y1.full(); p.x_out[2 * w + 1] = Y2.full(); }
        }
        const double2 s = block_sum2<BLOCK>(g, g * g);
        if (threadIdx.x == 0) p.part[(int64_t)jm * p.chunks + c] = s;
        __syncthreads();  // block_sum2's scratch is reused by the next member
    };
    auto steps_of = [&](int m) { return m < m1 ? p.obs[p.members[m]].nsteps : -1; };
    int m = G.x;
    while (steps_of(m) == 0) finish(m++, X1, X2);
    const int N = m < m1 ? steps_of(m1 - 1) : 0;
    int stop = steps_of(m) - 1;
    for (int n = 0; n < N; n += 2) {
        const u32x4 r = philox4x32_10(u32x4{(uint32_t)(n >> 1), pid, stream, p.inst}, p.key0, p.key1);
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const int nn = n + half;
            if (nn >= N) break;
            Real xi1, xi2;
            box_muller<Real>(half ? r.z : r.x, half ? r.w : r.y, xi1, xi2);
            Real x1[1] = {X1.val()}, x2[1] = {X2.val()}, v1[1], v2[1];
            velocity<Real, K, 1>(tab, x1, x2, v1, v2);
            while (nn == stop) {
                const ObsRec o = p.obs[p.members[m]];
                Coord<Real> Y1 = X1, Y2 = X2;
                em_update<Real>(Y1, v1[0], (Real)o.h_last, (Real)o.s_last, xi1);
                em_update<Real>(Y2, v2[0], (Real)o.h_last, (Real)o.s_last, xi2);
                Y1.wrap();
                Y2.wrap();
                finish(m++, Y1, Y2);
                stop = steps_of(m) - 1;
            }
            if (nn + 1 < N) {
                em_update<Real>(X1, v1[0], p.dt, p.s_dt, xi1);
                em_update<Real>(X2, v2[0], p.dt, p.s_dt, xi2);
                X1.wrap();
                X2.wrap();
            }
        }
    }
}

template <typename Real, int K>
cudaError_t launch_timedep(const TimedepLaunch& L, cudaStream_t stream)
{
    TimedepParams<Real, K> p;
    constexpr int smem = field_smem<Real, K>();
    if constexpr (K > kMaxUnrolledK) {
        static_assert(sizeof(Real) == 4, "wide K: float paths only");
        // The float table into the caller's device buffer (the host vector is
        // read before the copy call returns).
        if (!L.table_dev) return cudaErrorInvalidValue;
        std::vector<float> h((size_t)table_size(K));
        for (int t = 0; t < table_size(K); ++t) h[(size_t)t] = (float)L.coef[t];
        cudaError_t e = cudaMemcpyAsync(L.table_dev, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return e;
        p.table = reinterpret_cast<const float4*>(L.table_dev);
        e = cudaFuncSetAttribute(L.groups ? timedep_shared_kernel<Real, K, td_simt_rows(K)> : timedep_kernel<Real, K, td_simt_rows(K)>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    } else {
        for (int t = 0; t < table_size(K); ++t) p.field.c[t] = (Real)L.coef[t];
    }
    p.th.n = L.nq;
    for (int q = 0; q < kMaxTheta0; ++q) {
        const bool on = q < L.nq;
        p.th.k1[q] = on ? L.qk[2 * q] : 0;
        p.th.k2[q] = on ? L.qk[2 * q + 1] : 0;
        p.th.a[q] = on ? (Real)L.qa[q] : (Real)0;
        p.th.b[q] = on ? (Real)L.qb[q] : (Real)0;
    }
    p.obs = L.obs;
    p.order = L.order;
    p.part = L.part;
    p.g_out = L.g_out;
    p.x_out = L.x_out;
    p.dt = (Real)L.dt;
    p.s_dt = (Real)L.s_dt;
    p.M = L.M;
    p.path_offset = L.path_offset;
    p.n_obs = L.n_obs;
    p.chunks = L.chunks;
    p.inst = L.inst;
    p.key0 = L.key0;
    p.key1 = L.key1;
    p.groups = L.groups;
    p.members = L.members;
    if (L.groups) {
        const int64_t grid = (int64_t)L.n_groups * L.chunks;
        timedep_shared_kernel<Real, K, td_simt_rows(K)><<<(unsigned)grid, td_simt_rows(K), smem, stream>>>(p);
        return cudaGetLastError();
    }
    const int64_t grid = (int64_t)L.n_obs * L.chunks;
    timedep_kernel<Real, K, td_simt_rows(K)><<<(unsigned)grid, td_simt_rows(K), smem, stream>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Algorithm 2.  Persistent CTAs; every lane owns one path at a time and, when
// it exits, takes the next unclaimed path index from a global counter (one
// atomic per warp per refill, ranks by ballot).  Lanes stay in step-parity
// (refills happen every second step) so one Philox call serves two steps of
// every lane.  Per-path results go to g[pid]; a separate pass reduces them in
// path order, so the estimate does not depend on which lane ran which path.
// ---------------------------------------------------------------------------
template <typename Real, int K>
struct DirichletParams : FieldSource<Real, K> {
    double ga[kMaxBoundary];
    double gb[kMaxBoundary];
    double R, quad, f_const, dt;
    int32_t n_ang;
    Real drift_dt;  // drift_scale * dt
    Real s_dt;      // sqrt(2 kappa dt)
    Real R2hi, R2lo;
    const double* x;
    const int32_t* order;    // [n_obs] observation claimed in slot s, or nullptr
    int64_t n_obs, M, total, max_steps, path_offset;
    unsigned long long* counter;
    unsigned long long* n_unexited;
    unsigned long long* steps;   // total Euler steps taken (all paths)
    double* g;
    int32_t* exit_step;
    double* x_out;
    uint32_t inst, key0, key1;
};

template <typename Real, int K>
__device__ __forceinline__ void dirichlet_finish(const DirichletParams<Real, K>& p, int64_t pid, bool exited,
                                                 int64_t n, const Coord<Real>& X1, const Coord<Real>& X2)
{
    double g = 0.0;
    if (exited) {
        const double y1 = X1.full(), y2 = X2.full();
        const double r = sqrt(y1 * y1 + y2 * y2);
        const double c1 = y1 / r, s1 = y2 / r;           // cos phi, sin phi of the exit point
        const double R = p.R;
        g = p.quad * (R * R) * (c1 * c1 - s1 * s1);       // quad (y1^2 - y2^2) at y = R (c, s)
        double cm = 1.0, sm = 0.0;
        for (int m = 1; m <= p.n_ang; ++m) {               // cos m phi, sin m phi by recurrence
            const double cn = cm * c1 - sm * s1;
            sm = sm * c1 + cm * s1;
            cm = cn;
            g += p.ga[m - 1] * cm + p.gb[m - 1] * sm;
        }
        g -= p.f_const * ((double)n * p.dt);              // left-point integral of constant f
    } else {
        atomicAdd(p.n_unexited, 1ull);
    }
    p.g[pid] = g;
    if (p.exit_step) p.exit_step[pid] = exited ? (int32_t)n : -1;
    if (p.x_out) { p.x_out[2 * pid] = X1.full(); p.x_out[2 * pid + 1] = X2.full(); }
}

template <typename Real, int K>
__global__ void __launch_bounds__(kDirichletBlock) dirichlet_kernel(const __grid_constant__ DirichletParams<Real, K> p)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const auto tab = field_table<Real, K>(p);
    int64_t pid = -1;  // current path (global index j*M + i), -1 = none
    bool done = false;
    int64_t n = 0;
    uint32_t j = 0, i = 0;
    unsigned long long lane_steps = 0;
    Coord<Real> X1, X2;
    X1.set(0.0);
    X2.set(0.0);
    for (;;) {
        // Refill lanes without a path.
        const bool need = !done && pid < 0;
        const unsigned mask = __ballot_sync(full, need);
        if (mask) {
            unsigned long long base = 0;
            const int leader = __ffs(mask) - 1;
            if (lane == leader) base = atomicAdd(p.counter, (unsigned long long)__popc(mask));
            base = __shfl_sync(full, base, leader);
            if (need) {
                const int64_t cand = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
                if (cand < p.total) {
                    // claim order: slots in p.order (longest expected walks first)
                    const int64_t slot = cand / p.M, ii = cand - slot * p.M;
                    j = (uint32_t)(p.order ? (int64_t)p.order[slot] : slot);
                    i = (uint32_t)(ii + p.path_offset);
                    pid = (int64_t)j * p.M + ii;
                    X1.set(p.x[2 * (int64_t)j]);
                    X2.set(p.x[2 * (int64_t)j + 1]);
                    n = 0;
                    if (radial_excess(X1, X2, p.R2hi, p.R2lo) >= (Real)0) {  // starts outside
                        dirichlet_finish(p, pid, true, 0, X1, X2);
                        pid = -1;
                    }
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(full, done)) break;
        if (pid < 0) continue;
        const u32x4 r = philox4x32_10(u32x4{(uint32_t)(n >> 1), i, j, p.inst}, p.key0, p.key1);
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            Real xi1, xi2;
            box_muller<Real>(half ? r.z : r.x, half ? r.w : r.y, xi1, xi2);
            Real x1[1] = {X1.val()}, x2[1] = {X2.val()}, v1[1], v2[1];
            velocity<Real, K, 1>(tab, x1, x2, v1, v2);
            em_update<Real>(X1, v1[0], p.drift_dt, p.s_dt, xi1);
            em_update<Real>(X2, v2[0], p.drift_dt, p.s_dt, xi2);
            ++n;
            const bool exited = radial_excess(X1, X2, p.R2hi, p.R2lo) >= (Real)0;
            if (exited || n >= p.max_steps) {
                dirichlet_finish(p, pid, exited, n, X1, X2);
                lane_steps += (unsigned long long)n;
                pid = -1;
                break;
            }
        }
    }
    if (lane_steps) atomicAdd(p.steps, lane_steps);
}

template <typename Real, int K>
cudaError_t launch_dirichlet(const DirichletLaunch& L, cudaStream_t stream)
{
    DirichletParams<Real, K> p;
    constexpr int smem = field_smem<Real, K>();
    if constexpr (K > kMaxUnrolledK) {
        static_assert(sizeof(Real) == 4, "wide K: float paths only");
        if (!L.table_dev) return cudaErrorInvalidValue;
        std::vector<float> h((size_t)table_size(K));
        for (int t = 0; t < table_size(K); ++t) h[(size_t)t] = (float)L.coef[t];
        cudaError_t e = cudaMemcpyAsync(L.table_dev, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return e;
        p.table = reinterpret_cast<const float4*>(L.table_dev);
        e = cudaFuncSetAttribute(dirichlet_kernel<Real, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    } else {
        for (int t = 0; t < table_size(K); ++t) p.field.c[t] = (Real)L.coef[t];
    }
    for (int m = 0; m < kMaxBoundary; ++m) {
        p.ga[m] = m < L.n_ang ? L.ga[m] : 0.0;
        p.gb[m] = m < L.n_ang ? L.gb[m] : 0.0;
    }
    p.R = L.R;
    p.quad = L.quad;
    p.f_const = L.f_const;
    p.dt = L.dt;
    p.n_ang = L.n_ang;
    p.drift_dt = (Real)(L.drift_scale * L.dt);
    p.s_dt = (Real)L.s_dt;
    const double R2 = L.R * L.R;
    p.R2hi = (Real)R2;
    p.R2lo = (Real)(R2 - (double)p.R2hi);
    p.x = L.x;
    p.order = L.order;
    p.n_obs = L.n_obs;
    p.M = L.M;
    p.total = L.n_obs * L.M;
    p.max_steps = L.max_steps;
    p.path_offset = L.path_offset;
    p.counter = L.counter;
    p.n_unexited = L.n_unexited;
    p.steps = L.steps;
    p.g = L.g;
    p.exit_step = L.exit_step;
    p.x_out = L.x_out;
    p.inst = L.inst;
    p.key0 = L.key0;
    p.key1 = L.key1;
    dirichlet_kernel<Real, K><<<L.grid, kDirichletBlock, smem, stream>>>(p);
    return cudaGetLastError();
}

template <typename Real, int K>
int dirichlet_blocks_per_sm()
{
    constexpr int smem = field_smem<Real, K>();
    if constexpr (smem > 0) {
        if (cudaFuncSetAttribute(dirichlet_kernel<Real, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return 1;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dirichlet_kernel<Real, K>, kDirichletBlock, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

// ---------------------------------------------------------------------------
// Velocity at given points with the particle step's own device code.
// ---------------------------------------------------------------------------
template <typename Real, int K>
struct VelocityParams {
    FieldTable<Real, K> field;
    const double* x;
    double* v;
    int64_t n;
};

template <typename Real, int K>
__global__ void __launch_bounds__(128) velocity_kernel(const __grid_constant__ VelocityParams<Real, K> p)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= p.n) return;
    const ParamTable<Real, K> tab{p.field};
    Coord<Real> X1, X2;
    X1.set(p.x[2 * q]);
    X2.set(p.x[2 * q + 1]);
    Real x1[1] = {X1.val()}, x2[1] = {X2.val()}, v1[1], v2[1];
    velocity<Real, K, 1>(tab, x1, x2, v1, v2);
    p.v[2 * q] = (double)v1[0];
    p.v[2 * q + 1] = (double)v2[0];
}

template <typename Real, int K>
cudaError_t launch_velocity(const double* coef, const double* x, int64_t n, double* v, cudaStream_t stream)
{
    VelocityParams<Real, K> p;
    for (int t = 0; t < table_size(K); ++t) p.field.c[t] = (Real)coef[t];
    p.x = x;
    p.v = v;
    p.n = n;
    const int64_t grid = (n + 127) / 128;
    velocity_kernel<Real, K><<<(unsigned)grid, 128, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace pm

// Wide K: the time-dependent and Dirichlet maps (float paths).
#define PM_INSTANTIATE_WIDE(K)                                                                     \
    template cudaError_t pm::launch_timedep<float, K>(const pm::TimedepLaunch&, cudaStream_t);     \
    template cudaError_t pm::launch_dirichlet<float, K>(const pm::DirichletLaunch&, cudaStream_t); \
    template int pm::dirichlet_blocks_per_sm<float, K>();

// Explicit instantiation of the launchers for one precision and one K.
#define PM_INSTANTIATE(Real, K)                                                                        \
    template cudaError_t pm::launch_timedep<Real, K>(const pm::TimedepLaunch&, cudaStream_t);          \
    template cudaError_t pm::launch_dirichlet<Real, K>(const pm::DirichletLaunch&, cudaStream_t);      \
    template cudaError_t pm::launch_velocity<Real, K>(const double*, const double*, int64_t, double*, \
                                                       cudaStream_t);                                 \
    template int pm::dirichlet_blocks_per_sm<Real, K>();
