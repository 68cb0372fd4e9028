// pm_batched.cuh -- one persistent launch over many parameter samples u_b, each
// a time-dependent (Algorithm 1) or Dirichlet (Algorithm 2) instance with its
// own observations, path count and step size.
//
// Work distribution.  Every lane owns one path at a time.  Lanes of a warp
// take new paths of the warp's current instance from that instance's path
// counter (one atomic per warp per refill), so paths of uneven length keep the
// lanes busy.  The instance's velocity table sits in the warp's slice of
// shared memory; a warp moves to another instance only when its instance has
// no unclaimed paths left (then it drains, reloads the table, and goes on).
// Per-path results are stored by path index, so the estimates do not depend
// on which lane or warp ran which path.
#pragma once
#include "pm_kernels.cuh"

namespace pm {

constexpr int kBatchWarps = 4;  // warps per CTA of the batched kernel

// Boundary functional of Algorithm 2 at the exit point (radial projection).
__device__ __forceinline__ double boundary_value(const double* ga, const double* gb, int n_ang, double R, double quad,
                                                 double y1, double y2)
{
    const double r = sqrt(y1 * y1 + y2 * y2);
    const double c1 = y1 / r, s1 = y2 / r;
    double g = quad * (R * R) * (c1 * c1 - s1 * s1);
    double cm = 1.0, sm = 0.0;
    for (int m = 1; m <= n_ang; ++m) {
        const double cn = cm * c1 - sm * s1;
        sm = sm * c1 + cm * s1;
        cm = cn;
        g += ga[m - 1] * cm + gb[m - 1] * sm;
    }
    return g;
}

template <int K>
__global__ void __launch_bounds__(kBatchWarps * 32) batched_kernel(const __grid_constant__ BatchKernelParams p)
{
    constexpr int TS = table_size(K);
    extern __shared__ __align__(16) float s_tab_all[];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* s_tab = s_tab_all + warp * TS;
    const SharedTable tab{reinterpret_cast<const float4*>(s_tab)};

    const int gw = blockIdx.x * kBatchWarps + warp, nw = gridDim.x * kBatchWarps;
    int b = (int)(((long long)gw * p.B) / nw);   // spread warps over the instances
    bool have_inst = false;
    BatchInstDev I{};
    float s_dt = 0.f, drift_dt = 0.f, dt = 0.f;

    int64_t pid = -1;      // path index within the instance
    int64_t n = 0;
    int32_t N = 0;         // time-dependent: step count of the path's observation
    float h_last = 0.f, s_last = 0.f;
    uint32_t j = 0, i = 0;
    Coord<float> X1, X2;
    X1.set(0.0);
    X2.set(0.0);
    unsigned long long lane_steps = 0;

    bool exhausted = true;  // no unclaimed paths left in the warp's instance (warp-uniform)
    for (;;) {
        // ---- refill idle lanes from the current instance ------------------------
        if (!exhausted) {
            const bool need = pid < 0;
            const unsigned mask = __ballot_sync(full, need);
            if (mask) {
                unsigned long long base = 0;
                const int leader = __ffs(mask) - 1;
                if (lane == leader) base = atomicAdd(&p.next_path[b], (unsigned long long)__popc(mask));
                base = __shfl_sync(full, base, leader);
                if ((int64_t)(base + __popc(mask)) >= I.n_paths) exhausted = true;
                if (need) {
                    const int64_t cand = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
                    if (cand < I.n_paths) {
                        pid = cand;
                        j = (uint32_t)(cand / I.M);
                        i = (uint32_t)(cand - (int64_t)j * I.M);
                        const RowRec rr = p.rows[I.row0 + j];
                        X1.set(rr.x1);
                        X2.set(rr.x2);
                        n = 0;
                        N = rr.nsteps;
                        h_last = (float)rr.h_last;
                        s_last = (float)rr.s_last;
                        if (I.kind == 0 && N == 0) {                       // t_j = 0: theta0(x_j)
                            p.g[I.path_base + pid] = theta0_eval(p.th, X1, X2);
                            pid = -1;
                        } else if (I.kind == 1 && radial_excess(X1, X2, p.R2hi, p.R2lo) >= 0.f) {
                            p.g[I.path_base + pid] =
                                boundary_value(p.ga, p.gb, p.n_ang, p.R, p.quad, X1.full(), X2.full());
                            pid = -1;
                        }
                    }
                }
            }
        }
        // ---- every lane idle: continue this instance or move to another ----------
        if (__ballot_sync(full, pid >= 0) == 0) {
            if (!exhausted) continue;  // lanes finished at once (t = 0 or started outside): refill
            int found = -1;
            const int start = have_inst ? b + 1 : b;
            for (int base = 0; base < p.B && found < 0; base += 32) {
                const int q = base + lane;
                bool ok = false;
                int cand_b = 0;
                if (q < p.B) {
                    cand_b = (start + q) % p.B;
                    ok = (int64_t)(*(volatile unsigned long long*)&p.next_path[cand_b]) < p.inst[cand_b].n_paths;
                }
                const unsigned m2 = __ballot_sync(full, ok);
                if (m2) found = __shfl_sync(full, cand_b, __ffs(m2) - 1);
            }
            if (found < 0) break;  // nothing left anywhere: this warp is done
            // (lane step counts are flushed after the loop)
            b = found;
            I = p.inst[b];
            have_inst = true;
            exhausted = false;
            dt = (float)I.dt;
            s_dt = (float)sqrt(2.0 * I.kappa * I.dt);
            drift_dt = (float)(I.drift_scale * I.dt);
            __syncwarp();
            const float4* src = reinterpret_cast<const float4*>(p.tables + (size_t)b * TS);
            float4* dst = reinterpret_cast<float4*>(s_tab);
            for (int q = lane; q < TS / 4; q += 32) dst[q] = src[q];
            __syncwarp();
            continue;
        }
        if (pid < 0) continue;

        // ---- two Euler steps per Philox call ----------------------------------
        const u32x4 r = philox4x32_10(u32x4{(uint32_t)(n >> 1), i, j, I.stream}, I.key0, I.key1);
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            asm volatile("" ::: "memory");  // keeps the table loads inside the step
            float xi1, xi2;
            box_muller<float>(half ? r.z : r.x, half ? r.w : r.y, xi1, xi2);
            float x1[1] = {X1.val()}, x2[1] = {X2.val()}, v1[1], v2[1];
            velocity<float, K, 1>(tab, x1, x2, v1, v2);
            if (I.kind == 0) {
                const bool last = (n == N - 1);
                const float h = last ? h_last : dt, s = last ? s_last : s_dt;
                em_update<float>(X1, v1[0], h, s, xi1);
                em_update<float>(X2, v2[0], h, s, xi2);
                X1.wrap();
                X2.wrap();
                ++n;
                if (n >= N) {
                    p.g[I.path_base + pid] = theta0_eval(p.th, X1, X2);
                    lane_steps += (unsigned long long)n;
                    pid = -1;
                    break;
                }
            } else {
                em_update<float>(X1, v1[0], drift_dt, s_dt, xi1);
                em_update<float>(X2, v2[0], drift_dt, s_dt, xi2);
                ++n;
                const bool exited = radial_excess(X1, X2, p.R2hi, p.R2lo) >= 0.f;
                if (exited || n >= I.max_steps) {
                    double gv = 0.0;
                    if (exited) gv = boundary_value(p.ga, p.gb, p.n_ang, p.R, p.quad, X1.full(), X2.full()) -
                                     p.f_const * ((double)n * I.dt);
                    else atomicAdd(p.n_unexited, 1ull);
                    p.g[I.path_base + pid] = gv;
                    lane_steps += (unsigned long long)n;
                    pid = -1;
                    break;
                }
            }
        }
    }
    if (lane_steps) atomicAdd(p.steps, lane_steps);
}

// The dynamic shared-memory attribute is set by batched_blocks_per_sm, which
// the host calls before every launch (outside any stream capture).
template <int K>
cudaError_t launch_batched(const BatchKernelParams& p, int grid, cudaStream_t s)
{
    const size_t smem = (size_t)kBatchWarps * table_size(K) * sizeof(float);
    batched_kernel<K><<<grid, kBatchWarps * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int K>
int batched_blocks_per_sm()
{
    int nb = 0;
    const size_t smem = (size_t)kBatchWarps * table_size(K) * sizeof(float);
    cudaFuncSetAttribute(batched_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_kernel<K>, kBatchWarps * 32, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace pm

#define PM_INSTANTIATE_BATCHED(K)                                                                     \
    template cudaError_t pm::launch_batched<K>(const pm::BatchKernelParams&, int, cudaStream_t);        \
    template int pm::batched_blocks_per_sm<K>();
