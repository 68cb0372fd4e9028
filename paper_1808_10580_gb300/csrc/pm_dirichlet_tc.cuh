// pm_dirichlet_tc.cuh -- Algorithm 2 (walks to the first exit from the disk)
// with the velocity sum on the tensor cores, in a persistent kernel.
//
// Same per-lane refill as dirichlet_kernel (each lane takes the next unclaimed
// path as soon as its path exits; one atomic per warp per refill), but the 128
// lanes of a CTA step together: every Euler step is one CTA-wide matrix
// product of the lanes' x2 harmonics with the coefficient matrix (see
// pm_timedep_tc.cuh), so a lane without a path still supplies a row (whose
// result is ignored).  The CTA leaves when every lane has found the path
// counter exhausted.
#pragma once
#include <type_traits>
#include "pm_general_step.cuh"
#include "pm_timedep_tc.cuh"

namespace pm {
namespace tdtc {

// Wide K (above the unrolled bound) takes the time-dependent kernel's folded
// shape where that kernel folds (it keeps N within one MMA at K = 64), and
// reads W from global memory.
template <int K>
using DirShape = Shape<K, (K > kMaxUnrolledK) && fold_of<K>(), half_of<K>()>;

template <int K>
struct DirParams {
    // W^T (see build_W): in the parameter bank, or at Wg.
    float W[DirShape<K>::W_PARAM ? DirShape<K>::NP * DirShape<K>::WS : 1];
    const float* Wg;
    // Folded shape: the m = 0 terms of v1 and the n = 0 terms of v2 on the
    // FP32 pipes (the layout of Params<K>::T0 and N0).
    alignas(8) float T0[2 * K + 2];
    alignas(8) float N0[2 * K + 2];
    float inv_s;  // FP16 operands: 1 / (power-of-two scale of W)
    double ga[kMaxBoundary];
    double gb[kMaxBoundary];
    double R, quad, f_const, dt;
    int32_t n_ang;
    float drift_dt, s_dt, R2hi, R2lo;
    float band;              // exits_disk: 2^-16 R2hi
    const double* x;
    const int32_t* order;    // [n_obs] observation claimed in slot s, or nullptr
    int64_t n_obs, M, total, max_steps, path_offset;
    unsigned long long* counter;
    unsigned long long* n_unexited;
    unsigned long long* steps;
    double* g;
    int32_t* exit_step;
    double* x_out;
    uint32_t inst, key0, key1;
    uint32_t rk[20];      // Philox round keys of (key0, key1)
    unsigned* err;
    uint32_t wait_limit;  // polls of the per-step MMA wait (tc::kWaitLimit unless a test lowers it)
    int32_t refill_pairs; // pairs of Euler steps between lane refills (a launch shape: results do not depend on it)
    GeneralCoef<float> gc;  // the general map (kernel's GEN): sigma(x), Milstein, forcing
};

// integral: the path's int f (f_const n dt, or the general map's left-point sum)
template <int K>
__device__ __forceinline__ void dir_finish(const DirParams<K>& p, int64_t pid, bool exited, int64_t n,
                                           const Coord<float>& X1, const Coord<float>& X2, double integral)
{
    double g = 0.0;
    if (exited) {
        const double y1 = X1.full(), y2 = X2.full();
        const double rr = sqrt(y1 * y1 + y2 * y2);
        const double c1 = y1 / rr, s1 = y2 / rr;
        g = p.quad * (p.R * p.R) * (c1 * c1 - s1 * s1);
        double cm = 1.0, sm = 0.0;
        for (int m = 1; m <= p.n_ang; ++m) {
            const double cn = cm * c1 - sm * s1;
            sm = sm * c1 + cm * s1;
            cm = cn;
            g += p.ga[m - 1] * cm + p.gb[m - 1] * sm;
        }
        g -= integral;
    } else {
        atomicAdd(p.n_unexited, 1ull);
    }
    p.g[pid] = g;
    if (p.exit_step) p.exit_step[pid] = exited ? (int32_t)n : -1;
    if (p.x_out) { p.x_out[2 * pid] = X1.full(); p.x_out[2 * pid + 1] = X2.full(); }
}

// GEN: the general map (state-dependent diffusion with the Milstein term,
// Gaussian-source forcing; pm_general_step.cuh) instead of the constant
// diffusion and forcing; the velocity sum is the same.
// LIMIT: the per-step MMA wait takes the launch's poll limit (a test lowered
// it, pm_set_wait_limit); otherwise the compile-time full bound, with no
// per-step test of the setting.
template <int K, bool GEN = false, bool LIMIT = false>
__global__ void __launch_bounds__(128, DirShape<K>::MIN_CTAS) dirichlet_tc_kernel(const __grid_constant__ DirParams<K> p)
{
    using S = DirShape<K>;
    constexpr bool F = S::FOLD;
    constexpr bool H = S::HALF;
    // x1 harmonics streamed after the MMA wait (as in the time-dependent
    // kernel): 64 registers and 8 CTAs per SM at K = 10, 388.5 against 395.9 ms
    // on the disk workload with all of them computed during the product at 6.
    using Harm1 = HarmStream;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint8_t* A_hi = smem;
    uint8_t* A_lo = smem + S::A_BYTES;
    uint8_t* B_hi = smem + 2 * S::A_BYTES;
    uint8_t* B_lo = B_hi + S::B_BYTES;
    uint64_t* bar = (uint64_t*)(B_lo + S::B_BYTES);
    uint32_t* tmem_slot = (uint32_t*)(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned full = 0xffffffffu;
    const uint32_t bar_a = tc::smem_u32(bar);

    if constexpr (S::W_PARAM) stage_B<S>(B_hi, B_lo, tid, [&](int q) { return p.W[q]; });
    else stage_B<S>(B_hi, B_lo, tid, [&](int q) { return __ldg(p.Wg + q); });
    for (int c = 0; c < S::KC; ++c) {
        *reinterpret_cast<float4*>(A_hi + tile_off<S::KC>(tid, c)) = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(A_lo + tile_off<S::KC>(tid, c)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (tid == 0) {
        tc::mbar_init(bar_a, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                     "r"(S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);

    const uint32_t row = tile_off<S::KC>(tid, 0);
    const uint32_t sb = tc::smem_u32(A_hi);  // A_hi, A_lo, B_hi, B_lo back to back
    int64_t pid = -1;
    bool done = false;
    int32_t n = 0;  // steps of the lane's path (max_steps < 2^31)
    const int32_t max_steps = (int32_t)p.max_steps;
    uint32_t j = 0, i = 0;
    unsigned long long lane_steps = 0;
    uint32_t phase = 0;
    bool issued_any = false;  // a product has been issued (its parity is phase ^ 1 after the flip)
    bool failed = false, stop = false;
    Coord<float> X1, X2;
    X1.set(0.0);
    X2.set(0.0);
    ForcingSum<float> fs;  // the general map's forcing sum (GEN)

    // 2 refill_pairs Euler steps (a lane whose path exits waits for the next
    // refill; the RNG stays keyed by the step index).  Warps without a path
    // at the start take no part in the step's work but the barrier and the
    // phase (their rows of A keep old values, whose products nobody reads).
    auto run_interval = [&]() {
        const bool on = __any_sync(full, pid >= 0);
#pragma unroll 1
        for (int pair = 0; pair < p.refill_pairs && !stop; ++pair) {
            float2 z1, z2;  // the two steps' normals, formed during the first product
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
                float2 sx = make_float2(0.f, 0.f), cx = sx;
                float p0 = 0.f;
                if (on) {
                    sincos_turns2(make_float2(X1.val(), X2.val()), sx, cx);
                    p0 = write_row_stream<K, F, H>(sb + row, (uint32_t)S::A_BYTES, sx.y, cx.y, p.T0);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                // One barrier per step: the rows are in place, and a wait that gave
                // up in the previous step (any thread) stops the whole CTA.
                if (__syncthreads_or(failed)) { stop = true; break; }
                if (tid == 0) issue_step_mma<K, F, H>(tmem, sb, bar_a);
                issued_any = true;
                if (!on) {
                    phase ^= 1u;
                    continue;
                }
                // While the product runs: the Brownian increment and the x1 harmonics.
                if (half == 0) {
                    u32x4 r{0, 0, 0, 0};
                    if (pid >= 0) r = philox4x32_10_rk(u32x4{(uint32_t)(n >> 1), i, j, p.inst}, p.rk);
                    box_muller2(r.x, r.y, r.z, r.w, z1, z2);
                }
                const float xi1 = half ? z1.y : z1.x, xi2 = half ? z2.y : z2.x;
                Harm1 h1;  // its base from x1; the harmonics follow in the velocity sum
                h1.init(sx.x, cx.x);
                if constexpr (LIMIT) failed = !tc::mbar_wait(bar_a, phase, p.wait_limit);
                else failed = !tc::mbar_wait(bar_a, phase);
                phase ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float v1, v2;
                velocity_stream<K, F, H>(t_row, h1, p.N0, p0, p.inv_s, v1, v2);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                if (pid >= 0) {
                    if constexpr (GEN) {
                        const float x1v = X1.val(), x2v = X2.val();  // the step's start point
                        fs.add(p.gc.forcing(x1v, x2v));
                        X1.add(p.gc.increment(0, x1v, v1, p.drift_dt, xi1));
                        X2.add(p.gc.increment(1, x2v, v2, p.drift_dt, xi2));
                    } else {
                        em_update2(X1, X2, v1, v2, p.drift_dt, p.s_dt, xi1, xi2);
                    }
                    ++n;
                    const bool exited = exits_disk(X1, X2, p.R2hi, p.R2lo, p.band);
                    if (exited || n >= max_steps) {
                        dir_finish(p, pid, exited, n, X1, X2,
                                   GEN ? fs.value() * p.dt : p.f_const * ((double)n * p.dt));
                        lane_steps += (unsigned long long)n;
                        pid = -1;
                    }
                }
            }
        }
    };

    // Moves the CTA's `active` paths to lanes 0 .. active - 1 (in lane order)
    // through the A tiles, when that leaves fewer warps with a path; no
    // product is in flight here (every thread has waited for the last one).
    // The tiles' rows are cleared again afterwards (zero padding columns).
    auto compact_paths = [&](int active) {
        const unsigned bal = __ballot_sync(full, pid >= 0);
        const int warps_on = __syncthreads_count(lane == 0 && bal != 0u);
        if ((active + 31) / 32 >= warps_on) return;
        int* wc = reinterpret_cast<int*>(B_lo + S::B_BYTES) + 8;  // 4 ints after the barrier words
        if (lane == 0) wc[warp] = __popc(bal);
        __syncthreads();
        uint32_t* slot = reinterpret_cast<uint32_t*>(A_hi);  // 12 words per path
        if (pid >= 0) {
            int rank = __popc(bal & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) rank += wc[w];
            uint32_t* q = slot + 12 * rank;
            q[0] = j;
            q[1] = i;
            q[2] = (uint32_t)n;
            q[3] = (uint32_t)(uint64_t)pid;
            q[4] = (uint32_t)((uint64_t)pid >> 32);
            q[5] = __float_as_uint(X1.hi);
            q[6] = __float_as_uint(X1.lo);
            q[7] = __float_as_uint(X2.hi);
            q[8] = __float_as_uint(X2.lo);
            q[9] = __float_as_uint(fs.s);
            q[10] = __float_as_uint(fs.c);
        }
        __syncthreads();
        pid = -1;
        if (tid < active) {
            const uint32_t* q = slot + 12 * tid;
            j = q[0];
            i = q[1];
            n = (int32_t)q[2];
            pid = (int64_t)(((uint64_t)q[4] << 32) | q[3]);
            X1.hi = __uint_as_float(q[5]);
            X1.lo = __uint_as_float(q[6]);
            X2.hi = __uint_as_float(q[7]);
            X2.lo = __uint_as_float(q[8]);
            fs.s = __uint_as_float(q[9]);
            fs.c = __uint_as_float(q[10]);
        }
        __syncthreads();
        for (int c = 0; c < S::KC; ++c) {
            *reinterpret_cast<float4*>(A_hi + tile_off<S::KC>(tid, c)) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(A_lo + tile_off<S::KC>(tid, c)) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    };
    static_assert(12 * 4 * 128 <= 2 * S::A_BYTES, "the exchange fits the A tiles");

    for (;;) {
        // Refill (per warp).
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
                    fs = ForcingSum<float>{};
                    if (radial_excess(X1, X2, p.R2hi, p.R2lo) >= 0.f) {  // starts outside
                        dir_finish(p, pid, true, 0, X1, X2, 0.0);
                        pid = -1;
                    }
                } else {
                    done = true;
                }
            }
        }
        // Leave when every lane of the CTA is out of work; step while any lane has a path.
        const int active = __syncthreads_count(pid >= 0);
        if (active == 0) {
            if (__syncthreads_and(done)) break;
            continue;
        }
        // The tail: with at most three warps' worth of paths left and the path
        // counter exhausted (no lane is refilled again), move the paths to the
        // lowest lanes when that empties a warp, and let warps without a path
        // skip the step's work.  A path's state moves whole and its random
        // numbers are keyed by its own step index: every result is unchanged.
        if (active <= 96 && __syncthreads_or(done)) compact_paths(active);
        run_interval();
        if (stop) break;
    }
    if (failed) atomicExch(p.err, 1u);
    if (lane_steps) atomicAdd(p.steps, lane_steps);
    // No product may still write tensor memory when it is freed: after a wait
    // that gave up (stop), wait (full bound) for the last one issued.
    if (stop && issued_any) tc::mbar_wait(bar_a, phase ^ 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS) : "memory");
    }
}

template <int K>
cudaError_t launch_dirichlet_tc(const DirichletLaunch& L, unsigned* err, cudaStream_t stream)
{
    using S = DirShape<K>;
    DirParams<K> p;
    p.Wg = nullptr;
    for (int q = 0; q < 2 * K + 2; ++q) p.T0[q] = p.N0[q] = 0.f;
    if constexpr (S::FOLD) {
        auto T = [&](int m, int n, int q) { return L.coef[(size_t)(m * (K + 1) + n) * 8 + q]; };
        for (int n = 1; n <= K; ++n) {
            p.T0[n - 1] = (float)T(0, n, 0);
            p.T0[K + n - 1] = (float)T(0, n, 1);
            p.N0[n - 1] = (float)T(n, 0, 4);
            p.N0[K + n - 1] = (float)T(n, 0, 6);
        }
    }
    std::vector<float> Wv((size_t)(S::NP * S::WS));
    build_W<K, S::FOLD, S::HALF>(L.coef, Wv.data());
    p.inv_s = scale_W_host<S>(Wv.data(), p.N0, S::FOLD ? 2 * K : 0);
    if constexpr (S::W_PARAM) {
        for (size_t q = 0; q < Wv.size(); ++q) p.W[q] = Wv[q];
    } else {
        // into the caller's device buffer (the host vector is read before the copy call returns)
        if (!L.table_dev) return cudaErrorInvalidValue;
        const cudaError_t e = cudaMemcpyAsync(L.table_dev, Wv.data(), Wv.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return e;
        p.Wg = L.table_dev;
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
    p.drift_dt = (float)(L.drift_scale * L.dt);
    p.s_dt = (float)L.s_dt;
    const double R2 = L.R * L.R;
    p.R2hi = (float)R2;
    p.R2lo = (float)(R2 - (double)p.R2hi);
    p.band = std::ldexp(p.R2hi, -16);
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
    round_keys(L.key0, L.key1, p.rk);
    p.err = err;
    p.wait_limit = L.wait_limit;
    const bool limited = L.wait_limit < tc::kWaitLimit;
    p.refill_pairs = L.refill_pairs > 0 ? L.refill_pairs : 1;
    p.gc = GeneralCoef<float>{};
    if (L.gen) {  // the general map
        p.gc.set(*L.gen, L.dt, L.f_const);
        cudaError_t e = cudaFuncSetAttribute(limited ? dirichlet_tc_kernel<K, true, true> : dirichlet_tc_kernel<K, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        if (e != cudaSuccess) return e;
        if (limited) dirichlet_tc_kernel<K, true, true><<<L.grid, 128, S::SMEM, stream>>>(p);
        else dirichlet_tc_kernel<K, true><<<L.grid, 128, S::SMEM, stream>>>(p);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(limited ? dirichlet_tc_kernel<K, false, true> : dirichlet_tc_kernel<K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    if (limited) dirichlet_tc_kernel<K, false, true><<<L.grid, 128, S::SMEM, stream>>>(p);
    else dirichlet_tc_kernel<K><<<L.grid, 128, S::SMEM, stream>>>(p);
    return cudaGetLastError();
}

// Resident CTAs per SM of the kernel (gen: the general map's variant); also
// sets its dynamic shared-memory limit.
template <int K>
int dirichlet_tc_blocks_per_sm(bool gen)
{
    using S = DirShape<K>;
    if (gen) {
        cudaFuncSetAttribute(dirichlet_tc_kernel<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        return resident_ctas((const void*)dirichlet_tc_kernel<K, true>, 128, S::SMEM, (int)S::TMEM_COLS);
    }
    cudaFuncSetAttribute(dirichlet_tc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    return resident_ctas((const void*)dirichlet_tc_kernel<K>, 128, S::SMEM, (int)S::TMEM_COLS);
}

}  // namespace tdtc
}  // namespace pm

#define PM_INSTANTIATE_DIR_TC(K)                                                                                 \
    template cudaError_t pm::tdtc::launch_dirichlet_tc<K>(const pm::DirichletLaunch&, unsigned*, cudaStream_t); \
    template int pm::tdtc::dirichlet_tc_blocks_per_sm<K>(bool);
