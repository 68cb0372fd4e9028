// pm_batched_tc.cuh -- the batched persistent map (many instances u_b, mixed
// time-dependent and Dirichlet) with the velocity sum on the tensor cores.
//
// A CTA works on one instance at a time: that instance's coefficient matrix
// W_b is the B operand of the per-step MMA (see pm_timedep_tc.cuh), kept as
// hi / lo tiles (TF32, or FP16 with a per-instance power-of-two scale) in
// shared memory.  Its lanes take paths of the instance
// from the instance's path counter (one atomic per warp per refill) and step
// together; when the instance has no unclaimed paths left and every lane of
// the CTA has finished, the CTA moves to the next instance with work and
// rebuilds its tiles.  Results are stored per path, so the estimates do not
// depend on which CTA ran which path.
#pragma once
#include <type_traits>
#include "pm_batched.cuh"
#include "pm_timedep_tc.cuh"

namespace pm {
namespace tdtc {

// Entry W[k][nc] of the coefficient matrix from the product-basis table
// tab[(m (K+1) + n) 8 + q] (e0..e3, f0..f3): A column k holds S2_n
// (k = 2(n-1)), C2_n (k = 2(n-1)+1) or, unfolded, the constant 1 (k = 2K);
// accumulator column pcol(m, j) holds P1c, P1s, P2c, P2s (j = 0..3) of m and,
// unfolded, column p0col(K) P(0) (the layout of build_W).  The folded shape
// leaves the constant column and P(0) to the FP32 pipes.
template <int K, bool F = false>
__device__ __forceinline__ float w_entry(const float* tab, int nc, int k)
{
    int n = 0, type = 0;  // type 0: S2_n, 1: C2_n, 2: constant
    if (k < 2 * K) { n = k / 2 + 1; type = k & 1; }
    else if (!F && k == 2 * K) { type = 2; }
    else return 0.f;
    auto T = [&](int m, int nn, int q) { return tab[(m * (K + 1) + nn) * 8 + q]; };
    if (!F && nc == p0col(K)) return type == 0 ? T(0, n, 0) : type == 1 ? T(0, n, 1) : 0.f;  // P(0)
    if (nc >= p0col(K)) return 0.f;
    const int r = nc % 8, j = r / 2, m = 2 * (nc / 8) + 1 + (r & 1);  // inverse of pcol
    if (m > K) return 0.f;
    if (j == 0) return type == 0 ? T(m, n, 0) : type == 1 ? T(m, n, 1) : 0.f;          // P1c
    if (j == 1) return type == 0 ? T(m, n, 2) : type == 1 ? T(m, n, 3) : 0.f;          // P1s
    if (j == 2) return type == 1 ? T(m, n, 4) : type == 0 ? T(m, n, 5) : T(m, 0, 4);   // P2c
    return type == 1 ? T(m, n, 6) : type == 0 ? T(m, n, 7) : T(m, 0, 6);               // P2s
}

// Wide K: the folded shape where the time-dependent kernel folds (N within
// one MMA at K = 64), as in the Dirichlet kernel.
template <int K>
using BatShape = Shape<K, (K > kMaxUnrolledK) && fold_of<K>(), half_of<K>()>;

template <int K>
__global__ void __launch_bounds__(128, BatShape<K>::MIN_CTAS6) batched_tc_kernel(const __grid_constant__ BatchKernelParams p)
{
    using S = BatShape<K>;
    constexpr bool F = S::FOLD;
    constexpr bool H = S::HALF;
    // x1 harmonics: all of them during the product up to the unrolled bound,
    // streamed after the wait above it (registers).
    using Harm1 = std::conditional_t<(K > kMaxUnrolledK), HarmStream, HarmArray<K>>;
    constexpr int TS = table_size(K);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint8_t* A_hi = smem;
    uint8_t* A_lo = smem + S::A_BYTES;
    uint8_t* B_hi = smem + 2 * S::A_BYTES;
    uint8_t* B_lo = B_hi + S::B_BYTES;
    uint64_t* bar = (uint64_t*)(B_lo + S::B_BYTES);
    uint32_t* tmem_slot = (uint32_t*)(bar + 1);
    int* s_next = (int*)(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned full = 0xffffffffu;
    const uint32_t bar_a = tc::smem_u32(bar);

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

    int b = (int)(((long long)blockIdx.x * p.B) / gridDim.x);  // spread CTAs over the instances
    bool have_inst = false;
    bool exhausted = true;  // warp-uniform: no unclaimed paths left in b for this warp
    // The CTA's current instance lives in shared memory; only the fields the
    // step loop reads every step stay in registers.
    __shared__ BatchInstDev sI;
    __shared__ int s_wmax;  // FP16 operands: bits of max |table entry| of the instance
    // Folded shape: the instance's m = 0 terms of v1 and (scaled with W) n = 0
    // terms of v2, in the layout of Params<K>::T0 and N0.
    __shared__ __align__(8) float sT0[F ? 2 * K : 2];
    __shared__ __align__(8) float sN0[F ? 2 * K : 2];
    float inv_s = 1.f;      // FP16 operands: 1 / (power-of-two scale of W)
    int kind = 0;
    uint32_t stream = 0, key0 = 0, key1 = 0;
    float s_dt = 0.f, drift_dt = 0.f, dt = 0.f;
    int64_t pid = -1;
    int32_t n = 0, N = 0;  // steps taken and step count of the lane's path (max_steps < 2^31)
    float h_last = 0.f, s_last = 0.f;
    uint32_t j = 0, i = 0;
    unsigned long long lane_steps = 0;
    uint32_t phase = 0;
    bool issued_any = false;  // a product has been issued (its parity is phase ^ 1 after the flip)
    bool failed = false, stop = false;
    Coord<float> X1, X2;
    X1.set(0.0);
    X2.set(0.0);

    for (;;) {
        // ---- refill idle lanes of this warp from the CTA's instance --------------
        if (!exhausted) {
            const bool need = pid < 0;
            const unsigned mask = __ballot_sync(full, need);
            if (mask) {
                unsigned long long base = 0;
                const int leader = __ffs(mask) - 1;
                if (lane == leader) base = atomicAdd(&p.next_path[b], (unsigned long long)__popc(mask));
                base = __shfl_sync(full, base, leader);
                if ((int64_t)(base + __popc(mask)) >= sI.n_paths) exhausted = true;
                if (need) {
                    const int64_t cand = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
                    if (cand < sI.n_paths) {
                        pid = cand;
                        const int64_t Mi = sI.M;
                        j = (uint32_t)(cand / Mi);
                        i = (uint32_t)(cand - (int64_t)j * Mi);
                        const RowRec rr = p.rows[sI.row0 + j];
                        X1.set(rr.x1);
                        X2.set(rr.x2);
                        n = 0;
                        N = rr.nsteps;
                        h_last = (float)rr.h_last;
                        s_last = (float)rr.s_last;
                        if (kind == 0 && N == 0) {
                            p.g[sI.path_base + pid] = theta0_eval(p.th, X1, X2);
                            pid = -1;
                        } else if (kind == 1 && radial_excess(X1, X2, p.R2hi, p.R2lo) >= 0.f) {
                            p.g[sI.path_base + pid] =
                                boundary_value(p.ga, p.gb, p.n_ang, p.R, p.quad, X1.full(), X2.full());
                            pid = -1;
                        }
                    }
                }
            }
        }
        // ---- no lane of the CTA has a path: refill again, or change instance ------
        if (!__syncthreads_or(pid >= 0)) {
            if (!__syncthreads_and(exhausted)) continue;
            if (warp == 0) {
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
                if (lane == 0) *s_next = found;
                if (lane == 0) s_wmax = 0;
            }
            __syncthreads();
            const int found = *s_next;
            if (found < 0) break;
            b = found;
            if (tid == 0) sI = p.inst[b];  // visible after the barrier below
            const BatchInstDev& In = p.inst[b];
            have_inst = true;
            exhausted = false;
            kind = In.kind;
            stream = In.stream;
            key0 = In.key0;
            key1 = In.key1;
            dt = (float)In.dt;
            s_dt = (float)sqrt(2.0 * In.kappa * In.dt);
            drift_dt = (float)(In.drift_scale * In.dt);
            // coefficient tiles of the new instance (the previous MMA has completed)
            const float* tab = p.tables + (size_t)b * TS;
            float sc = 1.f;
            if constexpr (H) {
                // the scale of W: unfolded, every nonzero table entry is an
                // entry of W; folded, all but the m = 0 row and the n = 0
                // column (T0 and N0), as in scale_W_host
                float wm = 0.f;
                for (int q = tid; q < TS; q += 128) {
                    const int mn = q >> 3, m = mn / (K + 1), n = mn - m * (K + 1);
                    if (!F || (m > 0 && n > 0)) wm = fmaxf(wm, fabsf(tab[q]));
                }
                atomicMax(&s_wmax, __float_as_int(wm));
                __syncthreads();
                const int e = w_scale_exp(__int_as_float(s_wmax));
                sc = ldexpf(1.f, e);
                inv_s = ldexpf(1.f, -e);
            }
            for (int q = tid; q < S::NP * S::WS; q += 128) {
                const int nc = q / S::WS, k = q - nc * S::WS;
                const float w = w_entry<K, F>(tab, nc, k) * sc;
                if constexpr (H) {
                    const __half hi = __float2half_rn(w);
                    const __half lo = __float2half_rn(w - __half2float(hi));
                    const uint32_t off = tile_off<S::KC>(nc, k >> 3) + 2u * (uint32_t)(k & 7);
                    *reinterpret_cast<__half*>(B_hi + off) = hi;
                    *reinterpret_cast<__half*>(B_lo + off) = lo;
                } else {
                    const float hi = to_tf32(w);
                    const uint32_t off = tile_off<S::KC>(nc, k >> 2) + 4u * (uint32_t)(k & 3);
                    *reinterpret_cast<float*>(B_hi + off) = hi;
                    *reinterpret_cast<float*>(B_lo + off) = to_tf32(w - hi);
                }
            }
            if constexpr (F) {
                for (int q = tid; q < K; q += 128) {
                    sT0[q] = tab[(q + 1) * 8 + 0];                    // m = 0, n = q + 1: multiplies S2_n
                    sT0[K + q] = tab[(q + 1) * 8 + 1];                // multiplies C2_n
                    sN0[q] = tab[(q + 1) * (K + 1) * 8 + 4] * sc;     // n = 0 term of P2c(m = q + 1)
                    sN0[K + q] = tab[(q + 1) * (K + 1) * 8 + 6] * sc; // n = 0 term of P2s(m = q + 1)
                }
            }
            __syncthreads();
            continue;
        }

        // ---- two Euler steps per Philox call, one MMA per step, p.refill_pairs
        // pairs between refills (a lane whose path ends waits for the next refill)
#pragma unroll 1
        for (int pair = 0; pair < p.refill_pairs && !stop; ++pair) {
            float2 z1, z2;  // the two steps' normals, formed during the first product
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
                float2 sx, cx;
                sincos_turns2(make_float2(X1.val(), X2.val()), sx, cx);
                const float p0 = write_row_stream<K, F, H>(sb + row, (uint32_t)S::A_BYTES, sx.y, cx.y, sT0);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                // One barrier per step: the rows are in place, and a wait that gave
                // up in the previous step (any thread) stops the whole CTA.
                if (__syncthreads_or(failed)) { stop = true; break; }
                if (tid == 0) issue_step_mma<K, F, H>(tmem, sb, bar_a);
                // While the product runs: the Brownian increment and the x1 harmonics.
                if (half == 0) {
                    u32x4 r{0, 0, 0, 0};
                    if (pid >= 0) r = philox4x32_10(u32x4{(uint32_t)(n >> 1), i, j, stream}, key0, key1);
                    box_muller2(r.x, r.y, r.z, r.w, z1, z2);
                }
                const float xi1 = half ? z1.y : z1.x, xi2 = half ? z2.y : z2.x;
                Harm1 h1;  // during the product (HarmArray)
                h1.init(sx.x, cx.x);
                issued_any = true;
                failed = !tc::mbar_wait(bar_a, phase);
                phase ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float v1, v2;
                velocity_stream<K, F, H>(t_row, h1, sN0, p0, inv_s, v1, v2);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                if (pid < 0) continue;
                if (kind == 0) {
                    const bool last = (n == N - 1);
                    const float h = last ? h_last : dt, s = last ? s_last : s_dt;
                    em_update2(X1, X2, v1, v2, h, s, xi1, xi2);
                    if (last || wrap_due(n)) {  // the schedule of timedep_tc_kernel
                        X1.wrap();
                        X2.wrap();
                    }
                    ++n;
                    if (n >= N) {
                        p.g[sI.path_base + pid] = theta0_eval(p.th, X1, X2);
                        lane_steps += (unsigned long long)n;
                        pid = -1;
                    }
                } else {
                    em_update2(X1, X2, v1, v2, drift_dt, s_dt, xi1, xi2);
                    ++n;
                    const bool exited = exits_disk(X1, X2, p.R2hi, p.R2lo, p.band);
                    if (exited || n >= sI.max_steps) {
                        double gv = 0.0;
                        if (exited) gv = boundary_value(p.ga, p.gb, p.n_ang, p.R, p.quad, X1.full(), X2.full()) -
                                         p.f_const * ((double)n * sI.dt);
                        else atomicAdd(p.n_unexited, 1ull);
                        p.g[sI.path_base + pid] = gv;
                        lane_steps += (unsigned long long)n;
                        pid = -1;
                    }
                }
            }
        }
        if (stop) break;
    }
    if (failed && p.tc_err) atomicExch(p.tc_err, 1u);
    if (lane_steps) atomicAdd(p.steps, lane_steps);
    // No product may still write tensor memory when it is freed: after a wait
    // that gave up (stop), wait (full bound) for the last one issued.
    if (stop && issued_any) tc::mbar_wait(bar_a, phase ^ 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BatShape<K>::TMEM_COLS) : "memory");
    }
}

template <int K>
cudaError_t launch_batched_tc(const BatchKernelParams& p, int grid, cudaStream_t s)
{
    batched_tc_kernel<K><<<grid, 128, BatShape<K>::SMEM + 64, s>>>(p);
    return cudaGetLastError();
}

// Also sets the kernel's dynamic shared-memory limit (call outside any capture).
template <int K>
int batched_tc_blocks_per_sm()
{
    const int smem = BatShape<K>::SMEM + 64;
    cudaFuncSetAttribute(batched_tc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return resident_ctas((const void*)batched_tc_kernel<K>, 128, smem, (int)BatShape<K>::TMEM_COLS);
}

}  // namespace tdtc
}  // namespace pm

#define PM_INSTANTIATE_BATCHED_TC(K)                                                                        \
    template cudaError_t pm::tdtc::launch_batched_tc<K>(const pm::BatchKernelParams&, int, cudaStream_t); \
    template int pm::tdtc::batched_tc_blocks_per_sm<K>();
