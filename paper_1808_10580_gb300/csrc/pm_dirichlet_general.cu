// pm_dirichlet_general.cu -- Algorithm 2 in the disk |x| < R with a general
// forcing and a state-dependent diffusion (Theorem 3.2 with f(x) and
// sigma(x)) on the FP32 / FP64 pipes; the step's terms (the Milstein or
// Euler-Maruyama increment per coordinate, the left-point forcing sum) are in
// pm_general_step.cuh.  Everything else -- the product-basis velocity, the
// random numbers, the persistent lanes that take a new path as soon as theirs
// exits, the exit test, the boundary data, the per-path values reduced in path
// order -- is that of the constant-coefficient disk kernel (pm_kernels.cuh).
#include "pm_general_step.cuh"
#include "pm_kernels.cuh"

namespace pm {
namespace {

template <typename Real, int K>
struct GeneralParams {
    DirichletParams<Real, K> d;  // field, boundary data, paths, outputs (d.f_const: the constant part of f)
    GeneralCoef<Real> gc;
    double drift_scale;          // double paths: the drift factor and the step's
    double s0d[2], s1d[2];       // coefficients, applied in the plain sequential
    double sdt;                  // order of the scheme's statement
};

// Double paths: one coordinate's update with every operation rounded once in
// the order of the scheme's plain sequential statement,
// ((X - (d v) dt) + (sigma sqrt(dt)) xi) + (((1/2) sigma) sigma') (xi^2 - 1) dt.
__device__ __forceinline__ double update_d(double X, double v, double d, double dt, double s0, double s1, double sdt,
                                           bool milstein, double xi)
{
    const double sig = __dadd_rn(s0, __dmul_rn(s1, X));
    double Xn = __dadd_rn(__dsub_rn(X, __dmul_rn(__dmul_rn(d, v), dt)), __dmul_rn(__dmul_rn(sig, sdt), xi));
    if (milstein)
        Xn = __dadd_rn(Xn, __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(0.5, sig), s1), __dsub_rn(__dmul_rn(xi, xi), 1.0)), dt));
    return Xn;
}

template <typename Real, int K>
__device__ __forceinline__ void general_finish(const GeneralParams<Real, K>& gp, int64_t pid, bool exited, int64_t n,
                                               const Coord<Real>& X1, const Coord<Real>& X2, double integral)
{
    const DirichletParams<Real, K>& p = gp.d;
    double g = 0.0;
    if (exited) {
        const double y1 = X1.full(), y2 = X2.full();
        const double r = sqrt(y1 * y1 + y2 * y2);
        const double c1 = y1 / r, s1 = y2 / r;
        const double R = p.R;
        g = p.quad * (R * R) * (c1 * c1 - s1 * s1);
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

template <typename Real, int K>
__global__ void __launch_bounds__(kDirichletBlock)
    dirichlet_general_kernel(const __grid_constant__ GeneralParams<Real, K> gp)
{
    const DirichletParams<Real, K>& p = gp.d;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const ParamTable<Real, K> tab{p.field};
    int64_t pid = -1;
    bool done = false;
    int64_t n = 0;
    uint32_t j = 0, i = 0;
    unsigned long long lane_steps = 0;
    Coord<Real> X1, X2;
    X1.set(0.0);
    X2.set(0.0);
    ForcingSum<Real> fs;
    for (;;) {
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
                    const int64_t slot = cand / p.M, ii = cand - slot * p.M;
                    j = (uint32_t)(p.order ? (int64_t)p.order[slot] : slot);
                    i = (uint32_t)(ii + p.path_offset);
                    pid = (int64_t)j * p.M + ii;
                    X1.set(p.x[2 * (int64_t)j]);
                    X2.set(p.x[2 * (int64_t)j + 1]);
                    n = 0;
                    fs = ForcingSum<Real>{};
                    if (radial_excess(X1, X2, p.R2hi, p.R2lo) >= (Real)0) {
                        general_finish(gp, pid, true, 0, X1, X2, 0.0);
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
            const Real x1v = X1.val(), x2v = X2.val();
            fs.add(gp.gc.forcing(x1v, x2v));
            Real x1[1] = {x1v}, x2[1] = {x2v}, v1[1], v2[1];
            velocity<Real, K, 1>(tab, x1, x2, v1, v2);
            if constexpr (sizeof(Real) == 8) {
                const bool mil = gp.gc.half_dt_m != (Real)0;
                X1.hi = update_d(X1.hi, v1[0], gp.drift_scale, p.dt, gp.s0d[0], gp.s1d[0], gp.sdt, mil, xi1);
                X2.hi = update_d(X2.hi, v2[0], gp.drift_scale, p.dt, gp.s0d[1], gp.s1d[1], gp.sdt, mil, xi2);
            } else {
                X1.add(gp.gc.increment(0, x1v, v1[0], p.drift_dt, xi1));
                X2.add(gp.gc.increment(1, x2v, v2[0], p.drift_dt, xi2));
            }
            ++n;
            const bool exited = radial_excess(X1, X2, p.R2hi, p.R2lo) >= (Real)0;
            if (exited || n >= p.max_steps) {
                general_finish(gp, pid, exited, n, X1, X2, fs.value() * p.dt);
                lane_steps += (unsigned long long)n;
                pid = -1;
                break;
            }
        }
    }
    if (lane_steps) atomicAdd(p.steps, lane_steps);
}

}  // namespace

template <typename Real, int K>
cudaError_t launch_dirichlet_general(const DirichletLaunch& L, cudaStream_t stream)
{
    if (!L.gen) return cudaErrorInvalidValue;
    const DirichletGeneral& G = *L.gen;
    GeneralParams<Real, K> gp;
    DirichletParams<Real, K>& p = gp.d;
    for (int t = 0; t < table_size(K); ++t) p.field.c[t] = (Real)L.coef[t];
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
    p.s_dt = (Real)0;
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
    gp.gc.set(G, L.dt, L.f_const);
    gp.sdt = std::sqrt(L.dt);
    gp.drift_scale = L.drift_scale;
    for (int k = 0; k < 2; ++k) {
        gp.s0d[k] = G.s0[k];
        gp.s1d[k] = G.s1[k];
    }
    dirichlet_general_kernel<Real, K><<<L.grid, kDirichletBlock, 0, stream>>>(gp);
    return cudaGetLastError();
}

template <typename Real, int K>
int dirichlet_general_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dirichlet_general_kernel<Real, K>, kDirichletBlock, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

#define PM_GEN(R, K)                                                                          \
    template cudaError_t launch_dirichlet_general<R, K>(const DirichletLaunch&, cudaStream_t); \
    template int dirichlet_general_blocks_per_sm<R, K>();
#define PM_GEN_BOTH(K) PM_GEN(float, K) PM_GEN(double, K)
PM_GEN_BOTH(0)
PM_GEN_BOTH(1)
PM_GEN_BOTH(2)
PM_GEN_BOTH(3)
PM_GEN_BOTH(4)
PM_GEN_BOTH(5)
PM_GEN_BOTH(6)
PM_GEN_BOTH(8)
PM_GEN_BOTH(10)
PM_GEN_BOTH(12)
PM_GEN_BOTH(16)
#undef PM_GEN_BOTH
#undef PM_GEN

}  // namespace pm
