// pm_square_bvp.cu -- the optimal-forcing boundary-value problem of Section 4
// (Eq. bvp:ex1) by Algorithm 2 / Theorem 3.2: walks in the unit square with
// constant drift, each returning the boundary value at its exit and the time
// integrals of every Gaussian source profile along the way.
//
// Persistent kernel with per-lane refill (one atomic per warp per refill,
// lanes in step parity so one Philox call serves two steps), as for the disk
// problem; the drift is constant, so a step is the noise, the update, the
// exit test and n_src exponentials.  Per-path values go to
// out[(j (n_src+1) + q) M + i] and are reduced per (observation, functional)
// in path order.
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "pm_internal.h"
#include "pm_kernels.cuh"
#include "pm_launch.h"

namespace pm {
namespace {

constexpr int kSquareBlock = 128;

template <typename Real>
struct SquareParams {
    Real c1[PM_MAX_SOURCES], c2[PM_MAX_SOURCES];
    Real b1_dt, b2_dt, s_dt, w, dt_r;
    double dt, g_cos, g_quad;
    int32_t n_src;
    const double* x;
    int64_t n_obs, M, total, max_steps, path_offset;
    unsigned long long* counter;
    unsigned long long* n_unexited;
    unsigned long long* steps;
    double* out;
    int32_t* exit_step;
    uint32_t inst, key0, key1;
};

// Position outside the open interval (0, 1): for float paths the sign of
// X - 0 and X - 1 from the compensated pair (hi - 1 is exact near 1).
__device__ __forceinline__ bool outside01(const Coord<float>& X)
{
    const float d = X.hi - 1.0f;
    return X.hi < 0.0f || (X.hi == 0.0f && X.lo <= 0.0f) || d > 0.0f || (d == 0.0f && X.lo >= 0.0f);
}
__device__ __forceinline__ bool outside01(const Coord<double>& X) { return X.hi <= 0.0 || X.hi >= 1.0; }

__device__ __forceinline__ float exp_(float a) { return expf(a); }
__device__ __forceinline__ double exp_(double a) { return exp(a); }

// Running time integral of one source profile along a path.  Float paths
// keep a compensated (Kahan) float sum, so the step loop stays off the
// double-precision pipe; double paths add in double.
template <typename Real> struct PathSum;
template <> struct PathSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct PathSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

template <typename Real>
__device__ __forceinline__ void square_finish(const SquareParams<Real>& p, int64_t pid, bool exited, int64_t n,
                                              const Coord<Real>& X1, const Coord<Real>& X2,
                                              const PathSum<Real> (&sums)[PM_MAX_SOURCES])
{
    const int64_t nf = p.n_src + 1;
    const int64_t j = pid / p.M, i = pid - j * p.M;
    double* o = p.out + (j * nf) * p.M + i;
    if (exited) {
        const double y1 = fmin(fmax(X1.full(), 0.0), 1.0), y2 = fmin(fmax(X2.full(), 0.0), 1.0);
        const double h = 1.5707963267948966;  // pi / 2
        o[0] = p.g_cos * 0.5 * (cos(h * y1) + cos(h * y2)) + p.g_quad * (y1 * y1 - y2 * y2);
#pragma unroll
        for (int q = 0; q < PM_MAX_SOURCES; ++q)
            if (q < p.n_src) o[(q + 1) * p.M] = sums[q].value();
    } else {
        for (int64_t q = 0; q < nf; ++q) o[q * p.M] = 0.0;
        atomicAdd(p.n_unexited, 1ull);
    }
    if (p.exit_step) p.exit_step[pid] = exited ? (int32_t)n : -1;
}

template <typename Real>
__global__ void __launch_bounds__(kSquareBlock) square_bvp_kernel(const __grid_constant__ SquareParams<Real> p)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int64_t pid = -1;
    bool done = false;
    int64_t n = 0;
    uint32_t j = 0, i = 0;
    unsigned long long lane_steps = 0;
    PathSum<Real> sums[PM_MAX_SOURCES];
    Coord<Real> X1, X2;
    X1.set(0.0);
    X2.set(0.0);
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
                    pid = cand;
                    j = (uint32_t)(cand / p.M);
                    i = (uint32_t)(cand - (int64_t)j * p.M + p.path_offset);
                    X1.set(p.x[2 * (int64_t)j]);
                    X2.set(p.x[2 * (int64_t)j + 1]);
                    n = 0;
#pragma unroll
                    for (int q = 0; q < PM_MAX_SOURCES; ++q) sums[q] = PathSum<Real>{};
                    if (outside01(X1) || outside01(X2)) {  // starts on or outside the boundary
                        square_finish(p, pid, true, 0, X1, X2, sums);
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
            // left-point rule: the source profiles at X_n
            const Real x1 = X1.val(), x2 = X2.val();
#pragma unroll
            for (int q = 0; q < PM_MAX_SOURCES; ++q) {
                if (q < p.n_src) {
                    const Real d1 = x1 - p.c1[q], d2 = x2 - p.c2[q];
                    sums[q].add(exp_(-p.w * (d1 * d1 + d2 * d2)) * p.dt_r);
                }
            }
            Real xi1, xi2;
            box_muller<Real>(half ? r.z : r.x, half ? r.w : r.y, xi1, xi2);
            em_update<Real>(X1, p.b1_dt, (Real)1, p.s_dt, xi1);
            em_update<Real>(X2, p.b2_dt, (Real)1, p.s_dt, xi2);
            ++n;
            const bool exited = outside01(X1) || outside01(X2);
            if (exited || n >= p.max_steps) {
                square_finish(p, pid, exited, n, X1, X2, sums);
                lane_steps += (unsigned long long)n;
                pid = -1;
                break;
            }
        }
    }
    if (lane_steps) atomicAdd(p.steps, lane_steps);
}

template <typename Real>
int square_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, square_bvp_kernel<Real>, kSquareBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace
}  // namespace pm

using namespace pm;

extern "C" int pm_forward_square_bvp(pm_ctx* c, const pm_square_bvp* prob, const double* x, int64_t n_obs,
                                     int64_t M, double dt, int64_t max_steps, uint64_t seed, uint32_t flags,
                                     double* mean, double* var, int32_t* exit_step, int64_t* n_unexited,
                                     const pm_path_opts* opts)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    if (!prob) return fail(PM_EINVAL, "problem is NULL");
    if (prob->n_src < 0 || prob->n_src > PM_MAX_SOURCES) return fail(PM_EINVAL, "n_src must be in [0, %d]", PM_MAX_SOURCES);
    if (prob->n_src > 0 && (!prob->c || !finite_array(prob->c, 2 * (int64_t)prob->n_src)))
        return fail(PM_EINVAL, "source centres missing or not finite");
    if (!(std::isfinite(prob->b[0]) && std::isfinite(prob->b[1]) && std::isfinite(prob->kappa) && prob->kappa >= 0 &&
          std::isfinite(prob->w) && prob->w >= 0 && std::isfinite(prob->g_cos) && std::isfinite(prob->g_quad)))
        return fail(PM_EINVAL, "drift, kappa, w and boundary coefficients must be finite (kappa, w >= 0)");
    if (!(std::isfinite(dt) && dt > 0)) return fail(PM_EINVAL, "dt must be finite and > 0");
    if (max_steps < 1 || max_steps > 0x7fffffffLL) return fail(PM_EINVAL, "max_steps must be in [1, 2^31)");
    if (n_obs < 0 || M < 1) return fail(PM_EINVAL, "need n_obs >= 0 and M >= 1");
    if (n_obs == 0) return PM_OK;
    const int64_t off = opts ? opts->path_offset : 0;
    if (off < 0 || off + M > ((int64_t)1 << 32)) return fail(PM_EINVAL, "path_offset + M exceeds 2^32");
    if (!x || !mean) return fail(PM_EINVAL, "x and mean must not be NULL");
    double* g_out = opts ? opts->g_out : nullptr;
    int rc = check_ptrs(c, flags, {x, mean, var, exit_step, n_unexited, g_out});
    if (rc) return rc;
    if (!(flags & PM_DEVICE_PTRS) && !finite_array(x, 2 * n_obs)) return fail(PM_EINVAL, "x contains NaN or Inf");
    if ((rc = set_device(c))) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    const bool fp64 = flags & PM_FP64;
    const int64_t nf = prob->n_src + 1;
    const int64_t total = n_obs * M;
    const int64_t rows = n_obs * nf;

    auto layout = [&](Bump& b) {
        struct P { unsigned long long* ctr; double *out, *x, *mean, *var; int32_t* es; double2* rpart; } p{};
        p.ctr = b.take<unsigned long long>(4);  // next path, unexited, steps
        p.out = (dev && g_out) ? nullptr : b.take<double>((size_t)(rows * M));
        p.rpart = b.take<double2>((size_t)(rows * (int64_t)reduce_path_chunks(M)));
        if (!dev) {
            p.x = b.take<double>((size_t)(2 * n_obs));
            p.mean = b.take<double>((size_t)rows);
            p.var = var ? b.take<double>((size_t)rows) : nullptr;
            p.es = exit_step ? b.take<int32_t>((size_t)total) : nullptr;
        }
        return p;
    };
    Bump probe(nullptr);
    layout(probe);
    if ((rc = ensure_workspace(c, probe.off))) return rc;
    Bump bump(c->ws);
    auto W = layout(bump);

    const double* dx = x;
    double *dmean = mean, *dvar = var, *dout = (dev && g_out) ? g_out : W.out;
    int32_t* des = exit_step;
    if (!dev) {
        const size_t outb = (size_t)rows * 16 + (g_out ? (size_t)(rows * M) * 8 : 0) +
                            (exit_step ? (size_t)total * 4 : 0) + 256;
        const size_t inb = (size_t)n_obs * 16 + 64;
        if ((rc = ensure_host(c, inb > outb ? inb : outb))) return rc;
        memcpy(c->host, x, (size_t)n_obs * 16);
        PM_CUDA(cudaMemcpyAsync(W.x, c->host, (size_t)n_obs * 16, cudaMemcpyHostToDevice, c->stream), "copy x");
        dx = W.x;
        dmean = W.mean;
        dvar = W.var;
        des = W.es;
    }
    PM_CUDA(cudaMemsetAsync(W.ctr, 0, 32, c->stream), "clear counters");
    c->last_steps = -1;

    const double s_dt = std::sqrt(2.0 * prob->kappa * dt);
    const uint32_t inst = opts ? opts->instance : 0u;
    const int per_sm = fp64 ? square_blocks_per_sm<double>() : square_blocks_per_sm<float>();
    int64_t grid = (int64_t)per_sm * c->sm_count;
    const int64_t need = (total + kSquareBlock - 1) / kSquareBlock;
    if (grid > need) grid = need;
    c->last_grid = grid;
    if (c->timing) PM_CUDA(cudaEventRecord(c->ev0, c->stream), "event");
    auto fill = [&](auto& p) {
        using R = std::remove_reference_t<decltype(p.s_dt)>;
        for (int q = 0; q < PM_MAX_SOURCES; ++q) {
            p.c1[q] = q < prob->n_src ? (R)prob->c[2 * q] : (R)0;
            p.c2[q] = q < prob->n_src ? (R)prob->c[2 * q + 1] : (R)0;
        }
        p.b1_dt = (R)(prob->b[0] * dt);
        p.b2_dt = (R)(prob->b[1] * dt);
        p.s_dt = (R)s_dt;
        p.w = (R)prob->w;
        p.dt_r = (R)dt;
        p.dt = dt;
        p.g_cos = prob->g_cos;
        p.g_quad = prob->g_quad;
        p.n_src = prob->n_src;
        p.x = dx;
        p.n_obs = n_obs;
        p.M = M;
        p.total = total;
        p.max_steps = max_steps;
        p.path_offset = off;
        p.counter = W.ctr;
        p.n_unexited = W.ctr + 1;
        p.steps = W.ctr + 2;
        p.out = dout;
        p.exit_step = des;
        p.inst = inst;
        p.key0 = (uint32_t)(seed & 0xffffffffu);
        p.key1 = (uint32_t)(seed >> 32);
    };
    if (fp64) {
        SquareParams<double> p;
        fill(p);
        square_bvp_kernel<double><<<(unsigned)grid, kSquareBlock, 0, c->stream>>>(p);
    } else {
        SquareParams<float> p;
        fill(p);
        square_bvp_kernel<float><<<(unsigned)grid, kSquareBlock, 0, c->stream>>>(p);
    }
    PM_CUDA(cudaGetLastError(), "square kernel launch");
    if (c->timing) {
        PM_CUDA(cudaEventRecord(c->ev1, c->stream), "event");
        c->timed = true;
    }
    count_launch(c);
    PM_CUDA(launch_reduce_paths(dout, rows, M, dmean, dvar, c->stream, W.rpart), "reduce kernel");
    count_launch(c, reduce_path_chunks(M) > 0 ? 2 : 1);
    if (dev && n_unexited)
        PM_CUDA(cudaMemcpyAsync(n_unexited, W.ctr + 1, 8, cudaMemcpyDeviceToDevice, c->stream), "copy n_unexited");
    if (dev && (flags & PM_ASYNC)) return PM_OK;
    unsigned long long unexited = 0, steps_taken = 0;
    if (!dev) {
        char* h = (char*)c->host;
        size_t o = 0;
        PM_CUDA(cudaMemcpyAsync(h + o, dmean, (size_t)rows * 8, cudaMemcpyDeviceToHost, c->stream), "copy mean");
        o += (size_t)rows * 8;
        if (var) { PM_CUDA(cudaMemcpyAsync(h + o, dvar, (size_t)rows * 8, cudaMemcpyDeviceToHost, c->stream), "copy var"); o += (size_t)rows * 8; }
        if (g_out) { PM_CUDA(cudaMemcpyAsync(h + o, dout, (size_t)(rows * M) * 8, cudaMemcpyDeviceToHost, c->stream), "copy paths"); o += (size_t)(rows * M) * 8; }
        if (exit_step) PM_CUDA(cudaMemcpyAsync(h + o, des, (size_t)total * 4, cudaMemcpyDeviceToHost, c->stream), "copy exit steps");
    }
    PM_CUDA(cudaMemcpyAsync(&unexited, W.ctr + 1, 8, cudaMemcpyDeviceToHost, c->stream), "copy n_unexited");
    PM_CUDA(cudaMemcpyAsync(&steps_taken, W.ctr + 2, 8, cudaMemcpyDeviceToHost, c->stream), "copy step count");
    PM_CUDA(cudaStreamSynchronize(c->stream), "square bvp");
    c->last_steps = (int64_t)steps_taken;
    if (!dev) {
        const char* h = (const char*)c->host;
        size_t o = 0;
        memcpy(mean, h + o, (size_t)rows * 8);
        o += (size_t)rows * 8;
        if (var) { memcpy(var, h + o, (size_t)rows * 8); o += (size_t)rows * 8; }
        if (g_out) { memcpy(g_out, h + o, (size_t)(rows * M) * 8); o += (size_t)(rows * M) * 8; }
        if (exit_step) memcpy(exit_step, h + o, (size_t)total * 4);
        if (n_unexited) *n_unexited = (int64_t)unexited;
    }
    return unexited ? PM_WARN_UNEXITED : PM_OK;
}
