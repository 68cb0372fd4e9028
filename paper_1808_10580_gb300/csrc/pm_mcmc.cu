// pm_mcmc.cu -- pCN MCMC over the forward map, plain or with delayed
// acceptance through the learned surrogate.
//
// The paper computes its posteriors with preconditioned Crank-Nicolson MCMC
// (Section 4.1).  Chains live on the device.  One step of every chain:
//   propose   u' = sqrt(1 - beta^2) u + beta C^{1/2} xi   (prior C = diag(|k|^-4))
//   stage 1   (delayed acceptance only) Phi~(u') from the surrogate network;
//             accept with min(1, exp(Phi~(u) - Phi~(u')))  (Christen & Fox 2005)
//   stage 2   the particle map G(u') for the surviving proposals only (one
//             batched launch; every chain shares one RNG stream and seed, so G
//             is a deterministic function of u); Phi(u') in double; accept with
//             min(1, exp(Phi(u) - Phi(u') - Phi~(u) + Phi~(u')))  (plain pCN:
//             min(1, exp(Phi(u) - Phi(u'))))
// Random numbers: proposal normals of chain c at step s from Philox counters
// {s, c, q, 0x4D43} (four normals per counter by two Box-Muller pairs), the
// stage-1 / stage-2 uniforms from {s, c, 0xFFFFFFFF, 1 | 2}, all under the
// key of `seed`.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pm.h"
#include "pm_device.cuh"
#include "pm_internal.h"

using namespace pm;

namespace {

constexpr uint32_t kTagProposal = 0x4D43u;
constexpr uint32_t kQUniform = 0xFFFFFFFFu;

__device__ __forceinline__ double uniform_d(uint32_t r) { return ((double)(r >> 9) * 2.0 + 1.0) * 5.9604644775390625e-08; }

__global__ void propose_kernel(const double* __restrict__ U, double* __restrict__ Up, const double* __restrict__ std_,
                               int C, int n_u, double rho, double beta, uint32_t k0, uint32_t k1, uint32_t step)
{
    const int nq = (n_u + 3) / 4;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)C * nq) return;
    const int c = (int)(t / nq), q = (int)(t % nq);
    const u32x4 r = philox4x32_10(u32x4{step, (uint32_t)c, (uint32_t)q, kTagProposal}, k0, k1);
    double z[4];
    box_muller<double>(r.x, r.y, z[0], z[1]);
    box_muller<double>(r.z, r.w, z[2], z[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int h = 4 * q + k;
        if (h < n_u) Up[(size_t)c * n_u + h] = rho * U[(size_t)c * n_u + h] + beta * std_[h] * z[k];
    }
}

__global__ void screen_input_kernel(const double* __restrict__ Up, const double* __restrict__ shift,
                                    const float* __restrict__ scale, int C, int n_u, float* __restrict__ X)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)C * n_u) return;
    X[t] = (float)((Up[t] - shift[t % n_u]) * (double)scale[t % n_u]);
}

__device__ double misfit(const double* __restrict__ y, const float* __restrict__ Gf, const double* __restrict__ Gd,
                         int n_obs, double inv2s2)
{
    double s = 0.0;
    for (int j = 0; j < n_obs; ++j) {
        const double g = Gf ? (double)Gf[j] : Gd[j];
        const double r = y[j] - g;
        s += r * r;
    }
    return s * inv2s2;
}

// Stage 1 (one thread per chain).
__global__ void stage1_kernel(const double* __restrict__ y, const float* __restrict__ Gs, int C, int n_obs,
                              double inv2s2, const double* __restrict__ PhiS, double* __restrict__ PhiS_new,
                              int* __restrict__ pass, uint32_t k0, uint32_t k1, uint32_t step)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double ps = misfit(y, Gs + (size_t)c * n_obs, nullptr, n_obs, inv2s2);
    PhiS_new[c] = ps;
    const u32x4 r = philox4x32_10(u32x4{step, (uint32_t)c, kQUniform, 1u}, k0, k1);
    pass[c] = uniform_d(r.x) < exp(fmin(0.0, PhiS[c] - ps)) ? 1 : 0;
}

// G(u') = A u' for the listed chains (the linear test map).
__global__ void linear_map_kernel(const double* __restrict__ A, const double* __restrict__ Up,
                                  const int* __restrict__ idx, int n, int n_obs, int n_u, double* __restrict__ G)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n_obs) return;
    const int s = (int)(t / n_obs), j = (int)(t % n_obs);
    const double* u = Up + (size_t)idx[s] * n_u;
    double acc = 0.0;
    for (int h = 0; h < n_u; ++h) acc += A[(size_t)j * n_u + h] * u[h];
    G[t] = acc;
}

// Stage 2 / plain acceptance (one thread per listed chain).
__global__ void accept_kernel(const int* __restrict__ idx, int n, const double* __restrict__ y,
                              const double* __restrict__ G, int n_obs, double inv2s2, int da, double* __restrict__ Phi,
                              double* __restrict__ PhiS, const double* __restrict__ PhiS_new, double* __restrict__ U,
                              const double* __restrict__ Up, int n_u, uint32_t k0, uint32_t k1, uint32_t step,
                              unsigned long long* __restrict__ accepts, const double* __restrict__ std_,
                              double* __restrict__ jump)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int c = idx[s];
    const double ph = misfit(y, nullptr, G + (size_t)s * n_obs, n_obs, inv2s2);
    double a = Phi[c] - ph;
    if (da) a -= PhiS[c] - PhiS_new[c];
    const u32x4 r = philox4x32_10(u32x4{step, (uint32_t)c, kQUniform, 2u}, k0, k1);
    if (uniform_d(r.x) < exp(fmin(0.0, a))) {
        Phi[c] = ph;
        if (da) PhiS[c] = PhiS_new[c];
        double sq = 0.0;  // squared jump in prior-whitened coordinates
        for (int h = 0; h < n_u; ++h) {
            const double d = (Up[(size_t)c * n_u + h] - U[(size_t)c * n_u + h]) / std_[h];
            sq += d * d;
            U[(size_t)c * n_u + h] = Up[(size_t)c * n_u + h];
        }
        jump[c] += sq;
        atomicAdd(accepts, 1ull);
    }
}

__global__ void accumulate_kernel(const double* __restrict__ U, int C, int n_u, double* __restrict__ sum_u)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n_u) return;
    double s = 0.0;
    for (int c = 0; c < C; ++c) s += U[(size_t)c * n_u + h];
    sum_u[h] += s;
}

// Initial misfits: Phi of given maps for all chains.
__global__ void misfit_all_kernel(const double* __restrict__ y, const double* __restrict__ Gd,
                                  const float* __restrict__ Gf, int C, int n_obs, double inv2s2, double* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    out[c] = misfit(y, Gf ? Gf + (size_t)c * n_obs : nullptr, Gd ? Gd + (size_t)c * n_obs : nullptr, n_obs, inv2s2);
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct pm_pcn {
    int C = 0, n_u = 0, K = 0;
    int64_t n_obs = 0;
    double beta = 0, sigma = 0, rho = 0;
    uint64_t seed = 0;
    int64_t step = 0;
    bool linear = false;
    // particle map description (host copies)
    double kappa = 0, dt = 0;
    int64_t M = 0;
    uint64_t path_seed = 0;
    uint32_t map_flags = 0;     // PM_TENSOR or 0
    std::vector<int32_t> qk;
    std::vector<double> qa, qb;
    // screen
    const pm_mlp* screen = nullptr;
    // device state
    void* buf = nullptr;
    double *U, *Up, *stdv, *y, *A, *Phi, *PhiS, *PhiS_new, *G, *sum_u, *x_rep, *t_rep;
    float *scale, *X, *Gs;
    double* shift;              // surrogate input (u - shift) * scale
    double* jump;               // per chain: squared prior-whitened jumps of accepted moves in the current run
    int *pass, *idx;
    unsigned long long* accepts;
    int64_t n_summed = 0;
    std::vector<pm_instance> inst;
};

namespace {

// G for the chains listed in idx_h (device copy in p->idx): into p->G rows 0..n-1.
int forward_listed(pm_ctx* c, pm_pcn* p, const std::vector<int>& idx_h)
{
    const int n = (int)idx_h.size();
    if (n == 0) return PM_OK;
    PM_CUDA(cudaMemcpyAsync(p->idx, idx_h.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, c->stream), "copy index");
    if (p->linear) {
        linear_map_kernel<<<blocks((int64_t)n * p->n_obs, 128), 128, 0, c->stream>>>(p->A, p->Up, p->idx, n, (int)p->n_obs,
                                                                                     p->n_u, p->G);
        PM_CUDA(cudaGetLastError(), "linear map");
        count_launch(c);
        return PM_OK;
    }
    p->inst.resize((size_t)n);
    for (int s = 0; s < n; ++s) {
        pm_instance& I = p->inst[(size_t)s];
        memset(&I, 0, sizeof I);
        I.kind = PM_KIND_TIMEDEP;
        I.stream = 0;                      // one stream and seed for every evaluation
        I.u = p->Up + (size_t)idx_h[(size_t)s] * p->n_u;
        I.kappa = p->kappa;
        I.dt = p->dt;
        I.drift_scale = 1.0;
        I.row0 = (int64_t)s * p->n_obs;
        I.n_obs = p->n_obs;
        I.M = p->M;
        I.seed = p->path_seed;
    }
    pm_fourier th{(int32_t)p->qa.size(), 0, p->qk.data(), p->qa.data(), p->qb.data()};
    pm_batch b{};
    b.K = p->K;
    b.B = n;
    b.inst = p->inst.data();
    b.theta0 = &th;
    b.disk = nullptr;
    b.x = p->x_rep;
    b.t = p->t_rep;
    b.n_rows = (int64_t)n * p->n_obs;
    int rc = pm_forward_batched(c, &b, PM_DEVICE_PTRS | p->map_flags, p->G, nullptr, nullptr);
    return rc < 0 ? rc : PM_OK;
}

}  // namespace

extern "C" {

int pm_pcn_create(pm_ctx* c, pm_pcn** out, const pm_pcn_config* cfg, const double* u0, const pm_mlp* screen,
                  const float* screen_scale)
{
    if (!c || !out || !cfg || !u0) return fail(PM_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->n_chains < 1 || cfg->n_chains > 65536) return fail(PM_EINVAL, "n_chains out of range");
    if (!supported_K(cfg->K) || cfg->K < 1) return fail(PM_EINVAL, "unsupported K");
    if (!(cfg->beta > 0 && cfg->beta <= 1) || !(cfg->sigma > 0)) return fail(PM_EINVAL, "need 0 < beta <= 1, sigma > 0");
    if (cfg->n_obs < 1 || !cfg->y) return fail(PM_EINVAL, "observations missing");
    if (cfg->map_flags & ~(uint32_t)PM_TENSOR) return fail(PM_EINVAL, "map_flags: only PM_TENSOR");
    const bool linear = cfg->A != nullptr;
    if (!linear) {
        if (!cfg->theta0 || !cfg->x || !cfg->t || cfg->M < 1 || !(cfg->dt > 0) || !(cfg->kappa >= 0))
            return fail(PM_EINVAL, "particle map description incomplete");
        if (cfg->theta0->n < 0 || cfg->theta0->n > PM_MAX_THETA0_MODES) return fail(PM_EINVAL, "theta0 modes");
    }
    int rc = set_device(c);
    if (rc) return rc;
    pm_pcn* p = new (std::nothrow) pm_pcn;
    if (!p) return fail(PM_ENOMEM, "pcn object");
    p->C = cfg->n_chains;
    p->K = cfg->K;
    p->n_u = (2 * cfg->K + 1) * (2 * cfg->K + 1) - 1;
    p->n_obs = cfg->n_obs;
    p->beta = cfg->beta;
    p->rho = std::sqrt(1.0 - cfg->beta * cfg->beta);
    p->sigma = cfg->sigma;
    p->seed = cfg->seed;
    p->map_flags = cfg->map_flags;
    p->linear = linear;
    p->screen = screen;
    if (!linear) {
        p->kappa = cfg->kappa;
        p->dt = cfg->dt;
        p->M = cfg->M;
        p->path_seed = cfg->path_seed;
        const int nq = cfg->theta0->n;
        p->qk.assign(cfg->theta0->k, cfg->theta0->k + 2 * nq);
        p->qa.assign(cfg->theta0->a, cfg->theta0->a + nq);
        p->qb.assign(cfg->theta0->b, cfg->theta0->b + nq);
    }
    const int C = p->C, n_u = p->n_u;
    const int64_t n_obs = p->n_obs;
    Bump probe(nullptr);
    auto plan = [&](Bump& b) {
        p->U = b.take<double>((size_t)C * n_u); p->Up = b.take<double>((size_t)C * n_u);
        p->stdv = b.take<double>((size_t)n_u); p->y = b.take<double>((size_t)n_obs);
        p->A = linear ? b.take<double>((size_t)(n_obs * n_u)) : nullptr;
        p->Phi = b.take<double>((size_t)C); p->PhiS = b.take<double>((size_t)C); p->PhiS_new = b.take<double>((size_t)C);
        p->G = b.take<double>((size_t)(C * n_obs)); p->sum_u = b.take<double>((size_t)n_u);
        p->x_rep = linear ? nullptr : b.take<double>((size_t)(2 * C * n_obs));
        p->t_rep = linear ? nullptr : b.take<double>((size_t)(C * n_obs));
        p->scale = b.take<float>((size_t)n_u); p->X = b.take<float>((size_t)C * n_u);
        p->shift = b.take<double>((size_t)n_u);
        p->jump = b.take<double>((size_t)C);
        p->Gs = b.take<float>((size_t)(C * n_obs));
        p->pass = b.take<int>((size_t)C); p->idx = b.take<int>((size_t)C);
        p->accepts = b.take<unsigned long long>(4);
    };
    plan(probe);
    if (cudaMalloc(&p->buf, probe.off) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(PM_ENOMEM, "pcn state");
    }
    Bump real(p->buf);
    plan(real);
    // prior standard deviations |k_h|^-2 per real coefficient, in the field layout
    std::vector<double> sd((size_t)n_u);
    {
        int h = 0;
        auto put = [&](int m, int n) { const double s = 1.0 / ((double)m * m + (double)n * n); sd[(size_t)h++] = s; sd[(size_t)h++] = s; };
        for (int n = 1; n <= p->K; ++n) put(0, n);
        for (int m = 1; m <= p->K; ++m)
            for (int n = -p->K; n <= p->K; ++n) put(m, n);
    }
    std::vector<float> sc((size_t)n_u, 1.0f);
    if (screen_scale) memcpy(sc.data(), screen_scale, sizeof(float) * (size_t)n_u);
    std::vector<double> sh((size_t)n_u, 0.0);
    if (cfg->screen_shift) memcpy(sh.data(), cfg->screen_shift, sizeof(double) * (size_t)n_u);
    cudaError_t e = cudaMemcpyAsync(p->U, u0, sizeof(double) * (size_t)C * n_u, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->Up, u0, sizeof(double) * (size_t)C * n_u, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->stdv, sd.data(), sizeof(double) * (size_t)n_u, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->y, cfg->y, sizeof(double) * (size_t)n_obs, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && linear)
        e = cudaMemcpyAsync(p->A, cfg->A, sizeof(double) * (size_t)(n_obs * n_u), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->scale, sc.data(), sizeof(float) * (size_t)n_u, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->shift, sh.data(), sizeof(double) * (size_t)n_u, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->sum_u, 0, sizeof(double) * (size_t)n_u, c->stream);
    if (e == cudaSuccess && !linear) {
        std::vector<double> xr((size_t)(2 * C * n_obs)), tr((size_t)(C * n_obs));
        for (int q = 0; q < C; ++q) {
            memcpy(&xr[(size_t)(2 * q * n_obs)], cfg->x, sizeof(double) * (size_t)(2 * n_obs));
            memcpy(&tr[(size_t)(q * n_obs)], cfg->t, sizeof(double) * (size_t)n_obs);
        }
        e = cudaMemcpyAsync(p->x_rep, xr.data(), xr.size() * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->t_rep, tr.data(), tr.size() * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) { pm_pcn_destroy(p); return cuda_fail(e, "pcn init"); }
    // Initial misfits Phi(u0) (and Phi~(u0)).
    std::vector<int> all((size_t)C);
    for (int q = 0; q < C; ++q) all[(size_t)q] = q;
    const double inv2s2 = 1.0 / (2.0 * p->sigma * p->sigma);
    if ((rc = forward_listed(c, p, all))) { pm_pcn_destroy(p); return rc; }
    misfit_all_kernel<<<blocks(C, 128), 128, 0, c->stream>>>(p->y, p->G, nullptr, C, (int)n_obs, inv2s2, p->Phi);
    if (screen) {
        screen_input_kernel<<<blocks((int64_t)C * n_u, 256), 256, 0, c->stream>>>(p->Up, p->shift, p->scale, C, n_u, p->X);
        if ((rc = pm_surrogate_infer(c, screen, p->X, C, p->Gs, PM_DEVICE_PTRS))) { pm_pcn_destroy(p); return rc; }
        misfit_all_kernel<<<blocks(C, 128), 128, 0, c->stream>>>(p->y, nullptr, p->Gs, C, (int)n_obs, inv2s2, p->PhiS);
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { pm_pcn_destroy(p); return cuda_fail(e, "pcn init"); }
    *out = p;
    return PM_OK;
}

void pm_pcn_destroy(pm_pcn* p)
{
    if (!p) return;
    if (p->buf) cudaFree(p->buf);
    delete p;
}

int pm_pcn_run(pm_ctx* c, pm_pcn* p, int64_t n_steps, pm_pcn_stats* st)
{
    if (!c || !p) return fail(PM_EINVAL, "NULL argument");
    if (n_steps < 0) return fail(PM_EINVAL, "n_steps < 0");
    int rc = set_device(c);
    if (rc) return rc;
    const int C = p->C, n_u = p->n_u, n_obs = (int)p->n_obs;
    const double inv2s2 = 1.0 / (2.0 * p->sigma * p->sigma);
    const uint32_t k0 = (uint32_t)(p->seed & 0xffffffffu), k1 = (uint32_t)(p->seed >> 32);
    const bool da = p->screen != nullptr;
    std::vector<int> pass_h((size_t)C), idx_h;
    idx_h.reserve((size_t)C);
    pm_pcn_stats s{};
    PM_CUDA(cudaMemsetAsync(p->accepts, 0, 8, c->stream), "clear counter");
    PM_CUDA(cudaMemsetAsync(p->jump, 0, sizeof(double) * (size_t)C, c->stream), "clear jumps");
    cudaEvent_t e0, e1;
    PM_CUDA(cudaEventCreate(&e0), "event");
    PM_CUDA(cudaEventCreate(&e1), "event");
    PM_CUDA(cudaEventRecord(e0, c->stream), "event");
    for (int64_t it = 0; it < n_steps; ++it) {
        const uint32_t step = (uint32_t)p->step;
        propose_kernel<<<blocks((int64_t)C * ((n_u + 3) / 4), 128), 128, 0, c->stream>>>(p->U, p->Up, p->stdv, C, n_u, p->rho,
                                                                                        p->beta, k0, k1, step);
        PM_CUDA(cudaGetLastError(), "propose");
        count_launch(c);
        idx_h.clear();
        if (da) {
            screen_input_kernel<<<blocks((int64_t)C * n_u, 256), 256, 0, c->stream>>>(p->Up, p->shift, p->scale, C, n_u, p->X);
            PM_CUDA(cudaGetLastError(), "screen input");
            count_launch(c);
            if ((rc = pm_surrogate_infer(c, p->screen, p->X, C, p->Gs, PM_DEVICE_PTRS | PM_ASYNC))) return rc;
            stage1_kernel<<<blocks(C, 128), 128, 0, c->stream>>>(p->y, p->Gs, C, n_obs, inv2s2, p->PhiS, p->PhiS_new,
                                                                  p->pass, k0, k1, step);
            PM_CUDA(cudaGetLastError(), "stage 1");
            count_launch(c);
            PM_CUDA(cudaMemcpyAsync(pass_h.data(), p->pass, sizeof(int) * (size_t)C, cudaMemcpyDeviceToHost, c->stream), "copy pass");
            PM_CUDA(cudaStreamSynchronize(c->stream), "stage 1");
            for (int q = 0; q < C; ++q)
                if (pass_h[(size_t)q]) idx_h.push_back(q);
            s.stage1_accepts += (int64_t)idx_h.size();
        } else {
            for (int q = 0; q < C; ++q) idx_h.push_back(q);
        }
        if (!idx_h.empty()) {
            if ((rc = forward_listed(c, p, idx_h))) return rc;
            s.forward_evals += (int64_t)idx_h.size();
            accept_kernel<<<blocks((int64_t)idx_h.size(), 128), 128, 0, c->stream>>>(
                p->idx, (int)idx_h.size(), p->y, p->G, n_obs, inv2s2, da ? 1 : 0, p->Phi, p->PhiS, p->PhiS_new, p->U,
                p->Up, n_u, k0, k1, step, p->accepts, p->stdv, p->jump);
            PM_CUDA(cudaGetLastError(), "accept");
            count_launch(c);
        }
        accumulate_kernel<<<blocks(n_u, 128), 128, 0, c->stream>>>(p->U, C, n_u, p->sum_u);
        PM_CUDA(cudaGetLastError(), "accumulate");
        count_launch(c);
        p->step += 1;
        p->n_summed += C;
        s.steps += 1;
        s.proposals += C;
    }
    PM_CUDA(cudaEventRecord(e1, c->stream), "event");
    unsigned long long acc = 0;
    std::vector<double> jump_h((size_t)C);
    PM_CUDA(cudaMemcpyAsync(&acc, p->accepts, 8, cudaMemcpyDeviceToHost, c->stream), "copy accepts");
    PM_CUDA(cudaMemcpyAsync(jump_h.data(), p->jump, sizeof(double) * (size_t)C, cudaMemcpyDeviceToHost, c->stream),
            "copy jumps");
    PM_CUDA(cudaStreamSynchronize(c->stream), "pcn");
    for (int q = 0; q < C; ++q) s.sq_jump += jump_h[(size_t)q];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s.accepts = (int64_t)acc;
    s.seconds = ms / 1e3;
    if (st) *st = s;
    return PM_OK;
}

int pm_pcn_state(pm_ctx* c, const pm_pcn* p, double* u, double* phi, double* sum_u, int64_t* n_summed)
{
    if (!c || !p) return fail(PM_EINVAL, "NULL argument");
    int rc = set_device(c);
    if (rc) return rc;
    if (u) PM_CUDA(cudaMemcpyAsync(u, p->U, sizeof(double) * (size_t)p->C * p->n_u, cudaMemcpyDeviceToHost, c->stream), "copy u");
    if (phi) PM_CUDA(cudaMemcpyAsync(phi, p->Phi, sizeof(double) * (size_t)p->C, cudaMemcpyDeviceToHost, c->stream), "copy phi");
    if (sum_u) PM_CUDA(cudaMemcpyAsync(sum_u, p->sum_u, sizeof(double) * (size_t)p->n_u, cudaMemcpyDeviceToHost, c->stream), "copy sums");
    PM_CUDA(cudaStreamSynchronize(c->stream), "pcn state");
    if (n_summed) *n_summed = p->n_summed;
    return PM_OK;
}

}  // extern "C"
