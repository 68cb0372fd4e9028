// pm_batched_api.cu -- pm_forward_batched: validation, workspace layout, and
// the captured CUDA graph {copies, coefficient staging, row preparation,
// persistent kernel, reduction, copies} replayed for calls of the same shape.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/pm.h"
#include "pm_internal.h"
#include "pm_launch.h"

using namespace pm;

namespace {

constexpr int kBatchWarpsHost = 4;  // must match kBatchWarps of the kernel

cudaError_t launch_batched_K(int K, const BatchKernelParams& p, int grid, cudaStream_t s)
{
    switch (K) {
#define PM_CASE(k) case k: return launch_batched<k>(p, grid, s);
        PM_CASE(0) PM_CASE(1) PM_CASE(2) PM_CASE(3) PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(8) PM_CASE(10)
        PM_CASE(12) PM_CASE(16)
#undef PM_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batched_tc_K(int K, const BatchKernelParams& p, int grid, cudaStream_t s)
{
    switch (K) {
#define PM_CASE(k) case k: return tdtc::launch_batched_tc<k>(p, grid, s);
        PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(8) PM_CASE(10) PM_CASE(12) PM_CASE(16)
        PM_CASE(24) PM_CASE(32) PM_CASE(40) PM_CASE(48) PM_CASE(56) PM_CASE(64)
#undef PM_CASE
    }
    return cudaErrorInvalidValue;
}

int blocks_per_sm_tc_K(int K)
{
    switch (K) {
#define PM_CASE(k) case k: return tdtc::batched_tc_blocks_per_sm<k>();
        PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(8) PM_CASE(10) PM_CASE(12) PM_CASE(16)
        PM_CASE(24) PM_CASE(32) PM_CASE(40) PM_CASE(48) PM_CASE(56) PM_CASE(64)
#undef PM_CASE
    }
    return 1;
}

bool tc_supported(int K) { return K == 4 || K == 5 || K == 6 || K == 8 || K == 10 || K == 12 || K == 16 || wide_K(K); }

int blocks_per_sm_K(int K)
{
    switch (K) {
#define PM_CASE(k) case k: return batched_blocks_per_sm<k>();
        PM_CASE(0) PM_CASE(1) PM_CASE(2) PM_CASE(3) PM_CASE(4) PM_CASE(5) PM_CASE(6) PM_CASE(8) PM_CASE(10)
        PM_CASE(12) PM_CASE(16)
#undef PM_CASE
    }
    return 1;
}

uint64_t fnv(uint64_t h, const void* p, size_t n)
{
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

template <typename T>
uint64_t fnv_val(uint64_t h, const T& v) { return fnv(h, &v, sizeof v); }

}  // namespace

extern "C" int pm_set_graph_mode(pm_ctx* c, int on)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    c->graph_mode = on ? 1 : 0;
    return PM_OK;
}

extern "C" int pm_forward_batched(pm_ctx* c, const pm_batch* bt, uint32_t flags, double* mean, double* var,
                                  int64_t* n_unexited)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    if (!bt) return fail(PM_EINVAL, "batch is NULL");
    if (flags & PM_FP64) return fail(PM_EINVAL, "the batched map runs float paths only (PM_FP64 unsupported)");
    const int K = bt->K, B = bt->B;
    // The wide bounds run on the tensor cores only: the FP32-pipe kernel keeps
    // one velocity table per warp in shared memory, too large above K = 16.
    if (wide_K(K) && !(flags & PM_TENSOR))
        return fail(PM_EINVAL, "K=%d: the batched map runs the wide bounds with PM_TENSOR only", K);
    if (!supported_K(K) && !wide_K(K))
        return fail(PM_EINVAL, "K=%d is not one of the compiled bounds 0..6, 8, 10, 12, 16 (24, 32, 40, 48, 56, 64 with PM_TENSOR)", K);
    if (B < 1 || B > 65535) return fail(PM_EINVAL, "B must be in [1, 65535]");
    if (!bt->inst) return fail(PM_EINVAL, "instance array is NULL");
    if (bt->n_rows < 1 || bt->n_rows > ((int64_t)1 << 31)) return fail(PM_EINVAL, "n_rows out of range");
    if (!bt->x || !mean) return fail(PM_EINVAL, "x and mean must not be NULL");
    const bool dev = flags & PM_DEVICE_PTRS;
    const int64_t NU = (int64_t)(2 * K + 1) * (2 * K + 1) - 1;
    const int TS = table_size(K);

    // Instances: checks, row tiling, path layout.
    bool any_td = false, any_dir = false;
    int64_t total = 0, max_obs = 0;
    std::vector<std::pair<int64_t, int64_t>> ranges;
    std::vector<int64_t> path_base((size_t)B);
    for (int b = 0; b < B; ++b) {
        const pm_instance& I = bt->inst[b];
        if (I.kind != PM_KIND_TIMEDEP && I.kind != PM_KIND_DIRICHLET) return fail(PM_EINVAL, "instance %d: bad kind", b);
        if (!(std::isfinite(I.kappa) && I.kappa >= 0)) return fail(PM_EINVAL, "instance %d: kappa must be finite and >= 0", b);
        if (!(std::isfinite(I.dt) && I.dt > 0)) return fail(PM_EINVAL, "instance %d: dt must be finite and > 0", b);
        if (I.n_obs < 1 || I.n_obs > 0x7fffffff || I.M < 1 || I.M > ((int64_t)1 << 32))
            return fail(PM_EINVAL, "instance %d: need n_obs >= 1 and 1 <= M <= 2^32", b);
        if (I.row0 < 0 || I.row0 + I.n_obs > bt->n_rows) return fail(PM_EINVAL, "instance %d: rows out of range", b);
        if (NU > 0 && !I.u) return fail(PM_EINVAL, "instance %d: coefficients are NULL", b);
        if (I.kind == PM_KIND_DIRICHLET) {
            any_dir = true;
            if (!std::isfinite(I.drift_scale)) return fail(PM_EINVAL, "instance %d: drift_scale must be finite", b);
            if (I.max_steps < 1 || I.max_steps > 0x7fffffffLL) return fail(PM_EINVAL, "instance %d: max_steps out of range", b);
        } else {
            any_td = true;
        }
        if (NU > 0 && dev && !is_device_pointer(I.u, c->device)) return fail(PM_EINVAL, "instance %d: u is not device memory", b);
        if (NU > 0 && !dev && !finite_array(I.u, NU)) return fail(PM_EINVAL, "instance %d: coefficients not finite", b);
        if (I.n_obs > ((int64_t)1 << 62) / I.M) return fail(PM_EINVAL, "instance %d: too many paths", b);
        ranges.push_back({I.row0, I.n_obs});
        path_base[(size_t)b] = total;
        total += I.n_obs * I.M;
        max_obs = std::max(max_obs, I.n_obs);
    }
    std::sort(ranges.begin(), ranges.end());
    int64_t expect = 0;
    for (auto& r : ranges) {
        if (r.first != expect) return fail(PM_EINVAL, "instance rows must tile [0, n_rows) without gaps or overlap");
        expect = r.first + r.second;
    }
    if (expect != bt->n_rows) return fail(PM_EINVAL, "instance rows must tile [0, n_rows) without gaps or overlap");
    if (any_td && !bt->t) return fail(PM_EINVAL, "t is NULL but a time-dependent instance is present");
    const pm_fourier* th = bt->theta0;
    if (any_td) {
        if (!th || th->n < 0 || th->n > PM_MAX_THETA0_MODES) return fail(PM_EINVAL, "theta0 missing or too many modes");
        if (th->n > 0 && (!th->k || !th->a || !th->b || !finite_array(th->a, th->n) || !finite_array(th->b, th->n)))
            return fail(PM_EINVAL, "theta0 arrays NULL or not finite");
    }
    const pm_dirichlet_data* gd = bt->disk;
    if (any_dir) {
        if (!gd || !(std::isfinite(gd->R) && gd->R > 0) || !std::isfinite(gd->quad) || !std::isfinite(gd->f_const))
            return fail(PM_EINVAL, "disk data missing or not finite");
        if (gd->n_ang < 0 || gd->n_ang > PM_MAX_BOUNDARY_MODES) return fail(PM_EINVAL, "n_ang out of range");
        if (gd->n_ang > 0 && (!gd->a || !gd->b || !finite_array(gd->a, gd->n_ang) || !finite_array(gd->b, gd->n_ang)))
            return fail(PM_EINVAL, "boundary arrays NULL or not finite");
    }
    int rc = check_ptrs(c, flags, {bt->x, bt->t, mean, var, n_unexited});
    if (rc) return rc;
    if (!dev && !finite_array(bt->x, 2 * bt->n_rows)) return fail(PM_EINVAL, "x contains NaN or Inf");
    if ((rc = set_device(c))) return rc;

    // Device workspace.
    const int64_t n_rows = bt->n_rows;
    struct WS {
        BatchInstDev* inst; float* tables; RowRec* rows; unsigned long long* ctr; double* g;
        double* U; double* xt; double* mean; double* var;
    };
    auto layout = [&](Bump& bp) {
        WS w{};
        w.inst = bp.take<BatchInstDev>((size_t)B);
        w.tables = bp.take<float>((size_t)B * TS);
        w.rows = bp.take<RowRec>((size_t)n_rows);
        w.ctr = bp.take<unsigned long long>((size_t)B + 4);  // next_path[B], unexited, error flag, steps, tc flag
        w.g = bp.take<double>((size_t)total);
        if (!dev) {
            w.U = bp.take<double>((size_t)(B * std::max<int64_t>(NU, 1)));
            w.xt = bp.take<double>((size_t)(3 * n_rows));
            w.mean = bp.take<double>((size_t)n_rows);
            w.var = bp.take<double>((size_t)n_rows);
        }
        return w;
    };
    Bump probe(nullptr);
    layout(probe);
    if ((rc = ensure_workspace(c, probe.off))) return rc;
    // Pinned staging: instance records, host inputs, host outputs, flags.
    struct HS { BatchInstDev* inst; double* U; double* xt; double* out; unsigned long long* flags; };
    auto hlayout = [&](Bump& bp) {
        HS h{};
        h.inst = bp.take<BatchInstDev>((size_t)B);
        if (!dev) {
            h.U = bp.take<double>((size_t)(B * std::max<int64_t>(NU, 1)));
            h.xt = bp.take<double>((size_t)(3 * n_rows));
            h.out = bp.take<double>((size_t)(2 * n_rows));
        }
        h.flags = bp.take<unsigned long long>(4);
        return h;
    };
    Bump hprobe(nullptr);
    hlayout(hprobe);
    if ((rc = ensure_host(c, hprobe.off))) return rc;
    Bump bw(c->ws), bh(c->host);
    const WS W = layout(bw);
    const HS Hs = hlayout(bh);

    // The previous replay may still read the pinned staging: wait before rewriting it.
    PM_CUDA(cudaStreamSynchronize(c->stream), "batched: wait for previous call");
    for (int b = 0; b < B; ++b) {
        const pm_instance& I = bt->inst[b];
        BatchInstDev d{};
        d.u = dev ? I.u : (W.U + (size_t)b * std::max<int64_t>(NU, 1));
        d.kind = I.kind;
        d.n_obs = (int32_t)I.n_obs;
        d.M = I.M;
        d.row0 = I.row0;
        d.path_base = path_base[(size_t)b];
        d.n_paths = I.n_obs * I.M;
        d.max_steps = I.kind == PM_KIND_DIRICHLET ? I.max_steps : 0;
        d.dt = I.dt;
        d.kappa = I.kappa;
        d.drift_scale = I.kind == PM_KIND_DIRICHLET ? I.drift_scale : 1.0;
        d.key0 = (uint32_t)(I.seed & 0xffffffffu);
        d.key1 = (uint32_t)(I.seed >> 32);
        d.stream = I.stream;
        Hs.inst[b] = d;
        if (!dev && NU > 0) memcpy(Hs.U + (size_t)b * NU, I.u, (size_t)NU * 8);
    }
    if (!dev) {
        memcpy(Hs.xt, bt->x, (size_t)n_rows * 16);
        if (bt->t) memcpy(Hs.xt + 2 * n_rows, bt->t, (size_t)n_rows * 8);
        else memset(Hs.xt + 2 * n_rows, 0, (size_t)n_rows * 8);
    }

    // Kernel parameters (theta0 and disk data travel in the parameter bank).
    BatchKernelParams p;
    memset(&p, 0, sizeof p);
    p.th.n = any_td ? th->n : 0;
    for (int q = 0; q < p.th.n; ++q) {
        p.th.k1[q] = th->k[2 * q];
        p.th.k2[q] = th->k[2 * q + 1];
        p.th.a[q] = (float)th->a[q];
        p.th.b[q] = (float)th->b[q];
    }
    p.R = any_dir ? gd->R : 1.0;
    p.quad = any_dir ? gd->quad : 0.0;
    p.f_const = any_dir ? gd->f_const : 0.0;
    p.n_ang = any_dir ? gd->n_ang : 0;
    for (int m = 0; m < p.n_ang; ++m) { p.ga[m] = gd->a[m]; p.gb[m] = gd->b[m]; }
    const double R2 = p.R * p.R;
    p.R2hi = (float)R2;
    p.R2lo = (float)(R2 - (double)p.R2hi);
    p.band = std::ldexp(p.R2hi, -16);
    p.inst = W.inst;
    p.rows = W.rows;
    p.tables = W.tables;
    p.next_path = W.ctr;
    p.n_unexited = W.ctr + B;
    p.steps = W.ctr + B + 2;
    p.tc_err = (unsigned*)(W.ctr + B + 3);
    const bool use_tc = (flags & PM_TENSOR) && tc_supported(K);
    p.g = W.g;
    p.B = B;
    const int resident = use_tc ? blocks_per_sm_tc_K(K) : blocks_per_sm_K(K);  // also sets the shared-memory attribute
    const int per_sm = tuned_ctas_per_sm(c, PM_TUNE_BATCHED, K, use_tc ? PM_TENSOR : 0u, resident);
    p.refill_pairs = use_tc ? tuned_refill_pairs(c, PM_TUNE_BATCHED, K, PM_TENSOR, kBatchedRefillPairs) : 1;
    int64_t grid = (int64_t)per_sm * c->sm_count;
    const int64_t need = (total + kBatchWarpsHost * 32 - 1) / (kBatchWarpsHost * 32);
    grid = std::max<int64_t>(1, std::min(grid, need));
    c->last_grid = grid;

    const double* dx = dev ? bt->x : W.xt;
    const double* dt_ = dev ? bt->t : W.xt + 2 * n_rows;
    double* dmean = dev ? mean : W.mean;
    double* dvar = dev ? var : (var ? W.var : nullptr);
    unsigned* derr = (unsigned*)(W.ctr + B + 1);

    auto enqueue = [&]() -> cudaError_t {
        cudaStream_t s = c->stream;
        cudaError_t e = cudaMemcpyAsync(W.inst, Hs.inst, sizeof(BatchInstDev) * (size_t)B, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !dev && NU > 0)
            e = cudaMemcpyAsync(W.U, Hs.U, (size_t)(B * NU) * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(W.xt, Hs.xt, (size_t)n_rows * 24, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(W.ctr, 0, sizeof(unsigned long long) * ((size_t)B + 4), s);
        if (e == cudaSuccess) e = launch_stage_tables(W.inst, B, K, W.tables, s);
        if (e == cudaSuccess) e = launch_prep_rows(W.inst, B, (int)max_obs, dx, any_td ? dt_ : dx, W.rows, derr, s);
        if (e == cudaSuccess) e = use_tc ? launch_batched_tc_K(K, p, (int)grid, s) : launch_batched_K(K, p, (int)grid, s);
        if (e == cudaSuccess) e = launch_reduce_rows(W.inst, B, (int)max_obs, W.g, dmean, dvar, s);
        if (e == cudaSuccess && !dev) {
            e = cudaMemcpyAsync(Hs.out, W.mean, (size_t)n_rows * 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && var) e = cudaMemcpyAsync(Hs.out + n_rows, W.var, (size_t)n_rows * 8, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess && dev && n_unexited)
            e = cudaMemcpyAsync(n_unexited, W.ctr + B, 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Hs.flags, W.ctr + B, 32, cudaMemcpyDeviceToHost, s);
        return e;
    };
    // prep_rows reads t only for time-dependent instances; when there are none
    // x stands in for t so that the pointer is valid.

    // Shape key of the call: everything the captured graph bakes in.
    uint64_t key = 1469598103934665603ull;
    key = fnv_val(key, c->ws); key = fnv_val(key, c->host); key = fnv_val(key, K); key = fnv_val(key, B);
    key = fnv_val(key, n_rows); key = fnv_val(key, total); key = fnv_val(key, grid); key = fnv_val(key, dev);
    key = fnv_val(key, (const void*)bt->x); key = fnv_val(key, (const void*)bt->t);
    key = fnv_val(key, (const void*)mean); key = fnv_val(key, (const void*)var); key = fnv_val(key, (const void*)n_unexited);
    key = fnv(key, &p, sizeof p);
    key = fnv_val(key, use_tc);
    for (int b = 0; b < B; ++b) {
        const pm_instance& I = bt->inst[b];
        key = fnv_val(key, I.kind); key = fnv_val(key, I.row0); key = fnv_val(key, I.n_obs); key = fnv_val(key, I.M);
    }
    const bool capturable = c->graph_mode && c->stream != cudaStreamLegacy && c->stream != nullptr;
    if (capturable) {
        if (!c->graph_exec || c->graph_key != key) {
            if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
            cudaGraph_t graph = nullptr;
            PM_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e = enqueue();
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
            if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "batched capture"); }
            if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
            e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { c->graph_exec = nullptr; return cuda_fail(e, "graph instantiate"); }
            c->graph_key = key;
        }
        PM_CUDA(cudaGraphLaunch(c->graph_exec, c->stream), "graph launch");
    } else {
        cudaError_t e = enqueue();
        if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    }
    count_launch(c, 4);
    c->last_steps = -1;
    if (dev && (flags & PM_ASYNC)) return PM_OK;
    PM_CUDA(cudaStreamSynchronize(c->stream), "batched");
    c->last_steps = (int64_t)Hs.flags[2];
    if (!dev) {
        memcpy(mean, Hs.out, (size_t)n_rows * 8);
        if (var) memcpy(var, Hs.out + n_rows, (size_t)n_rows * 8);
        if (n_unexited) *n_unexited = (int64_t)Hs.flags[0];
    }
    if (Hs.flags[1] & 0xffffffffull)
        return fail(PM_EINVAL, "observation points or times are not finite, a time is negative, or a step count exceeds 2^31");
    if (Hs.flags[3] & 0xffffffffull) return fail(PM_ETIMEOUT, "a tensor-core wait in the batched kernel timed out");
    return Hs.flags[0] ? PM_WARN_UNEXITED : PM_OK;
}

// Autotuning of the batched kernel's persistent grid (pm_autotune.cu).
extern "C" int pm_autotune_batched(pm_ctx* c, const pm_batch* bt, uint32_t flags, int32_t* best_ctas_per_sm)
{
    if (!c || !bt) return fail(PM_EINVAL, "ctx or batch is NULL");
    if (bt->n_rows < 1 || bt->B < 1) return fail(PM_EINVAL, "autotuning needs a non-empty batch");
    if (!supported_K(bt->K) && !(wide_K(bt->K) && (flags & PM_TENSOR)))
        return fail(PM_EINVAL, "unsupported K %d (24 ... 64 with PM_TENSOR only)", bt->K);
    int rc = set_device(c);
    if (rc) return rc;
    flags &= ~PM_ASYNC;
    const bool dev = flags & PM_DEVICE_PTRS;
    const int K = bt->K;
    const bool use_tc = (flags & PM_TENSOR) && tc_supported(K);
    const int resident = use_tc ? blocks_per_sm_tc_K(K) : blocks_per_sm_K(K);
    std::vector<double> hmean;
    double* mean = nullptr;
    if (dev) {
        PM_CUDA(cudaMalloc(&mean, (size_t)bt->n_rows * 8), "autotune output");
    } else {
        hmean.resize((size_t)bt->n_rows);
        mean = hmean.data();
    }
    auto run = [&]() { return pm_forward_batched(c, bt, flags, mean, nullptr, nullptr); };
    rc = autotune_loop(c, PM_TUNE_BATCHED, K, use_tc ? PM_TENSOR : 0u, resident, use_tc, run, best_ctas_per_sm);
    if (dev) cudaFree(mean);
    return rc;
}
