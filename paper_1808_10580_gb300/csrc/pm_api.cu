// pm_api.cu -- the C ABI of include/pm.h: argument checking, coefficient
// staging, workspace management and kernel sequencing.  Every arithmetic step
// of the forward maps runs in the CUDA kernels (pm_kernels.cuh,
// pm_support.cu); the host only validates, stages and copies.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pm.h"
#include "pm_internal.h"
#include "pm_launch.h"

using namespace pm;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
namespace {
thread_local char g_err[512] = "";
}  // namespace

namespace pm {
int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(PM_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(PM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool supported_K(int K)
{
    switch (K) {
    case 0: case 1: case 2: case 3: case 4: case 5: case 6: case 8: case 10: case 12: case 16: return true;
    default: return false;
    }
}
}  // namespace pm

namespace {

#define PM_K_LIST(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(8) X(10) X(12) X(16)

template <typename Real>
cudaError_t dispatch_timedep(int K, const TimedepLaunch& L, cudaStream_t s)
{
    switch (K) {
#define PM_CASE(k) case k: return launch_timedep<Real, k>(L, s);
        PM_K_LIST(PM_CASE)
#undef PM_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t dispatch_dirichlet(int K, const DirichletLaunch& L, cudaStream_t s)
{
    switch (K) {
#define PM_CASE(k) case k: return launch_dirichlet<Real, k>(L, s);
        PM_K_LIST(PM_CASE)
#undef PM_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
int dispatch_dirichlet_occupancy(int K)
{
    switch (K) {
#define PM_CASE(k) case k: return dirichlet_blocks_per_sm<Real, k>();
        PM_K_LIST(PM_CASE)
#undef PM_CASE
    }
    return 1;
}

template <typename Real>
cudaError_t dispatch_velocity(int K, const double* coef, const double* x, int64_t n, double* v, cudaStream_t s)
{
    switch (K) {
#define PM_CASE(k) case k: return launch_velocity<Real, k>(coef, x, n, v, s);
        PM_K_LIST(PM_CASE)
#undef PM_CASE
    }
    return cudaErrorInvalidValue;
}

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Half-mode index of (m, n) in the coefficient layout of pm_field.
inline int64_t half_index(int K, int m, int n) { return m == 0 ? (n - 1) : K + (int64_t)(m - 1) * (2 * K + 1) + (n + K); }

}  // namespace

namespace pm {

// Section 4.1, Eq. v_expand: stream-function coefficients (a_h, b_h) of the
// half-plane modes -> the product-basis velocity table the kernels read.
// For m, n >= 1 the pair (m, n), (m, -n) folds into
//   A = a(m,n) + a(m,-n), B = b(m,n) - b(m,-n), G = b(m,n) + b(m,-n), D = a(m,-n) - a(m,n)
// (psi = A C1 C2 + B C1 S2 + G S1 C2 + D S1 S2); then e = 2 pi n (A, -B, G, -D)
// feed v1 = -d2 psi and f = 2 pi m (G, D, -A, -B) feed v2 = d1 psi.
void stage_coefficients_into(int K, const double* u, double* tab)
{
    for (int q = 0; q < table_size(K); ++q) tab[q] = 0.0;
    auto a = [&](int m, int n) { return u[2 * half_index(K, m, n)]; };
    auto b = [&](int m, int n) { return u[2 * half_index(K, m, n) + 1]; };
    for (int m = 0; m <= K; ++m) {
        for (int n = 0; n <= K; ++n) {
            double A = 0, B = 0, G = 0, D = 0;
            if (m == 0 && n == 0) continue;
            if (m == 0) { A = a(0, n); B = b(0, n); }
            else if (n == 0) { A = a(m, 0); G = b(m, 0); }
            else {
                A = a(m, n) + a(m, -n);
                B = b(m, n) - b(m, -n);
                G = b(m, n) + b(m, -n);
                D = a(m, -n) - a(m, n);
            }
            double* e = &tab[(size_t)(m * (K + 1) + n) * 8];
            const double sn = kTwoPi * n, sm = kTwoPi * m;
            e[0] = sn * A; e[1] = -sn * B; e[2] = sn * G; e[3] = -sn * D;
            e[4] = sm * G; e[5] = sm * D; e[6] = -sm * A; e[7] = -sm * B;
        }
    }
}

}  // namespace pm

namespace {

std::vector<double> stage_coefficients(int K, const double* u)
{
    std::vector<double> tab((size_t)table_size(K), 0.0);
    pm::stage_coefficients_into(K, u, tab.data());
    return tab;
}

}  // namespace

namespace pm {
bool finite_array(const double* p, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Device (or managed) memory that belongs to `device`: a pointer into another
// GPU's memory is rejected, since the kernels would read it over the peer
// link or fault.
bool is_device_pointer(const void* p, int device)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == device;
}
}  // namespace pm

// Records a message for pm_last_error() from other translation units.
int pm::set_error(int code, const char* msg) { return fail(code, "%s", msg); }

// ---------------------------------------------------------------------------
// Context helpers (pm_internal.h)
// ---------------------------------------------------------------------------
namespace pm {

int ensure_workspace(pm_ctx* c, size_t bytes)
{
    if (bytes <= c->ws_size) return PM_OK;
    if (c->ws) {
        PM_CUDA(cudaStreamSynchronize(c->stream), "workspace resize");
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_size = 0;
    }
    size_t want = bytes + bytes / 4 + 4096;
    PM_CUDA(cudaMalloc(&c->ws, want), "device workspace");
    c->ws_size = want;
    return PM_OK;
}

int ensure_host(pm_ctx* c, size_t bytes)
{
    if (bytes <= c->host_size) return PM_OK;
    if (c->host) {
        PM_CUDA(cudaStreamSynchronize(c->stream), "staging resize");
        cudaFreeHost(c->host);
        c->host = nullptr;
        c->host_size = 0;
    }
    size_t want = bytes + bytes / 4 + 4096;
    PM_CUDA(cudaHostAlloc(&c->host, want, cudaHostAllocDefault), "pinned staging");
    c->host_size = want;
    return PM_OK;
}

int set_device(pm_ctx* c)
{
    PM_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    return PM_OK;
}

// Common checks of a field description.
int check_field(const pm_field* f, bool allow_wide, bool allow_simt_wide)
{
    if (!f) return fail(PM_EINVAL, "field is NULL");
    if ((allow_wide && wide_K(f->K)) || (allow_simt_wide && simt_wide_K(f->K))) {
        // accepted: float paths (checked by the caller)
    } else if (!supported_K(f->K)) {
        return fail(PM_EINVAL, "K=%d is not one of the compiled bounds 0..6, 8, 10, 12, 16%s%s", f->K,
                    allow_wide ? " (24, 32, 40, 48, 56, 64: float paths)" : "",
                    allow_simt_wide ? " (80: float paths on the FP32 pipes)" : "");
    }
    const int64_t nu = (int64_t)(2 * f->K + 1) * (2 * f->K + 1) - 1;
    if (nu > 0 && !f->u) return fail(PM_EINVAL, "field coefficients are NULL");
    if (nu > 0 && !finite_array(f->u, nu)) return fail(PM_EINVAL, "field coefficients contain NaN or Inf");
    return PM_OK;
}

int check_ptrs(const pm_ctx* c, uint32_t flags, std::initializer_list<const void*> ptrs)
{
    if (!(flags & PM_DEVICE_PTRS)) return PM_OK;
    for (const void* p : ptrs)
        if (p && !is_device_pointer(p, c->device))
            return fail(PM_EINVAL, "PM_DEVICE_PTRS is set but a pointer is not device memory of the context's device %d",
                        c->device);
    return PM_OK;
}

int check_theta0(const pm_fourier* th)
{
    if (!th) return fail(PM_EINVAL, "theta0 is NULL");
    if (th->n < 0 || th->n > PM_MAX_THETA0_MODES) return fail(PM_EINVAL, "theta0 has %d modes (max %d)", th->n, PM_MAX_THETA0_MODES);
    if (th->n > 0 && (!th->k || !th->a || !th->b)) return fail(PM_EINVAL, "theta0 arrays are NULL");
    if (th->n > 0 && (!finite_array(th->a, th->n) || !finite_array(th->b, th->n)))
        return fail(PM_EINVAL, "theta0 amplitudes contain NaN or Inf");
    // The float kernels reduce the phase k.x modulo 1 in float: exact only
    // while |k| x stays far below 2^23.
    for (int q = 0; q < th->n; ++q)
        if (std::abs(th->k[2 * q]) > 4096 || std::abs(th->k[2 * q + 1]) > 4096)
            return fail(PM_EINVAL, "theta0 wave number out of range (|k| <= 4096)");
    return PM_OK;
}

void count_launch(pm_ctx* c, int n) { c->launches += n; }

uint32_t take_wait_limit(pm_ctx* c)
{
    const int64_t v = c->wait_limit_next;
    c->wait_limit_next = -1;
    return v < 0 ? kWaitPolls : (uint32_t)v;
}

}  // namespace pm

extern "C" {

int pm_version(void) { return 10000; }

const char* pm_last_error(void) { return g_err; }

int pm_create(pm_ctx** out, int device, void* cuda_stream)
{
    if (!out) return fail(PM_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(PM_EINVAL, "device %d out of range (%d devices)", device, ndev);
    pm_ctx* c = new (std::nothrow) pm_ctx;
    if (!c) return fail(PM_ENOMEM, "context allocation");
    c->device = device;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) c->stream = (cudaStream_t)cuda_stream;
        else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    cudaDeviceProp prop{};
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        pm_destroy(c);
        return cuda_fail(e, "pm_create");
    }
    c->device_name = prop.name;
    load_tune_cache(c);
    *out = c;
    return PM_OK;
}

void pm_destroy(pm_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->ws) cudaFree(c->ws);
    if (c->host) cudaFreeHost(c->host);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

void* pm_stream(const pm_ctx* c) { return c ? (void*)c->stream : nullptr; }

int pm_set_kernel_timing(pm_ctx* c, int on)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    c->timing = on != 0;
    c->timed = false;
    return PM_OK;
}

float pm_last_kernel_ms(pm_ctx* c)
{
    if (!c || !c->timed) return -1.0f;
    if (cudaEventSynchronize(c->ev1) != cudaSuccess) return -1.0f;
    float ms = -1.0f;
    if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) != cudaSuccess) return -1.0f;
    return ms;
}

int64_t pm_launch_count(const pm_ctx* c) { return c ? c->launches : 0; }

int pm_set_wait_limit(pm_ctx* c, int64_t polls)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    c->wait_limit_next = polls < 0 ? -1 : (polls > (int64_t)kWaitPolls ? (int64_t)kWaitPolls : polls);
    return PM_OK;
}

int64_t pm_last_step_count(const pm_ctx* c) { return c ? c->last_steps : -1; }

int64_t pm_last_grid(const pm_ctx* c) { return c ? c->last_grid : 0; }

// ---------------------------------------------------------------------------
// Observation groups that share paths (PM_SHARE_PATHS): observations at
// bit-identical x, members sorted by step count then index, the RNG stream
// the lowest member index; groups in launch order (largest step count first,
// then by stream).  Step counts as the prep kernel forms them.
// ---------------------------------------------------------------------------
namespace {

struct PathGroups {
    std::vector<int4> groups;      // {m0, m1, stream, nmax}
    std::vector<int32_t> members;  // observation indices, group by group
    int64_t steps_per_path = 0;    // sum of nmax
};

int make_path_groups(const double* x, const double* t, int64_t n, double dt, PathGroups& G)
{
    std::vector<int32_t> N((size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        const double tj = t[j];
        if (!std::isfinite(tj) || tj < 0.0 || !std::isfinite(x[2 * j]) || !std::isfinite(x[2 * j + 1])) return PM_EINVAL;
        const double steps = tj > 0.0 ? std::ceil(tj / dt - 1e-9) : 0.0;
        if (steps > 2147483646.0) return PM_EINVAL;
        N[(size_t)j] = (int32_t)steps;
    }
    auto bits = [&](int64_t j, int c) {
        uint64_t b;
        memcpy(&b, &x[2 * j + c], 8);
        return b;
    };
    std::vector<int32_t> idx((size_t)n);
    for (int64_t j = 0; j < n; ++j) idx[(size_t)j] = (int32_t)j;
    std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
        const uint64_t a1 = bits(a, 0), b1 = bits(b, 0);
        if (a1 != b1) return a1 < b1;
        const uint64_t a2 = bits(a, 1), b2 = bits(b, 1);
        if (a2 != b2) return a2 < b2;
        if (N[(size_t)a] != N[(size_t)b]) return N[(size_t)a] < N[(size_t)b];
        return a < b;
    });
    std::vector<int4> runs;  // m0, m1 over idx, stream, nmax
    for (size_t s = 0; s < (size_t)n;) {
        size_t e = s + 1;
        while (e < (size_t)n && bits(idx[e], 0) == bits(idx[s], 0) && bits(idx[e], 1) == bits(idx[s], 1)) ++e;
        int32_t stream = idx[s];
        for (size_t k = s; k < e; ++k) stream = std::min(stream, idx[k]);
        runs.push_back(make_int4((int)s, (int)e, stream, N[(size_t)idx[e - 1]]));
        s = e;
    }
    std::stable_sort(runs.begin(), runs.end(), [](const int4& a, const int4& b) {
        if (a.w != b.w) return a.w > b.w;
        return a.z < b.z;
    });
    G.groups.clear();
    G.members.clear();
    G.steps_per_path = 0;
    for (const int4& r : runs) {
        const int m0 = (int)G.members.size();
        for (int k = r.x; k < r.y; ++k) G.members.push_back(idx[(size_t)k]);
        G.groups.push_back(make_int4(m0, (int)G.members.size(), r.z, r.w));
        G.steps_per_path += r.w;
    }
    return PM_OK;
}

}  // namespace

int pm_path_groups(const double* x, const double* t, int64_t n_obs, double dt, int32_t* group_of, int32_t* stream_of,
                   int64_t* n_groups, int64_t* steps_per_path)
{
    if (!x || !t || n_obs < 0 || !(std::isfinite(dt) && dt > 0)) return PM_EINVAL;
    PathGroups G;
    const int rc = make_path_groups(x, t, n_obs, dt, G);
    if (rc) return rc;
    for (size_t g = 0; g < G.groups.size(); ++g)
        for (int m = G.groups[g].x; m < G.groups[g].y; ++m) {
            const int32_t j = G.members[(size_t)m];
            if (group_of) group_of[j] = (int32_t)g;
            if (stream_of) stream_of[j] = G.groups[g].z;
        }
    if (n_groups) *n_groups = (int64_t)G.groups.size();
    if (steps_per_path) *steps_per_path = G.steps_per_path;
    return PM_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 1
// ---------------------------------------------------------------------------
int pm_forward_timedep(pm_ctx* c, const pm_field* field, double kappa, const pm_fourier* th, const double* x,
                       const double* t, int64_t n_obs, int64_t M, double dt, uint64_t seed, uint32_t flags,
                       double* mean, double* var, const pm_path_opts* opts)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    int rc = check_field(field, true, true);
    if (rc) return rc;
    if ((wide_K(field->K) || simt_wide_K(field->K)) && (flags & PM_FP64))
        return fail(PM_EINVAL, "K=%d runs with float paths only", field->K);
    if ((rc = check_theta0(th))) return rc;
    if (!(std::isfinite(kappa) && kappa >= 0)) return fail(PM_EINVAL, "kappa must be finite and >= 0");
    if (!(std::isfinite(dt) && dt > 0)) return fail(PM_EINVAL, "dt must be finite and > 0");
    if (n_obs < 0) return fail(PM_EINVAL, "n_obs < 0");
    if (n_obs == 0) return PM_OK;
    if (n_obs > (int64_t)1 << 30) return fail(PM_EINVAL, "n_obs too large");
    if (M < 1) return fail(PM_EINVAL, "M must be >= 1");
    const int64_t off = opts ? opts->path_offset : 0;
    if (off < 0 || off + M > ((int64_t)1 << 32)) return fail(PM_EINVAL, "path_offset + M exceeds 2^32");
    if (!x || !t || !mean) return fail(PM_EINVAL, "x, t and mean must not be NULL");
    double* g_out = opts ? opts->g_out : nullptr;
    double* x_out = opts ? opts->x_out : nullptr;
    if ((rc = check_ptrs(c, flags, {x, t, mean, var, g_out, x_out}))) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    const bool fp64 = flags & PM_FP64;
    const int K = field->K;
    const bool tc = !fp64 && (flags & PM_TENSOR) && (K == 4 || K == 5 || K == 6 || K == 8 || K == 10 || K == 12 || K == 16 ||
                                                     wide_K(K));
    const bool wide = wide_K(K) || simt_wide_K(K);  // (K = 80: never on the tensor cores, tc is false)
    const int rows = tc ? td_tc_rows(K) : td_simt_rows(K);  // paths per CTA
    const int64_t chunks64 = (M + rows - 1) / rows;
    if (n_obs * chunks64 > 0x7fffffffLL) return fail(PM_EINVAL, "n_obs * ceil(M/%d) exceeds the grid limit", rows);
    const int32_t chunks = (int32_t)chunks64;
    const bool share = flags & PM_SHARE_PATHS;
    if ((rc = set_device(c))) return rc;

    // Shared paths: the groups, from host copies of x and t.
    PathGroups PG;
    if (share) {
        std::vector<double> hx, ht;
        const double *gx = x, *gt = t;
        if (dev) {
            hx.resize((size_t)(2 * n_obs));
            ht.resize((size_t)n_obs);
            PM_CUDA(cudaMemcpyAsync(hx.data(), x, (size_t)n_obs * 16, cudaMemcpyDeviceToHost, c->stream), "copy x");
            PM_CUDA(cudaMemcpyAsync(ht.data(), t, (size_t)n_obs * 8, cudaMemcpyDeviceToHost, c->stream), "copy t");
            PM_CUDA(cudaStreamSynchronize(c->stream), "copy x, t");
            gx = hx.data();
            gt = ht.data();
        }
        if (make_path_groups(gx, gt, n_obs, dt, PG))
            return fail(PM_EINVAL, "observation points or times are not finite, a time is negative, or a step count exceeds 2^31");
    }

    // Workspace layout.
    const bool sort = n_obs <= 8192 && !share;
    auto layout = [&](Bump& b) {
        struct P { unsigned* err; unsigned long long* steps; ObsRec* rec; int32_t* order; double2* part; int4* grp; int32_t* mem; float* tab; double *x, *t, *mean, *var, *g, *xo; } p{};
        p.err = b.take<unsigned>(64);     // error flag, then the step counter 128 bytes on
        p.tab = wide ? b.take<float>((size_t)wide_table_floats(K)) : nullptr;
        p.steps = (unsigned long long*)(p.err ? p.err + 32 : nullptr);
        p.rec = b.take<ObsRec>((size_t)n_obs);
        p.order = sort ? b.take<int32_t>((size_t)n_obs) : nullptr;
        p.part = b.take<double2>((size_t)(n_obs * chunks));
        p.grp = share ? b.take<int4>(PG.groups.size()) : nullptr;
        p.mem = share ? b.take<int32_t>((size_t)n_obs) : nullptr;
        if (!dev) {
            p.x = b.take<double>((size_t)(3 * n_obs));  // x then t, one copy
            p.t = p.x + 2 * n_obs;
            p.mean = b.take<double>((size_t)n_obs);
            p.var = var ? b.take<double>((size_t)n_obs) : nullptr;
            p.g = g_out ? b.take<double>((size_t)(n_obs * M)) : nullptr;
            p.xo = x_out ? b.take<double>((size_t)(2 * n_obs * M)) : nullptr;
        }
        return p;
    };
    Bump probe(nullptr);
    layout(probe);
    if ((rc = ensure_workspace(c, probe.off))) return rc;
    Bump bump(c->ws);
    auto W = layout(bump);

    const double *dx = x, *dtm = t;
    double *dmean = mean, *dvar = var, *dg = g_out, *dxo = x_out;
    size_t hbytes = 0;
    if (!dev) {
        hbytes = (size_t)n_obs * 8 * 3 + 64;
        const size_t outb = (size_t)n_obs * 8 * 2 + (g_out ? (size_t)(n_obs * M) * 8 : 0) +
                            (x_out ? (size_t)(2 * n_obs * M) * 8 : 0) + 64;
        if ((rc = ensure_host(c, hbytes > outb ? hbytes : outb))) return rc;
        double* h = (double*)c->host;
        memcpy(h, x, (size_t)n_obs * 16);
        memcpy(h + 2 * n_obs, t, (size_t)n_obs * 8);
        PM_CUDA(cudaMemcpyAsync(W.x, h, (size_t)n_obs * 24, cudaMemcpyHostToDevice, c->stream), "copy x, t");
        dx = W.x;
        dtm = W.t;
        dmean = W.mean;
        dvar = W.var;
        dg = W.g;
        dxo = W.xo;
    }

    const std::vector<double> tab = stage_coefficients(field->K, field->u);
    PM_CUDA(cudaMemsetAsync(W.err, 0, 256, c->stream), "clear flags");
    PM_CUDA(launch_prep_timedep(dx, dtm, n_obs, dt, kappa, W.rec, W.order, W.err, c->stream, share ? nullptr : W.steps, M),
            "prep kernel");
    c->last_steps = -1;
    count_launch(c, sort ? 2 : 1);
    if (share) {
        PM_CUDA(cudaMemcpyAsync(W.grp, PG.groups.data(), PG.groups.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream),
                "copy groups");
        PM_CUDA(cudaMemcpyAsync(W.mem, PG.members.data(), PG.members.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                c->stream),
                "copy group members");
    }

    TimedepLaunch L{};
    L.coef = tab.data();
    L.nq = th->n;
    L.qk = th->k;
    L.qa = th->a;
    L.qb = th->b;
    L.obs = W.rec;
    L.order = W.order;
    L.part = W.part;
    L.g_out = dg;
    L.x_out = dxo;
    L.dt = dt;
    L.s_dt = std::sqrt(2.0 * kappa * dt);
    L.M = M;
    L.path_offset = off;
    L.n_obs = (int32_t)n_obs;
    L.chunks = chunks;
    L.groups = share ? W.grp : nullptr;
    L.members = share ? W.mem : nullptr;
    L.n_groups = (int32_t)PG.groups.size();
    L.table_dev = W.tab;
    L.wait_limit = take_wait_limit(c);
    c->last_grid = (share ? (int64_t)PG.groups.size() : n_obs) * (int64_t)chunks;
    L.inst = opts ? opts->instance : 0u;
    L.key0 = (uint32_t)(seed & 0xffffffffu);
    L.key1 = (uint32_t)(seed >> 32);
    if (c->timing) PM_CUDA(cudaEventRecord(c->ev0, c->stream), "event");
    cudaError_t e;
    if (tc) {
        switch (K) {
        case 4: e = tdtc::launch_timedep_tc<4>(L, W.err + 1, c->stream); break;
        case 5: e = tdtc::launch_timedep_tc<5>(L, W.err + 1, c->stream); break;
        case 6: e = tdtc::launch_timedep_tc<6>(L, W.err + 1, c->stream); break;
        case 8: e = tdtc::launch_timedep_tc<8>(L, W.err + 1, c->stream); break;
        case 10: e = tdtc::launch_timedep_tc<10>(L, W.err + 1, c->stream); break;
        case 12: e = tdtc::launch_timedep_tc<12>(L, W.err + 1, c->stream); break;
        case 24: e = tdtc::launch_timedep_tc<24>(L, W.err + 1, c->stream); break;
        case 32: e = tdtc::launch_timedep_tc<32>(L, W.err + 1, c->stream); break;
        case 40: e = tdtc::launch_timedep_tc<40>(L, W.err + 1, c->stream); break;
        case 48: e = tdtc::launch_timedep_tc<48>(L, W.err + 1, c->stream); break;
        case 56: e = tdtc::launch_timedep_tc<56>(L, W.err + 1, c->stream); break;
        case 64: e = tdtc::launch_timedep_tc<64>(L, W.err + 1, c->stream); break;
        default: e = tdtc::launch_timedep_tc<16>(L, W.err + 1, c->stream); break;
        }
    } else if (wide) {
        switch (K) {
        case 24: e = launch_timedep<float, 24>(L, c->stream); break;
        case 32: e = launch_timedep<float, 32>(L, c->stream); break;
        case 40: e = launch_timedep<float, 40>(L, c->stream); break;
        case 48: e = launch_timedep<float, 48>(L, c->stream); break;
        case 56: e = launch_timedep<float, 56>(L, c->stream); break;
        case 64: e = launch_timedep<float, 64>(L, c->stream); break;
        case 80: e = launch_timedep<float, 80>(L, c->stream); break;
        default: return fail(PM_EINVAL, "K=%d has no float-path kernel", K);
        }
    } else {
        e = fp64 ? dispatch_timedep<double>(K, L, c->stream) : dispatch_timedep<float>(K, L, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "timedep kernel launch");
    if (c->timing) {
        PM_CUDA(cudaEventRecord(c->ev1, c->stream), "event");
        c->timed = true;
    }
    count_launch(c);
    PM_CUDA(launch_reduce(W.part, n_obs, chunks, M, dmean, dvar, c->stream), "reduce kernel");
    count_launch(c);

    if (dev && (flags & PM_ASYNC)) return PM_OK;
    unsigned err_flag = 0;
    if (!dev) {
        double* h = (double*)c->host;
        size_t o = 0;
        PM_CUDA(cudaMemcpyAsync(h + o, dmean, (size_t)n_obs * 8, cudaMemcpyDeviceToHost, c->stream), "copy mean");
        o += (size_t)n_obs;
        if (var) { PM_CUDA(cudaMemcpyAsync(h + o, dvar, (size_t)n_obs * 8, cudaMemcpyDeviceToHost, c->stream), "copy var"); o += (size_t)n_obs; }
        if (g_out) { PM_CUDA(cudaMemcpyAsync(h + o, dg, (size_t)(n_obs * M) * 8, cudaMemcpyDeviceToHost, c->stream), "copy g"); o += (size_t)(n_obs * M); }
        if (x_out) { PM_CUDA(cudaMemcpyAsync(h + o, dxo, (size_t)(2 * n_obs * M) * 8, cudaMemcpyDeviceToHost, c->stream), "copy x_out"); }
    }
    unsigned long long steps_taken = 0;
    unsigned tc_flag = 0;
    PM_CUDA(cudaMemcpyAsync(&tc_flag, W.err + 1, 4, cudaMemcpyDeviceToHost, c->stream), "copy flags");
    PM_CUDA(cudaMemcpyAsync(&err_flag, W.err, 4, cudaMemcpyDeviceToHost, c->stream), "copy flags");
    PM_CUDA(cudaMemcpyAsync(&steps_taken, W.steps, 8, cudaMemcpyDeviceToHost, c->stream), "copy step count");
    PM_CUDA(cudaStreamSynchronize(c->stream), "timedep");
    c->last_steps = share ? PG.steps_per_path * M : (int64_t)steps_taken;
    if (!dev) {
        const double* h = (const double*)c->host;
        size_t o = 0;
        memcpy(mean, h + o, (size_t)n_obs * 8);
        o += (size_t)n_obs;
        if (var) { memcpy(var, h + o, (size_t)n_obs * 8); o += (size_t)n_obs; }
        if (g_out) { memcpy(g_out, h + o, (size_t)(n_obs * M) * 8); o += (size_t)(n_obs * M); }
        if (x_out) memcpy(x_out, h + o, (size_t)(2 * n_obs * M) * 8);
    }
    if (err_flag) return fail(PM_EINVAL, "observation points or times are not finite, a time is negative, or a step count exceeds 2^31");
    if (tc_flag) return fail(PM_ETIMEOUT, "a tensor-core wait in the particle kernel timed out");
    return PM_OK;
}

// Dirichlet launch shape: the tensor-core kernel for float paths with
// PM_TENSOR at K in {4,5,6,8,10,12,16}; resident CTAs per SM of the kernel used.
namespace {
bool dirichlet_uses_tc(int K, uint32_t flags)
{
    return !(flags & PM_FP64) && (flags & PM_TENSOR) &&
           (K == 4 || K == 5 || K == 6 || K == 8 || K == 10 || K == 12 || K == 16 || wide_K(K));
}

int dirichlet_resident(int K, bool fp64, bool use_tc, bool gen = false)
{
    if (use_tc) {
        switch (K) {
        case 4: return tdtc::dirichlet_tc_blocks_per_sm<4>(gen);
        case 5: return tdtc::dirichlet_tc_blocks_per_sm<5>(gen);
        case 6: return tdtc::dirichlet_tc_blocks_per_sm<6>(gen);
        case 8: return tdtc::dirichlet_tc_blocks_per_sm<8>(gen);
        case 10: return tdtc::dirichlet_tc_blocks_per_sm<10>(gen);
        case 12: return tdtc::dirichlet_tc_blocks_per_sm<12>(gen);
        case 24: return tdtc::dirichlet_tc_blocks_per_sm<24>(gen);
        case 32: return tdtc::dirichlet_tc_blocks_per_sm<32>(gen);
        case 40: return tdtc::dirichlet_tc_blocks_per_sm<40>(gen);
        case 48: return tdtc::dirichlet_tc_blocks_per_sm<48>(gen);
        case 56: return tdtc::dirichlet_tc_blocks_per_sm<56>(gen);
        case 64: return tdtc::dirichlet_tc_blocks_per_sm<64>(gen);
        default: return tdtc::dirichlet_tc_blocks_per_sm<16>(gen);
        }
    }
    switch (K) {
    case 24: return dirichlet_blocks_per_sm<float, 24>();
    case 32: return dirichlet_blocks_per_sm<float, 32>();
    case 40: return dirichlet_blocks_per_sm<float, 40>();
    case 48: return dirichlet_blocks_per_sm<float, 48>();
    case 56: return dirichlet_blocks_per_sm<float, 56>();
    case 64: return dirichlet_blocks_per_sm<float, 64>();
    default: break;
    }
    return fp64 ? dispatch_dirichlet_occupancy<double>(K) : dispatch_dirichlet_occupancy<float>(K);
}

// The wide-K FP32-pipe Dirichlet launch (table in shared memory).
cudaError_t launch_dirichlet_wide(int K, const DirichletLaunch& L, cudaStream_t s)
{
    switch (K) {
    case 24: return launch_dirichlet<float, 24>(L, s);
    case 32: return launch_dirichlet<float, 32>(L, s);
    case 40: return launch_dirichlet<float, 40>(L, s);
    case 48: return launch_dirichlet<float, 48>(L, s);
    case 56: return launch_dirichlet<float, 56>(L, s);
    case 64: return launch_dirichlet<float, 64>(L, s);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace

// ---------------------------------------------------------------------------
// Algorithm 2
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

template <typename Real>
cudaError_t dispatch_dirichlet_general(int K, const DirichletLaunch& L, cudaStream_t s)
{
    switch (K) {
#define PM_CASE(k) case k: return launch_dirichlet_general<Real, k>(L, s);
        PM_K_LIST(PM_CASE)
#undef PM_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
int dispatch_dirichlet_general_occupancy(int K)
{
    switch (K) {
#define PM_CASE(k) case k: return dirichlet_general_blocks_per_sm<Real, k>();
        PM_K_LIST(PM_CASE)
#undef PM_CASE
    }
    return 1;
}

// Algorithm 2 in the disk: the constant-coefficient map (gen == nullptr) or the
// general forcing / state-dependent diffusion of pm_forward_dirichlet_general.
int dirichlet_call(pm_ctx* c, const pm_field* field, double drift_scale, double kappa, const pm_dirichlet_data* gd,
                   const DirichletGeneral* gen, const double* x, int64_t n_obs, int64_t M, double dt,
                   int64_t max_steps, uint64_t seed, uint32_t flags, double* mean, double* var, int32_t* exit_step,
                   int64_t* n_unexited, const pm_path_opts* opts)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    int rc = check_field(field, true);
    if (rc) return rc;
    const bool wide = wide_K(field->K);
    if (wide && (flags & PM_FP64)) return fail(PM_EINVAL, "K=%d runs with float paths only", field->K);
    if (wide && gen && !(flags & PM_TENSOR))
        return fail(PM_EINVAL, "K=%d: the general disk map runs the wide bounds with PM_TENSOR only", field->K);
    if (!gd) return fail(PM_EINVAL, "boundary data is NULL");
    if (!(std::isfinite(gd->R) && gd->R > 0)) return fail(PM_EINVAL, "R must be finite and > 0");
    if (!std::isfinite(gd->quad) || !std::isfinite(gd->f_const)) return fail(PM_EINVAL, "quad and f_const must be finite");
    if (gd->n_ang < 0 || gd->n_ang > PM_MAX_BOUNDARY_MODES) return fail(PM_EINVAL, "n_ang out of range (max %d)", PM_MAX_BOUNDARY_MODES);
    if (gd->n_ang > 0 && (!gd->a || !gd->b)) return fail(PM_EINVAL, "boundary arrays are NULL");
    if (gd->n_ang > 0 && (!finite_array(gd->a, gd->n_ang) || !finite_array(gd->b, gd->n_ang)))
        return fail(PM_EINVAL, "boundary amplitudes contain NaN or Inf");
    if (!std::isfinite(drift_scale)) return fail(PM_EINVAL, "drift_scale must be finite");
    if (!(std::isfinite(kappa) && kappa >= 0)) return fail(PM_EINVAL, "kappa must be finite and >= 0");
    if (!(std::isfinite(dt) && dt > 0)) return fail(PM_EINVAL, "dt must be finite and > 0");
    if (max_steps < 1 || max_steps > 0x7fffffffLL) return fail(PM_EINVAL, "max_steps must be in [1, 2^31)");
    if (n_obs < 0) return fail(PM_EINVAL, "n_obs < 0");
    if (n_obs == 0) {
        if (n_unexited && !(flags & PM_DEVICE_PTRS)) *n_unexited = 0;
        return PM_OK;
    }
    if (M < 1) return fail(PM_EINVAL, "M must be >= 1");
    if (n_obs > 0xffffffffLL) return fail(PM_EINVAL, "n_obs too large");
    const int64_t off = opts ? opts->path_offset : 0;
    if (off < 0 || off + M > ((int64_t)1 << 32)) return fail(PM_EINVAL, "path_offset + M exceeds 2^32");
    if (n_obs > (((int64_t)1 << 62) / M)) return fail(PM_EINVAL, "n_obs * M too large");
    if (!x || !mean) return fail(PM_EINVAL, "x and mean must not be NULL");
    double* g_out = opts ? opts->g_out : nullptr;
    double* x_out = opts ? opts->x_out : nullptr;
    if ((rc = check_ptrs(c, flags, {x, mean, var, exit_step, n_unexited, g_out, x_out}))) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    const bool fp64 = flags & PM_FP64;
    if (!dev && !finite_array(x, 2 * n_obs)) return fail(PM_EINVAL, "observation points contain NaN or Inf");
    if ((rc = set_device(c))) return rc;
    const int64_t total = n_obs * M;
    // Claim order of the observations: longest expected walk first, by the
    // driftless mean exit time (R^2 - |x|^2) / (4 kappa), so that the heavy
    // tail of exit times meets the end of the call as rarely as possible.
    // Paths keep their (j, i) streams and slots, so results do not change.
    const bool order_obs = n_obs >= 2 && n_obs <= ((int64_t)1 << 24);
    std::vector<int32_t> obs_order;
    double walk_steps = 0.0;  // mean driftless exit time in steps, (R^2 - |x|^2) / (4 kappa dt)
    if (order_obs) {
        std::vector<double> hx;
        const double* px = x;
        if (dev) {
            hx.resize((size_t)(2 * n_obs));
            PM_CUDA(cudaMemcpyAsync(hx.data(), x, (size_t)n_obs * 16, cudaMemcpyDeviceToHost, c->stream), "copy x");
            PM_CUDA(cudaStreamSynchronize(c->stream), "copy x");
            px = hx.data();
        }
        obs_order.resize((size_t)n_obs);
        for (int64_t j = 0; j < n_obs; ++j) obs_order[(size_t)j] = (int32_t)j;
        auto r2 = [&](int32_t j) { return px[2 * (int64_t)j] * px[2 * (int64_t)j] + px[2 * (int64_t)j + 1] * px[2 * (int64_t)j + 1]; };
        std::stable_sort(obs_order.begin(), obs_order.end(), [&](int32_t a, int32_t b) { return r2(a) < r2(b); });
        // (the general map: kappa of its diffusion at the origin, the mean of
        // sigma_i(0)^2 / 2 over the two coordinates)
        const double kap = gen ? 0.25 * (gen->s0[0] * gen->s0[0] + gen->s0[1] * gen->s0[1]) : kappa;
        if (kap > 0) {
            double sum = 0.0;
            for (int64_t j = 0; j < n_obs; ++j) sum += std::max(gd->R * gd->R - r2((int32_t)j), 0.0);
            walk_steps = sum / (double)n_obs / (4.0 * kap * dt);
        }
    }

    auto layout = [&](Bump& b) {
        struct P { unsigned long long* ctr; double *g, *x, *mean, *var, *xo; int32_t* es; double2* rpart; int32_t* order; float* tab; } p{};
        p.ctr = b.take<unsigned long long>(4);  // next path, unexited, steps, tensor-core error flag
        p.tab = wide ? b.take<float>((size_t)wide_table_floats(field->K)) : nullptr;
        p.order = order_obs ? b.take<int32_t>((size_t)n_obs) : nullptr;
        p.rpart = b.take<double2>((size_t)(n_obs * (int64_t)reduce_path_chunks(M)));
        p.g = (dev && g_out) ? nullptr : b.take<double>((size_t)total);
        if (!dev) {
            p.x = b.take<double>((size_t)(2 * n_obs));
            p.mean = b.take<double>((size_t)n_obs);
            p.var = var ? b.take<double>((size_t)n_obs) : nullptr;
            p.es = exit_step ? b.take<int32_t>((size_t)total) : nullptr;
            p.xo = x_out ? b.take<double>((size_t)(2 * total)) : nullptr;
        }
        return p;
    };
    Bump probe(nullptr);
    layout(probe);
    if ((rc = ensure_workspace(c, probe.off))) return rc;
    Bump bump(c->ws);
    auto W = layout(bump);

    const double* dx = x;
    double *dmean = mean, *dvar = var, *dg = (dev && g_out) ? g_out : W.g, *dxo = x_out;
    int32_t* des = exit_step;
    if (!dev) {
        const size_t outb = (size_t)n_obs * 16 + (g_out ? (size_t)total * 8 : 0) + (exit_step ? (size_t)total * 4 : 0) +
                            (x_out ? (size_t)total * 16 : 0) + 256;
        const size_t inb = (size_t)n_obs * 16 + 64;
        if ((rc = ensure_host(c, inb > outb ? inb : outb))) return rc;
        memcpy(c->host, x, (size_t)n_obs * 16);
        PM_CUDA(cudaMemcpyAsync(W.x, c->host, (size_t)n_obs * 16, cudaMemcpyHostToDevice, c->stream), "copy x");
        dx = W.x;
        dmean = W.mean;
        dvar = W.var;
        des = W.es;
        dxo = W.xo;
    }
    const std::vector<double> tab = stage_coefficients(field->K, field->u);
    PM_CUDA(cudaMemsetAsync(W.ctr, 0, 32, c->stream), "clear counters");
    if (order_obs)
        PM_CUDA(cudaMemcpyAsync(W.order, obs_order.data(), (size_t)n_obs * 4, cudaMemcpyHostToDevice, c->stream),
                "copy order");
    c->last_steps = -1;

    DirichletLaunch L{};
    L.coef = tab.data();
    L.drift_scale = drift_scale;
    L.R = gd->R;
    L.quad = gd->quad;
    L.f_const = gd->f_const;
    L.n_ang = gd->n_ang;
    L.ga = gd->a;
    L.gb = gd->b;
    L.x = dx;
    L.order = W.order;
    L.n_obs = n_obs;
    L.M = M;
    L.dt = dt;
    L.s_dt = std::sqrt(2.0 * kappa * dt);
    L.max_steps = max_steps;
    L.counter = W.ctr;
    L.n_unexited = W.ctr + 1;
    L.steps = W.ctr + 2;
    L.g = dg;
    L.exit_step = des;
    L.x_out = dxo;
    L.path_offset = off;
    L.inst = opts ? opts->instance : 0u;
    L.key0 = (uint32_t)(seed & 0xffffffffu);
    L.key1 = (uint32_t)(seed >> 32);
    L.gen = gen;
    L.table_dev = W.tab;
    const int Kd = field->K;
    const bool use_tc = dirichlet_uses_tc(Kd, flags);
    int per_sm;
    // Untuned: longer walks take longer intervals between refills (fewer
    // refill barriers against a longer wait of the lanes whose paths ended;
    // the autotuner picked 16 pairs on walks of ~3e4 driftless steps).
    const int def_pairs = walk_steps >= 16384.0 ? 16 : walk_steps >= 4096.0 ? 8 : kDefaultRefillPairs;
    if (gen && use_tc) {
        per_sm = dirichlet_resident(Kd, false, true, true);
        L.refill_pairs = def_pairs;
    } else if (gen) {
        per_sm = fp64 ? dispatch_dirichlet_general_occupancy<double>(Kd) : dispatch_dirichlet_general_occupancy<float>(Kd);
    } else {
        per_sm = dirichlet_resident(Kd, fp64, use_tc);
        per_sm = tuned_ctas_per_sm(c, PM_TUNE_DIRICHLET, Kd, flags & (PM_FP64 | (use_tc ? PM_TENSOR : 0u)), per_sm);
        if (use_tc) L.refill_pairs = tuned_refill_pairs(c, PM_TUNE_DIRICHLET, Kd, PM_TENSOR, def_pairs);
    }
    int64_t grid = (int64_t)per_sm * c->sm_count;
    const int64_t need = (total + kDirichletBlock - 1) / kDirichletBlock;
    if (grid > need) grid = need;
    L.grid = (int)(grid > 0 ? grid : 1);
    L.wait_limit = take_wait_limit(c);
    c->last_grid = L.grid;
    if (c->timing) PM_CUDA(cudaEventRecord(c->ev0, c->stream), "event");
    cudaError_t e;
    unsigned* tc_err = (unsigned*)(W.ctr + 3);
    if (gen && !use_tc) {
        e = fp64 ? dispatch_dirichlet_general<double>(Kd, L, c->stream) : dispatch_dirichlet_general<float>(Kd, L, c->stream);
    } else if (use_tc) {  // L.gen selects the general map's variant
        switch (Kd) {
        case 4: e = tdtc::launch_dirichlet_tc<4>(L, tc_err, c->stream); break;
        case 5: e = tdtc::launch_dirichlet_tc<5>(L, tc_err, c->stream); break;
        case 6: e = tdtc::launch_dirichlet_tc<6>(L, tc_err, c->stream); break;
        case 8: e = tdtc::launch_dirichlet_tc<8>(L, tc_err, c->stream); break;
        case 10: e = tdtc::launch_dirichlet_tc<10>(L, tc_err, c->stream); break;
        case 12: e = tdtc::launch_dirichlet_tc<12>(L, tc_err, c->stream); break;
        case 24: e = tdtc::launch_dirichlet_tc<24>(L, tc_err, c->stream); break;
        case 32: e = tdtc::launch_dirichlet_tc<32>(L, tc_err, c->stream); break;
        case 40: e = tdtc::launch_dirichlet_tc<40>(L, tc_err, c->stream); break;
        case 48: e = tdtc::launch_dirichlet_tc<48>(L, tc_err, c->stream); break;
        case 56: e = tdtc::launch_dirichlet_tc<56>(L, tc_err, c->stream); break;
        case 64: e = tdtc::launch_dirichlet_tc<64>(L, tc_err, c->stream); break;
        default: e = tdtc::launch_dirichlet_tc<16>(L, tc_err, c->stream); break;
        }
    } else if (wide) {
        e = launch_dirichlet_wide(Kd, L, c->stream);
    } else {
        e = fp64 ? dispatch_dirichlet<double>(Kd, L, c->stream) : dispatch_dirichlet<float>(Kd, L, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "dirichlet kernel launch");
    if (c->timing) {
        PM_CUDA(cudaEventRecord(c->ev1, c->stream), "event");
        c->timed = true;
    }
    count_launch(c);
    PM_CUDA(launch_reduce_paths(dg, n_obs, M, dmean, dvar, c->stream, W.rpart), "reduce kernel");
    count_launch(c, reduce_path_chunks(M) > 0 ? 2 : 1);
    if (dev && n_unexited)
        PM_CUDA(cudaMemcpyAsync(n_unexited, W.ctr + 1, 8, cudaMemcpyDeviceToDevice, c->stream), "copy n_unexited");
    if (dev && (flags & PM_ASYNC)) return PM_OK;

    unsigned long long unexited = 0;
    if (!dev) {
        char* h = (char*)c->host;
        size_t o = 0;
        PM_CUDA(cudaMemcpyAsync(h + o, dmean, (size_t)n_obs * 8, cudaMemcpyDeviceToHost, c->stream), "copy mean");
        o += (size_t)n_obs * 8;
        if (var) { PM_CUDA(cudaMemcpyAsync(h + o, dvar, (size_t)n_obs * 8, cudaMemcpyDeviceToHost, c->stream), "copy var"); o += (size_t)n_obs * 8; }
        if (g_out) { PM_CUDA(cudaMemcpyAsync(h + o, dg, (size_t)total * 8, cudaMemcpyDeviceToHost, c->stream), "copy g"); o += (size_t)total * 8; }
        if (x_out) { PM_CUDA(cudaMemcpyAsync(h + o, dxo, (size_t)total * 16, cudaMemcpyDeviceToHost, c->stream), "copy x_out"); o += (size_t)total * 16; }
        if (exit_step) { PM_CUDA(cudaMemcpyAsync(h + o, des, (size_t)total * 4, cudaMemcpyDeviceToHost, c->stream), "copy exit steps"); }
    }
    unsigned long long steps_taken = 0;
    PM_CUDA(cudaMemcpyAsync(&unexited, W.ctr + 1, 8, cudaMemcpyDeviceToHost, c->stream), "copy n_unexited");
    PM_CUDA(cudaMemcpyAsync(&steps_taken, W.ctr + 2, 8, cudaMemcpyDeviceToHost, c->stream), "copy step count");
    unsigned tc_flag = 0;
    PM_CUDA(cudaMemcpyAsync(&tc_flag, tc_err, 4, cudaMemcpyDeviceToHost, c->stream), "copy flag");
    PM_CUDA(cudaStreamSynchronize(c->stream), "dirichlet");
    c->last_steps = (int64_t)steps_taken;
    if (!dev) {
        const char* h = (const char*)c->host;
        size_t o = 0;
        memcpy(mean, h + o, (size_t)n_obs * 8);
        o += (size_t)n_obs * 8;
        if (var) { memcpy(var, h + o, (size_t)n_obs * 8); o += (size_t)n_obs * 8; }
        if (g_out) { memcpy(g_out, h + o, (size_t)total * 8); o += (size_t)total * 8; }
        if (x_out) { memcpy(x_out, h + o, (size_t)total * 16); o += (size_t)total * 16; }
        if (exit_step) memcpy(exit_step, h + o, (size_t)total * 4);
        if (n_unexited) *n_unexited = (int64_t)unexited;
    }
    if (tc_flag) return fail(PM_ETIMEOUT, "a tensor-core wait in the particle kernel timed out");
    return unexited ? PM_WARN_UNEXITED : PM_OK;
}

}  // namespace

extern "C" {

int pm_forward_dirichlet(pm_ctx* c, const pm_field* field, double drift_scale, double kappa,
                         const pm_dirichlet_data* gd, const double* x, int64_t n_obs, int64_t M, double dt,
                         int64_t max_steps, uint64_t seed, uint32_t flags, double* mean, double* var,
                         int32_t* exit_step, int64_t* n_unexited, const pm_path_opts* opts)
{
    return dirichlet_call(c, field, drift_scale, kappa, gd, nullptr, x, n_obs, M, dt, max_steps, seed, flags, mean,
                          var, exit_step, n_unexited, opts);
}

int pm_forward_dirichlet_general(pm_ctx* c, const pm_field* field, double drift_scale, const pm_dirichlet_data* gd,
                                 const pm_diffusion_forcing* df, const double* x, int64_t n_obs, int64_t M, double dt,
                                 int64_t max_steps, uint64_t seed, uint32_t flags, double* mean, double* var,
                                 int32_t* exit_step, int64_t* n_unexited, const pm_path_opts* opts)
{
    if (!df) return fail(PM_EINVAL, "diffusion / forcing description is NULL");
    for (int k = 0; k < 2; ++k)
        if (!std::isfinite(df->s0[k]) || !std::isfinite(df->s1[k]))
            return fail(PM_EINVAL, "diffusion coefficients must be finite");
    if (df->n_src < 0 || df->n_src > PM_MAX_SOURCES) return fail(PM_EINVAL, "n_src must be in [0, %d]", PM_MAX_SOURCES);
    if (!(std::isfinite(df->w) && df->w >= 0)) return fail(PM_EINVAL, "w must be finite and >= 0");
    if (df->n_src > 0 && (!df->c || !df->F || !finite_array(df->c, 2 * df->n_src) || !finite_array(df->F, df->n_src)))
        return fail(PM_EINVAL, "source arrays NULL or not finite");
    if (df->milstein != 0 && df->milstein != 1) return fail(PM_EINVAL, "milstein must be 0 or 1");
    DirichletGeneral G{};
    for (int k = 0; k < 2; ++k) {
        G.s0[k] = df->s0[k];
        G.s1[k] = df->s1[k];
    }
    G.milstein = df->milstein;
    G.n_src = df->n_src;
    G.w = df->w;
    for (int q = 0; q < df->n_src; ++q) {
        G.c[2 * q] = df->c[2 * q];
        G.c[2 * q + 1] = df->c[2 * q + 1];
        G.F[q] = df->F[q];
    }
    return dirichlet_call(c, field, drift_scale, 0.0, gd, &G, x, n_obs, M, dt, max_steps, seed, flags,
                          mean, var, exit_step, n_unexited, opts);
}

// ---------------------------------------------------------------------------
// Diagnostics
// ---------------------------------------------------------------------------
int pm_philox(pm_ctx* c, const uint32_t* ctr, uint32_t key0, uint32_t key1, int64_t n, uint32_t* out, uint32_t flags)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    if (n < 0) return fail(PM_EINVAL, "n < 0");
    if (n == 0) return PM_OK;
    if (!ctr || !out) return fail(PM_EINVAL, "NULL array");
    int rc = check_ptrs(c, flags, {ctr, out});
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    const uint32_t* dctr = ctr;
    uint32_t* dout = out;
    if (!dev) {
        Bump probe(nullptr);
        probe.take<uint32_t>((size_t)(4 * n));
        probe.take<uint32_t>((size_t)(4 * n));
        if ((rc = ensure_workspace(c, probe.off))) return rc;
        Bump b(c->ws);
        uint32_t* a = b.take<uint32_t>((size_t)(4 * n));
        dout = b.take<uint32_t>((size_t)(4 * n));
        PM_CUDA(cudaMemcpyAsync(a, ctr, (size_t)n * 16, cudaMemcpyHostToDevice, c->stream), "copy counters");
        dctr = a;
    }
    PM_CUDA(launch_philox(dctr, key0, key1, n, dout, c->stream), "philox kernel");
    count_launch(c);
    if (!dev) PM_CUDA(cudaMemcpyAsync(out, dout, (size_t)n * 16, cudaMemcpyDeviceToHost, c->stream), "copy out");
    if (dev && (flags & PM_ASYNC)) return PM_OK;
    PM_CUDA(cudaStreamSynchronize(c->stream), "philox");
    return PM_OK;
}

int pm_sincos_turns(pm_ctx* c, const float* x, int64_t n, float* s, float* co)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    if (n < 0) return fail(PM_EINVAL, "n < 0");
    if (n == 0) return PM_OK;
    if (!x || !s || !co) return fail(PM_EINVAL, "NULL array");
    int rc = check_ptrs(c, PM_DEVICE_PTRS, {x, s, co});
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    PM_CUDA(launch_sincos_turns(x, n, s, co, c->stream), "sincos kernel");
    count_launch(c);
    PM_CUDA(cudaStreamSynchronize(c->stream), "sincos");
    return PM_OK;
}

int pm_normals(pm_ctx* c, uint64_t seed, uint32_t b, uint32_t j, uint32_t i, int64_t n0, int64_t count, double* out,
               uint32_t flags)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    if (count < 0 || n0 < 0) return fail(PM_EINVAL, "negative step range");
    if (count == 0) return PM_OK;
    if (!out) return fail(PM_EINVAL, "out is NULL");
    int rc = check_ptrs(c, flags, {out});
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    double* dout = out;
    if (!dev) {
        if ((rc = ensure_workspace(c, (size_t)count * 16 + 256))) return rc;
        dout = (double*)c->ws;
    }
    const bool packed = !(flags & PM_FP64) && (flags & PM_TENSOR);
    PM_CUDA(launch_normals(seed, b, j, i, n0, count, dout, flags & PM_FP64, packed, c->stream), "normals kernel");
    count_launch(c);
    if (!dev) PM_CUDA(cudaMemcpyAsync(out, dout, (size_t)count * 16, cudaMemcpyDeviceToHost, c->stream), "copy out");
    if (dev && (flags & PM_ASYNC)) return PM_OK;
    PM_CUDA(cudaStreamSynchronize(c->stream), "normals");
    return PM_OK;
}

int pm_velocity(pm_ctx* c, const pm_field* field, const double* x, int64_t npts, double* v, uint32_t flags)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    int rc = check_field(field);
    if (rc) return rc;
    if (npts < 0) return fail(PM_EINVAL, "npts < 0");
    if (npts == 0) return PM_OK;
    if (!x || !v) return fail(PM_EINVAL, "NULL array");
    if ((rc = check_ptrs(c, flags, {x, v}))) return rc;
    if ((rc = set_device(c))) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    const double* dx = x;
    double* dv = v;
    if (!dev) {
        Bump probe(nullptr);
        probe.take<double>((size_t)(2 * npts));
        probe.take<double>((size_t)(2 * npts));
        if ((rc = ensure_workspace(c, probe.off))) return rc;
        Bump b(c->ws);
        double* a = b.take<double>((size_t)(2 * npts));
        dv = b.take<double>((size_t)(2 * npts));
        PM_CUDA(cudaMemcpyAsync(a, x, (size_t)npts * 16, cudaMemcpyHostToDevice, c->stream), "copy x");
        dx = a;
    }
    const std::vector<double> tab = stage_coefficients(field->K, field->u);
    cudaError_t e = (flags & PM_FP64) ? dispatch_velocity<double>(field->K, tab.data(), dx, npts, dv, c->stream)
                                      : dispatch_velocity<float>(field->K, tab.data(), dx, npts, dv, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "velocity kernel");
    count_launch(c);
    if (!dev) PM_CUDA(cudaMemcpyAsync(v, dv, (size_t)npts * 16, cudaMemcpyDeviceToHost, c->stream), "copy v");
    if (dev && (flags & PM_ASYNC)) return PM_OK;
    PM_CUDA(cudaStreamSynchronize(c->stream), "velocity");
    return PM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuning of the Dirichlet kernel's persistent grid (pm_autotune.cu)
// ---------------------------------------------------------------------------
int pm_autotune_dirichlet(pm_ctx* c, const pm_field* field, double drift_scale, double kappa,
                          const pm_dirichlet_data* g, const double* x, int64_t n_obs, int64_t M, double dt,
                          int64_t max_steps, uint64_t seed, uint32_t flags, int32_t* best_ctas_per_sm)
{
    if (!c) return fail(PM_EINVAL, "ctx is NULL");
    int rc = check_field(field, true);
    if (rc) return rc;
    if (wide_K(field->K) && (flags & PM_FP64)) return fail(PM_EINVAL, "K=%d runs with float paths only", field->K);
    if (n_obs < 1 || M < 1) return fail(PM_EINVAL, "autotuning needs n_obs >= 1 and M >= 1");
    if ((rc = set_device(c))) return rc;
    flags &= ~PM_ASYNC;
    const bool dev = flags & PM_DEVICE_PTRS;
    const int K = field->K;
    const bool use_tc = dirichlet_uses_tc(K, flags);
    const int resident = dirichlet_resident(K, flags & PM_FP64, use_tc);
    std::vector<double> hmean;
    double* mean = nullptr;
    if (dev) {
        PM_CUDA(cudaMalloc(&mean, (size_t)n_obs * 8), "autotune output");
    } else {
        hmean.resize((size_t)n_obs);
        mean = hmean.data();
    }
    auto run = [&]() {
        return pm_forward_dirichlet(c, field, drift_scale, kappa, g, x, n_obs, M, dt, max_steps, seed, flags, mean,
                                    nullptr, nullptr, nullptr, nullptr);
    };
    rc = autotune_loop(c, PM_TUNE_DIRICHLET, K, flags & (PM_FP64 | (use_tc ? PM_TENSOR : 0u)), resident, use_tc, run,
                       best_ctas_per_sm);
    if (dev) cudaFree(mean);
    return rc;
}
