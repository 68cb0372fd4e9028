// pm_noalloc.cu -- pm_forward_timedep_noalloc: the time-dependent forward map
// for callers that must not allocate GPU memory.
//
// Some callers cannot call cudaMalloc: code that runs while another allocator
// owns the device memory (a caching allocator that has reserved the pool, or
// a process that has handed all memory to a fixed arena), code on a latency
// path where cudaMalloc's implicit device synchronisation is not acceptable,
// and embedded or real-time hosts that forbid allocation after start-up.  For
// them this entry point runs the same kernels as pm_forward_timedep but takes
// its scratch (per-observation records, processing order, per-CTA partial
// sums, an error flag) from one fixed array in device memory that the library
// declares at file scope.  Every GPU that loads the library holds that array
// until the process exits.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/pm.h"
#include "pm_launch.h"

using namespace pm;

namespace {

constexpr size_t kScratchBytes = PM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The shared scratch.  In host code `g_noalloc_scratch` names a host-side
// stand-in, not the device array: kernels receive the device address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_dev[kMaxDevices] = {};

// Messages go to the same per-thread slot pm_last_error() reads.
int nfail(int code, const char* msg) { return pm::set_error(code, msg); }

int nfail_cuda(cudaError_t e, const char* what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return pm::set_error(e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA, buf);
}

// Device address of the scratch on the current device, looked up once per device.
int scratch_address(int device, void** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return nfail_cuda(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_dev[device] = p;
    }
    *out = g_scratch_dev[device];
    return PM_OK;
}

bool finite_all(const double* p, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

bool on_device(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Same product-basis table as the main entry point builds (see pm_api.cu),
// written into caller-provided storage so that nothing is allocated.
void fill_table(int K, const double* u, double* tab)
{
    const int n = table_size(K);
    for (int q = 0; q < n; ++q) tab[q] = 0.0;
    auto idx = [&](int m, int nn) -> int64_t { return m == 0 ? (nn - 1) : K + (int64_t)(m - 1) * (2 * K + 1) + (nn + K); };
    for (int m = 0; m <= K; ++m)
        for (int nn = 0; nn <= K; ++nn) {
            if (m == 0 && nn == 0) continue;
            double A = 0, B = 0, G = 0, D = 0;
            if (m == 0) { A = u[2 * idx(0, nn)]; B = u[2 * idx(0, nn) + 1]; }
            else if (nn == 0) { A = u[2 * idx(m, 0)]; G = u[2 * idx(m, 0) + 1]; }
            else {
                const double ap = u[2 * idx(m, nn)], bp = u[2 * idx(m, nn) + 1];
                const double am = u[2 * idx(m, -nn)], bm = u[2 * idx(m, -nn) + 1];
                A = ap + am; B = bp - bm; G = bp + bm; D = am - ap;
            }
            double* e = tab + (size_t)(m * (K + 1) + nn) * 8;
            const double sn = kTwoPi * nn, sm = kTwoPi * m;
            e[0] = sn * A; e[1] = -sn * B; e[2] = sn * G; e[3] = -sn * D;
            e[4] = sm * G; e[5] = sm * D; e[6] = -sm * A; e[7] = -sm * B;
        }
}

template <typename Real>
cudaError_t dispatch(int K, const TimedepLaunch& L, cudaStream_t s)
{
    switch (K) {
    case 0: return launch_timedep<Real, 0>(L, s);
    case 1: return launch_timedep<Real, 1>(L, s);
    case 2: return launch_timedep<Real, 2>(L, s);
    case 3: return launch_timedep<Real, 3>(L, s);
    case 4: return launch_timedep<Real, 4>(L, s);
    case 5: return launch_timedep<Real, 5>(L, s);
    case 6: return launch_timedep<Real, 6>(L, s);
    case 8: return launch_timedep<Real, 8>(L, s);
    case 10: return launch_timedep<Real, 10>(L, s);
    case 12: return launch_timedep<Real, 12>(L, s);
    case 16: return launch_timedep<Real, 16>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

extern "C" int pm_forward_timedep_noalloc(const pm_field* field, double kappa, const pm_fourier* th, const double* x,
                                          const double* t, int64_t n_obs, int64_t M, double dt, uint64_t seed,
                                          uint32_t flags, double* mean, double* var, void* cuda_stream)
{
    if (!field) return nfail(PM_EINVAL, "field is NULL");
    const int K = field->K;
    if (!(K >= 0 && K <= 6) && K != 8 && K != 10 && K != 12 && K != 16)
        return nfail(PM_EINVAL, "K is not one of the compiled bounds 0..6, 8, 10, 12, 16");
    const int64_t nu = (int64_t)(2 * K + 1) * (2 * K + 1) - 1;
    if (nu > 0 && (!field->u || !finite_all(field->u, nu))) return nfail(PM_EINVAL, "field coefficients NULL or not finite");
    if (!th || th->n < 0 || th->n > PM_MAX_THETA0_MODES) return nfail(PM_EINVAL, "theta0 missing or too many modes");
    if (th->n > 0 && (!th->k || !th->a || !th->b || !finite_all(th->a, th->n) || !finite_all(th->b, th->n)))
        return nfail(PM_EINVAL, "theta0 arrays NULL or not finite");
    if (!(std::isfinite(kappa) && kappa >= 0)) return nfail(PM_EINVAL, "kappa must be finite and >= 0");
    if (!(std::isfinite(dt) && dt > 0)) return nfail(PM_EINVAL, "dt must be finite and > 0");
    if (n_obs < 0 || M < 1 || M > ((int64_t)1 << 32)) return nfail(PM_EINVAL, "need n_obs >= 0 and 1 <= M <= 2^32");
    if (n_obs == 0) return PM_OK;
    if (!x || !t || !mean) return nfail(PM_EINVAL, "x, t and mean must not be NULL");
    if (!on_device(x) || !on_device(t) || !on_device(mean) || (var && !on_device(var)))
        return nfail(PM_EINVAL, "x, t, mean and var must be device pointers on the current device");

    // Scratch layout: flag | records | order | per-CTA partials.
    const int64_t chunks = (M + kTimedepBlock - 1) / kTimedepBlock;
    if (n_obs > ((int64_t)1 << 26) || n_obs * chunks > 0x7fffffffLL) return nfail(PM_EINVAL, "problem too large");
    const bool sort = n_obs <= 8192;
    const size_t off_rec = 256;
    const size_t off_order = off_rec + align256((size_t)n_obs * sizeof(ObsRec));
    const size_t off_part = off_order + (sort ? align256((size_t)n_obs * 4) : 0);
    const size_t need = off_part + (size_t)(n_obs * chunks) * sizeof(double2);
    if (need > kScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "problem needs %zu bytes of scratch; the fixed scratch holds %zu (n_obs * ceil(M/%d) too large)",
                 need, kScratchBytes, kTimedepBlock);
        return nfail(PM_EINVAL, buf);
    }

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return nfail_cuda(e, "cudaGetDevice");
    if (device < 0 || device >= kMaxDevices) return nfail(PM_EINVAL, "device index out of range");
    void* base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc) return rc;
    char* s = (char*)base;
    unsigned* err = (unsigned*)s;
    ObsRec* rec = (ObsRec*)(s + off_rec);
    int32_t* order = sort ? (int32_t*)(s + off_order) : nullptr;
    double2* part = (double2*)(s + off_part);
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // The flag keeps the previous call's value: clear it.  Records, order and
    // partials are fully rewritten by this call's kernels before they are read.
    e = cudaMemsetAsync(err, 0, 16, stream);
    if (e != cudaSuccess) return nfail_cuda(e, "clear flag");
    e = launch_prep_timedep(x, t, n_obs, dt, kappa, rec, order, err, stream);
    if (e != cudaSuccess) return nfail_cuda(e, "prep kernel");

    double tab[table_size(16)];
    fill_table(K, field->u, tab);
    TimedepLaunch L{};
    L.coef = tab;
    L.nq = th->n;
    L.qk = th->k;
    L.qa = th->a;
    L.qb = th->b;
    L.obs = rec;
    L.order = order;
    L.part = part;
    L.dt = dt;
    L.s_dt = std::sqrt(2.0 * kappa * dt);
    L.M = M;
    L.path_offset = 0;
    L.n_obs = (int32_t)n_obs;
    L.chunks = (int32_t)chunks;
    L.key0 = (uint32_t)(seed & 0xffffffffu);
    L.key1 = (uint32_t)(seed >> 32);
    e = (flags & PM_FP64) ? dispatch<double>(K, L, stream) : dispatch<float>(K, L, stream);
    if (e != cudaSuccess) return nfail_cuda(e, "timedep kernel");
    e = launch_reduce(part, n_obs, (int32_t)chunks, M, mean, var, stream);
    if (e != cudaSuccess) return nfail_cuda(e, "reduce kernel");
    if (flags & PM_ASYNC) return PM_OK;

    unsigned flag = 0;
    e = cudaMemcpyAsync(&flag, err, sizeof flag, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return nfail_cuda(e, "synchronise");
    if (flag) return nfail(PM_EINVAL, "observation points or times are not finite, a time is negative, or a step count exceeds 2^31");
    return PM_OK;
}
