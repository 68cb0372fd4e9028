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

#include "../../include/pm.h"
#include "pm_internal.h"
#include "pm_launch.h"

using namespace pm;

namespace {

constexpr size_t kScratchBytes = PM_NOALLOC_SCRATCH_BYTES;

// The shared scratch.  In host code `g_noalloc_scratch` names a host-side
// stand-in, not the device array: kernels receive the device address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Messages go to the same per-thread slot pm_last_error() reads.
int nfail(int code, const char* msg) { return pm::set_error(code, msg); }

int nfail_cuda(cudaError_t e, const char* what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return pm::set_error(e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA, buf);
}

// Device address of the scratch in the current device's context, looked up on
// every call: after a cudaDeviceReset the module is loaded again in a new
// context and the array may sit elsewhere, so no address is kept between
// calls.  Once the module is loaded the lookup allocates nothing.
int scratch_address(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return nfail_cuda(e, "cudaGetSymbolAddress(scratch)");
    *out = p;
    return PM_OK;
}

// Device (or managed) memory of `device`; a pointer into another GPU's memory
// is rejected (the kernels would read it over the peer link, or fault).
bool on_device(const void* p, int device)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == device;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

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
    if (nu > 0 && (!field->u || !pm::finite_array(field->u, nu))) return nfail(PM_EINVAL, "field coefficients NULL or not finite");
    int rc = pm::check_theta0(th);
    if (rc) return rc;
    if (!(std::isfinite(kappa) && kappa >= 0)) return nfail(PM_EINVAL, "kappa must be finite and >= 0");
    if (!(std::isfinite(dt) && dt > 0)) return nfail(PM_EINVAL, "dt must be finite and > 0");
    if (n_obs < 0 || M < 1 || M > ((int64_t)1 << 32)) return nfail(PM_EINVAL, "need n_obs >= 0 and 1 <= M <= 2^32");
    if (n_obs == 0) return PM_OK;
    if (!x || !t || !mean) return nfail(PM_EINVAL, "x, t and mean must not be NULL");
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return nfail_cuda(e, "cudaGetDevice");
    if (!on_device(x, device) || !on_device(t, device) || !on_device(mean, device) || (var && !on_device(var, device)))
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

    void* base = nullptr;
    if ((rc = scratch_address(&base))) return rc;
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
    pm::stage_coefficients_into(K, field->u, tab);
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
