// pm_internal.h -- the context object and host helpers shared by the C-ABI
// translation units (pm_api.cu, pm_batched_api.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <functional>
#include <initializer_list>
#include <map>
#include <string>

#include <cuda_runtime.h>

#include "../../include/pm.h"

struct pm_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* ws = nullptr;      // device workspace (grows)
    size_t ws_size = 0;
    void* host = nullptr;    // pinned staging (grows)
    size_t host_size = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timing = false;
    bool timed = false;
    int64_t launches = 0;
    int64_t last_steps = -1;     // Euler steps of the last synchronous forward call
    int64_t last_grid = 0;       // CTAs of the last particle-kernel launch
    // Batched map: the last captured CUDA graph and the key of the call shape it serves.
    uint64_t graph_key = 0;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0;  // kernels per replay
    int graph_mode = 1;          // 1: capture and replay when the stream allows it
    // Autotuned resident CTAs per SM of the persistent kernels, and the pairs of
    // Euler steps between lane refills of their tensor-core forms, by tune_key().
    std::map<uint64_t, int> ctas_per_sm;
    std::map<uint64_t, int> refill_pairs;
    std::string device_name;
    // Test setting: polls of the tensor-core progress waits of the next forward
    // or GEMM call (pm_set_wait_limit); -1 = the full bound.
    int64_t wait_limit_next = -1;
};

namespace pm {

// Bump allocator over the workspace (256-byte aligned slices); a null base only measures.
struct Bump {
    char* base;
    size_t off = 0;
    explicit Bump(void* b) : base((char*)b) {}
    template <typename T> T* take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
bool supported_K(int K);
bool finite_array(const double* p, int64_t n);
bool is_device_pointer(const void* p, int device);
int ensure_workspace(pm_ctx* c, size_t bytes);
int ensure_host(pm_ctx* c, size_t bytes);
int set_device(pm_ctx* c);
int check_field(const pm_field* f, bool allow_wide = false, bool allow_simt_wide = false);
int check_ptrs(const pm_ctx* c, uint32_t flags, std::initializer_list<const void*> ptrs);
// theta0 description: modes within PM_MAX_THETA0_MODES, arrays present and
// finite, wave numbers |k| <= 4096 (the float phase reduction's range).
int check_theta0(const pm_fourier* th);
// Section 4.1, Eq. v_expand: the product-basis table of the stream-function
// coefficients u (2|H_K| doubles) into tab (table_size(K) doubles, caller's storage).
void stage_coefficients_into(int K, const double* u, double* tab);
void count_launch(pm_ctx* c, int n = 1);
// The progress-wait bound of this call (pm_set_wait_limit), then back to the full bound.
uint32_t take_wait_limit(pm_ctx* c);

// Autotuner (pm_autotune.cu).  kind: PM_TUNE_DIRICHLET or PM_TUNE_BATCHED.
uint64_t tune_key(int kind, int K, uint32_t flags);
// CTAs per SM for a persistent launch: the tuned value (at most `resident`)
// unless PM_AUTOTUNE=0 or none is known, else `resident`.
int tuned_ctas_per_sm(pm_ctx* c, int kind, int K, uint32_t flags, int resident);
// Pairs of Euler steps between lane refills of a persistent tensor-core
// kernel: the tuned value unless PM_AUTOTUNE=0 or none is known, else `def`.
int tuned_refill_pairs(pm_ctx* c, int kind, int K, uint32_t flags, int def);
constexpr int kDefaultRefillPairs = 4;
// Untuned refill interval of the batched tensor-core kernel (what its
// autotuner picked on 256 mixed instances of 100 observations x 4096 paths).
constexpr int kBatchedRefillPairs = 8;
// Reads this device's entries of the PM_AUTOTUNE_CACHE file into the context.
void load_tune_cache(pm_ctx* c);
// Runs the timing sweep over CTAs per SM in [1, resident] and, with
// tune_refill, then over the refill interval (see pm_autotune.cu).
int autotune_loop(pm_ctx* c, int kind, int K, uint32_t flags, int resident, bool tune_refill,
                  const std::function<int()>& run, int32_t* best);

}  // namespace pm

#define PM_CUDA(call, what)                                    \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return pm::cuda_fail(e_, what); \
    } while (0)
