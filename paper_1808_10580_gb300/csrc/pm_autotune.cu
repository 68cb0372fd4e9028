// pm_autotune.cu -- the autotuner of the persistent kernels' launch shape.
//
// The Dirichlet and batched kernels are persistent: a grid of (CTAs per SM) x
// SMs whose lanes claim paths from counters.  Their results do not depend on
// the grid (every path's value is stored and reduced in path order), so their
// one free shape is the number of CTAs per SM.  The occupancy limit is not
// always the fastest: more CTAs hide more latency, fewer leave each CTA more
// issue slots and L1.  pm_autotune_* time one forward call per candidate on
// the caller's problem and keep the fastest in the context, keyed by (kernel,
// K, precision and tensor flags); with PM_AUTOTUNE_CACHE naming a JSON file,
// the choices for this device are read from it when a context is created and
// written back after tuning.  PM_AUTOTUNE=0 makes every launch use the
// occupancy limit.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "pm_internal.h"

namespace pm {

uint64_t tune_key(int kind, int K, uint32_t flags)
{
    return ((uint64_t)(uint32_t)kind << 40) | ((uint64_t)(uint32_t)(K & 0xffff) << 8) | (flags & (PM_FP64 | PM_TENSOR));
}

static bool autotune_off()
{
    const char* e = std::getenv("PM_AUTOTUNE");
    return e && e[0] == '0';
}

int tuned_ctas_per_sm(pm_ctx* c, int kind, int K, uint32_t flags, int resident)
{
    if (autotune_off()) return resident;
    const auto it = c->ctas_per_sm.find(tune_key(kind, K, flags));
    if (it == c->ctas_per_sm.end()) return resident;
    return std::max(1, std::min(it->second, resident));
}

// Cache file: one flat JSON object {"<device>|<kind>|<K>|<flags>": n, ...}.
static std::string entry_name(const pm_ctx* c, uint64_t key)
{
    char buf[64];
    std::snprintf(buf, sizeof buf, "|%u|%u|%u", (unsigned)(key >> 40), (unsigned)((key >> 8) & 0xffff),
                  (unsigned)(key & 0xff));
    return c->device_name + buf;
}

static std::map<std::string, int> read_cache(const char* path)
{
    std::map<std::string, int> out;
    FILE* f = std::fopen(path, "rb");
    if (!f) return out;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
    std::fclose(f);
    size_t pos = 0;
    for (;;) {
        const size_t q0 = text.find('"', pos);
        if (q0 == std::string::npos) break;
        const size_t q1 = text.find('"', q0 + 1);
        if (q1 == std::string::npos) break;
        const size_t colon = text.find(':', q1);
        if (colon == std::string::npos) break;
        const int v = std::atoi(text.c_str() + colon + 1);
        out[text.substr(q0 + 1, q1 - q0 - 1)] = v;
        pos = colon + 1;
    }
    return out;
}

static bool write_cache(const char* path, const std::map<std::string, int>& entries)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return false;
    std::fprintf(f, "{");
    bool first = true;
    for (const auto& e : entries) {
        std::fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", e.first.c_str(), e.second);
        first = false;
    }
    std::fprintf(f, "\n}\n");
    const bool ok = std::fclose(f) == 0;
    return ok && std::rename(tmp.c_str(), path) == 0;
}

void load_tune_cache(pm_ctx* c)
{
    const char* path = std::getenv("PM_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    const std::string prefix = c->device_name + "|";
    for (const auto& e : read_cache(path)) {
        if (e.first.compare(0, prefix.size(), prefix) != 0) continue;
        unsigned kind = 0, K = 0, flags = 0;
        if (std::sscanf(e.first.c_str() + prefix.size(), "%u|%u|%u", &kind, &K, &flags) == 3 && e.second > 0)
            c->ctas_per_sm[tune_key((int)kind, (int)K, flags)] = e.second;
    }
}

// Times run() (one synchronous forward call) for every candidate number of
// CTAs per SM in [1, resident], twice each (the first call may capture a
// graph), with events on the context's stream around the second; keeps the
// fastest.
int autotune_loop(pm_ctx* c, int kind, int K, uint32_t flags, int resident, const std::function<int()>& run,
                  int32_t* best)
{
    const uint64_t key = tune_key(kind, K, flags);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "autotune events");
    }
    float best_ms = 0.f;
    int best_n = resident;
    int rc = PM_OK;
    for (int n = 1; n <= resident && rc >= 0; ++n) {
        c->ctas_per_sm[key] = n;
        rc = run();
        if (rc < 0) break;
        cudaEventRecord(e0, c->stream);
        rc = run();
        cudaEventRecord(e1, c->stream);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "autotune timing");
            break;
        }
        if (rc >= 0 && (n == 1 || ms < best_ms)) {
            best_ms = ms;
            best_n = n;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc < 0) {
        c->ctas_per_sm.erase(key);
        return rc;
    }
    c->ctas_per_sm[key] = best_n;
    if (best) *best = best_n;
    const char* path = std::getenv("PM_AUTOTUNE_CACHE");
    if (path && *path) {
        auto entries = read_cache(path);
        entries[entry_name(c, key)] = best_n;
        if (!write_cache(path, entries)) return fail(PM_EINVAL, "cannot write the autotune cache %s", path);
    }
    return PM_OK;
}

}  // namespace pm

extern "C" int pm_set_ctas_per_sm(pm_ctx* c, int32_t kind, int32_t K, uint32_t flags, int32_t ctas_per_sm)
{
    if (!c) return pm::fail(PM_EINVAL, "ctx is NULL");
    if (kind != PM_TUNE_DIRICHLET && kind != PM_TUNE_BATCHED) return pm::fail(PM_EINVAL, "unknown kernel kind %d", kind);
    const uint64_t key = pm::tune_key(kind, K, flags);
    if (ctas_per_sm <= 0) c->ctas_per_sm.erase(key);
    else c->ctas_per_sm[key] = ctas_per_sm;
    return PM_OK;
}
