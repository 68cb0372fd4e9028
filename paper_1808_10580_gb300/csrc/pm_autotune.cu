// pm_autotune.cu -- the autotuner of the persistent kernels' launch shape.
//
// The Dirichlet and batched kernels are persistent: a grid of (CTAs per SM) x
// SMs whose lanes claim paths from counters.  Their results do not depend on
// the launch shape (every path's value is stored and reduced in path order,
// and its random numbers are keyed by its own step index), so two shapes are
// free: the number of CTAs per SM, and, for the tensor-core forms whose CTAs
// step together through one product per step, the number of step pairs
// between two refills of the lanes whose paths have ended (frequent refills
// keep lanes busy and cost a ballot, an atomic and a CTA barrier each).  The
// occupancy limit and a fixed interval are not always the fastest.
// pm_autotune_* time forward calls on the caller's problem by coordinate
// descent -- CTAs per SM from 1 to the occupancy limit at the current refill
// interval, then the interval over {1, 2, 4, 8, 16} pairs at the best grid --
// and keep the fastest in the context, keyed by (kernel, K, precision and
// tensor flags); with PM_AUTOTUNE_CACHE naming a JSON file, the choices for
// this device are read from it when a context is created and written back
// after tuning.  PM_AUTOTUNE=0 makes every launch use the occupancy limit and
// the default interval.
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

int tuned_refill_pairs(pm_ctx* c, int kind, int K, uint32_t flags, int def)
{
    if (autotune_off()) return def;
    const auto it = c->refill_pairs.find(tune_key(kind, K, flags));
    return it == c->refill_pairs.end() ? def : std::max(1, std::min(it->second, 64));
}

// Cache file: one flat JSON object {"<device>|<kind>|<K>|<flags>": n, ...};
// the refill interval under the same name with "|refill" appended.
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
        char tail[16] = "";
        const int nf = std::sscanf(e.first.c_str() + prefix.size(), "%u|%u|%u|%15s", &kind, &K, &flags, tail);
        if (nf >= 3 && e.second > 0) {
            if (nf == 4 && std::strcmp(tail, "refill") == 0) c->refill_pairs[tune_key((int)kind, (int)K, flags)] = e.second;
            else if (nf == 3) c->ctas_per_sm[tune_key((int)kind, (int)K, flags)] = e.second;
        }
    }
}

// Times run() (one synchronous forward call) twice per candidate (the first
// call may capture a graph), with events on the context's stream around the
// second: CTAs per SM in [1, resident] at the current refill interval, then
// (tune_refill) the refill interval at the best grid; keeps the fastest.
int autotune_loop(pm_ctx* c, int kind, int K, uint32_t flags, int resident, bool tune_refill,
                  const std::function<int()>& run, int32_t* best)
{
    const uint64_t key = tune_key(kind, K, flags);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "autotune events");
    }
    auto timed = [&](float& ms) -> int {
        int r = run();
        if (r < 0) return r;
        cudaEventRecord(e0, c->stream);
        r = run();
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "autotune timing");
        return r;
    };
    float best_ms = 0.f;
    int best_n = resident;
    int rc = PM_OK;
    if (!c->refill_pairs.count(key)) c->refill_pairs[key] = kDefaultRefillPairs;
    for (int n = 1; n <= resident && rc >= 0; ++n) {
        c->ctas_per_sm[key] = n;
        float ms = 0.f;
        rc = timed(ms);
        if (rc >= 0 && (n == 1 || ms < best_ms)) {
            best_ms = ms;
            best_n = n;
        }
    }
    c->ctas_per_sm[key] = best_n;
    int best_r = c->refill_pairs[key];
    if (tune_refill && rc >= 0) {
        for (int r : {1, 2, 4, 8, 16}) {
            if (r == best_r) continue;
            c->refill_pairs[key] = r;
            float ms = 0.f;
            rc = timed(ms);
            if (rc < 0) break;
            if (ms < best_ms) {
                best_ms = ms;
                best_r = r;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc < 0) {
        c->ctas_per_sm.erase(key);
        c->refill_pairs.erase(key);
        return rc;
    }
    c->refill_pairs[key] = best_r;
    if (best) *best = best_n;
    const char* path = std::getenv("PM_AUTOTUNE_CACHE");
    if (path && *path) {
        auto entries = read_cache(path);
        entries[entry_name(c, key)] = best_n;
        if (tune_refill) entries[entry_name(c, key) + "|refill"] = best_r;
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

extern "C" int pm_set_refill_pairs(pm_ctx* c, int32_t kind, int32_t K, uint32_t flags, int32_t pairs)
{
    if (!c) return pm::fail(PM_EINVAL, "ctx is NULL");
    if (kind != PM_TUNE_DIRICHLET && kind != PM_TUNE_BATCHED) return pm::fail(PM_EINVAL, "unknown kernel kind %d", kind);
    const uint64_t key = pm::tune_key(kind, K, flags);
    if (pairs <= 0) c->refill_pairs.erase(key);
    else c->refill_pairs[key] = pairs > 64 ? 64 : pairs;
    return PM_OK;
}

extern "C" int pm_tuned_shape(pm_ctx* c, int32_t kind, int32_t K, uint32_t flags, int32_t* ctas_per_sm,
                              int32_t* refill_pairs)
{
    if (!c) return pm::fail(PM_EINVAL, "ctx is NULL");
    const uint64_t key = pm::tune_key(kind, K, flags);
    const auto a = c->ctas_per_sm.find(key);
    const auto b = c->refill_pairs.find(key);
    if (ctas_per_sm) *ctas_per_sm = a == c->ctas_per_sm.end() ? 0 : a->second;
    if (refill_pairs) *refill_pairs = b == c->refill_pairs.end() ? 0 : b->second;
    return PM_OK;
}
