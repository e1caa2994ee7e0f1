// Autotuner: candidate schedules of a workload are timed on the device (CUDA
// events around the kernel they change) and the fastest is kept per workload
// signature, process-wide, optionally persisted to a text file so that later
// processes skip the timing.  The callers (api.cu) decide what a candidate is;
// this file only owns the cache.
//
// File format (POPCORN_TUNE_CACHE names the file; one entry per line):
//   target precision a b c d e sms : p0 p1 p2 p3 ms
// Later lines override earlier ones with the same key.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "popcorn.h"
#include "popcorn_internal.cuh"

namespace popcorn {
namespace {

using KeyTuple = std::tuple<int32_t, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t>;

KeyTuple as_tuple(const TuneKey& k) { return KeyTuple(k.target, k.precision, k.a, k.b, k.c, k.d, k.e, k.sms); }

struct Cache {
    std::mutex mu;
    std::map<KeyTuple, TuneValue> map;
    bool loaded = false;
};

Cache& cache() {
    static Cache c;
    return c;
}

const char* cache_path() {
    const char* p = std::getenv("POPCORN_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

void load_locked(Cache& c) {
    if (c.loaded) return;
    c.loaded = true;
    const char* path = cache_path();
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        TuneKey k{};
        TuneValue v{};
        if (std::sscanf(line, "%d %d %d %d %d %d %d %d : %d %d %d %d %f", &k.target, &k.precision, &k.a, &k.b, &k.c,
                        &k.d, &k.e, &k.sms, &v.p[0], &v.p[1], &v.p[2], &v.p[3], &v.ms) == 13)
            c.map[as_tuple(k)] = v;
    }
    std::fclose(f);
}

}  // namespace

int32_t log2_bucket(double x) { return x > 0 ? (int32_t)std::lround(4.0 * std::log2(x)) : -1; }

bool tune_lookup(const TuneKey& k, TuneValue* v) {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    load_locked(c);
    auto it = c.map.find(as_tuple(k));
    if (it == c.map.end()) return false;
    *v = it->second;
    return true;
}

void tune_store(const TuneKey& k, const TuneValue& v) {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    load_locked(c);
    c.map[as_tuple(k)] = v;
    const char* path = cache_path();
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;   // the in-memory entry still serves this process
    std::fprintf(f, "%d %d %d %d %d %d %d %d : %d %d %d %d %.6f\n", k.target, k.precision, k.a, k.b, k.c, k.d, k.e,
                 k.sms, v.p[0], v.p[1], v.p[2], v.p[3], (double)v.ms);
    std::fclose(f);
}

}  // namespace popcorn

extern "C" {

POPCORN_API int32_t popcorn_autotune_entries(void) {
    popcorn::Cache& c = popcorn::cache();
    std::lock_guard<std::mutex> lk(c.mu);
    popcorn::load_locked(c);
    return (int32_t)c.map.size();
}

POPCORN_API void popcorn_autotune_clear(void) {
    popcorn::Cache& c = popcorn::cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.map.clear();
    c.loaded = true;   // the file is left alone; a cleared process does not re-read it
}

}  // extern "C"
