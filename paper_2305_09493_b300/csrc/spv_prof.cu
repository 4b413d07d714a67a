// spv_prof.cu -- per-kernel timing of the library's own launches with CUDA
// events recorded on the launching stream (off by default).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <mutex>
#include <vector>

#include "../../include/spv.h"
#include "spv_prof.h"

namespace {
struct Rec { const char *name; cudaEvent_t a, b; };
struct Agg { const char *name; int64_t n; double ms; };
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;
std::vector<Agg> g_agg;

cudaEvent_t get_event()
{
    if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void drain_locked()
{
    for (Rec &r : g_pending) {
        float ms = 0;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        bool found = false;
        for (Agg &a : g_agg) if (a.name == r.name || !strcmp(a.name, r.name)) { a.n++; a.ms += ms; found = true; break; }
        if (!found) g_agg.push_back({r.name, 1, (double)ms});
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.clear();
}
}  // namespace

namespace spvprof {
bool enabled() { return g_on; }

int begin(const char *name, cudaStream_t st)
{
    if (!g_on) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{name, get_event(), get_event()};
    cudaEventRecord(r.a, st);
    g_pending.push_back(r);
    return (int)g_pending.size() - 1;
}

void end(int token, cudaStream_t st)
{
    if (token < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (token < (int)g_pending.size()) cudaEventRecord(g_pending[token].b, st);
}
}  // namespace spvprof

extern "C" int spv_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (on) { drain_locked(); g_agg.clear(); }
    g_on = on != 0;
    return SPV_SUCCESS;
}

extern "C" int spv_profile_read(int max, const char **names, int64_t *launches, double *total_ms)
{
    if (max < 0 || (max > 0 && (!names || !launches || !total_ms))) return SPV_E_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    int n = (int)g_agg.size();
    for (int i = 0; i < n && i < max; i++) {
        names[i] = g_agg[i].name;
        launches[i] = g_agg[i].n;
        total_ms[i] = g_agg[i].ms;
    }
    return n;
}
