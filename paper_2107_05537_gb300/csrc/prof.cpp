// Per-kernel CUDA-event timing and a launch counter.  Every kernel launch of
// the library goes through pm_prof_begin / pm_prof_end; when profiling is on
// each launch is bracketed by two events on its own stream, and
// pmlsh_profile_read() reduces them to launches and total milliseconds per
// kernel name.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pmlsh_impl.h"

namespace {
struct Rec {
    const char *name;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<long long> g_launches{0};

cudaEvent_t take()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

int pm_prof_begin(const char *name, cudaStream_t st)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return -1;
    Rec r{name, take(), take()};
    cudaEventRecord(r.a, st);
    g_recs.push_back(r);
    return (int)g_recs.size() - 1;
}

void pm_prof_end(int token, cudaStream_t st)
{
    if (token < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (token < (int)g_recs.size()) cudaEventRecord(g_recs[token].b, st);
}

extern "C" {

pmlsh_status pmlsh_profile(int enable)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = enable != 0;
    return PMLSH_OK;
}

long long pmlsh_launch_count(void) { return g_launches.load(); }

pmlsh_status pmlsh_profile_read(char *buf, int64_t cap)
{
    std::lock_guard<std::mutex> lk(g_mu);
    std::map<std::string, std::pair<long long, double>> agg;
    for (Rec &r : g_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) { cudaGetLastError(); ms = 0.f; }
        auto &e = agg[r.name];
        e.first += 1;
        e.second += ms;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    std::string out = "{";
    bool first = true;
    for (auto &kv : agg) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(),
                 kv.second.first, kv.second.second);
        out += tmp;
        first = false;
    }
    out += "}";
    if (!buf || cap <= (int64_t)out.size()) {
        pm_set_error("profile buffer too small (%zu bytes needed)", out.size() + 1);
        return PMLSH_EINVAL;
    }
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return PMLSH_OK;
}

}  // extern "C"
