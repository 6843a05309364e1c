// Kernel timing trace: when enabled, every kernel the library launches is
// bracketed by a pair of CUDA events recorded on the launch's own stream, so
// the per-kernel device time of a real workload can be read without a
// profiler. Off by default; when off the cost is one relaxed load per launch.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pgen.h"
#include "pg_internal.h"
#include "pg_trace.h"

namespace pgen {

std::atomic<uint64_t> g_launch_count{0};

namespace {

struct Rec {
    const char* name;
    cudaEvent_t a, b;
};

std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

TraceScope::TraceScope(const char* name, cudaStream_t s) : idx_(-1), s_(s)
{
    if (!g_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{name, get_event(), get_event()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    idx_ = (int)g_recs.size() - 1;
}

TraceScope::~TraceScope()
{
    if (idx_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (idx_ < (int)g_recs.size()) cudaEventRecord(g_recs[idx_].b, s_);
}

}  // namespace pgen

using namespace pgen;

extern "C" {

void pg_trace_enable(int on) { g_on.store(on ? 1 : 0); }

uint64_t pg_launch_count(void) { return g_launch_count.load(std::memory_order_relaxed); }

size_t pg_trace_dump(char* buf, size_t len)
{
    std::lock_guard<std::mutex> lk(g_mu);
    std::map<std::string, std::pair<long, double>> agg;
    for (const Rec& r : g_recs) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) ms = 0.f;
        auto& v = agg[r.name];
        v.first += 1;
        v.second += ms;
    }
    std::string out = "{";
    bool first = true;
    for (const auto& kv : agg) {
        char item[256];
        std::snprintf(item, sizeof(item), "%s\"%s\": [%ld, %.6f]", first ? "" : ", ",
                      kv.first.c_str(), kv.second.first, kv.second.second);
        out += item;
        first = false;
    }
    out += "}";
    if (!buf || len < out.size() + 1) return out.size() + 1;   // size query: keep the record
    std::memcpy(buf, out.data(), out.size() + 1);
    for (const Rec& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return out.size() + 1;
}

}  // extern "C"
