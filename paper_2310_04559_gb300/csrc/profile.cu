// profile.cu -- optional per-phase device timing (CUDA events on the caller's
// stream) and a count of the library's kernel launches, for the benchmark and
// for tracing.  Disabled by default; when disabled a ProfScope costs nothing but
// a branch and an NVTX range (every phase is an NVTX range named after it, which
// timeline profilers show; without one attached the range calls do nothing).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cc_internal.cuh"

namespace cc {
namespace {

struct Pending {
    std::string name;
    cudaEvent_t e0, e1;
    double flops, bytes;
};
struct Total {
    std::string name;
    int launches;
    double ms, flops, bytes;
};

std::atomic<long long> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<Total> g_totals;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event()
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

void drain_locked()
{
    for (auto& p : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.e1);
        cudaEventElapsedTime(&ms, p.e0, p.e1);
        bool found = false;
        for (auto& t : g_totals)
            if (t.name == p.name) {
                t.launches += 1; t.ms += ms; t.flops += p.flops; t.bytes += p.bytes;
                found = true;
                break;
            }
        if (!found) g_totals.push_back(Total{p.name, 1, ms, p.flops, p.bytes});
        g_pool.push_back(p.e0);
        g_pool.push_back(p.e1);
    }
    g_pending.clear();
}

}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfScope::ProfScope(const char* name, cudaStream_t s, double flops, double bytes)
    : name_(name), s_(s), flops_(flops), bytes_(bytes), e0_(nullptr)
{
    nvtxRangePushA(name);
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    e0_ = get_event();
    cudaEventRecord((cudaEvent_t)e0_, s_);
}

ProfScope::~ProfScope()
{
    nvtxRangePop();
    if (!e0_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e1 = get_event();
    cudaEventRecord(e1, s_);
    g_pending.push_back(Pending{name_, (cudaEvent_t)e0_, e1, flops_, bytes_});
}

}  // namespace cc

extern "C" {

void cc_ladder_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(cc::g_mu);
    cc::drain_locked();
    cc::g_totals.clear();
    cc::g_enabled.store(on ? 1 : 0);
}

int cc_ladder_profile_read(cc_ladder_profile_entry* out, int max_entries)
{
    std::lock_guard<std::mutex> lk(cc::g_mu);
    cc::drain_locked();
    const int n = (int)cc::g_totals.size();
    if (out) {
        for (int i = 0; i < n && i < max_entries; ++i) {
            std::memset(&out[i], 0, sizeof(out[i]));
            std::strncpy(out[i].name, cc::g_totals[i].name.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = cc::g_totals[i].launches;
            out[i].ms = cc::g_totals[i].ms;
            out[i].flops = cc::g_totals[i].flops;
            out[i].bytes = cc::g_totals[i].bytes;
        }
    }
    return n;
}

long long cc_ladder_launch_count(void) { return cc::g_launches.load(); }

}  // extern "C"
