// Per-kernel CUDA-event timing and launch counting for the library's kernels.
//
// Every launch site opens a Prof scope: the launch counter always advances;
// when profiling is on, a start and a stop event are recorded on the
// launching stream around the launch, and tc_profile_read resolves them.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace tc {
namespace {

std::atomic<long long> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;

struct Rec {
    const char* name;
    cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
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

Prof::Prof(const char* name, cudaStream_t st) : name_(name), st_(st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = take_event();
    b_ = take_event();
    if (a_ && b_) cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
}

Prof::~Prof() {
    if (!a_ || !b_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(static_cast<cudaEvent_t>(b_), st_);
    g_recs.push_back(Rec{name_, static_cast<cudaEvent_t>(a_), static_cast<cudaEvent_t>(b_)});
}

}  // namespace tc

using namespace tc;

extern "C" {

long long tc_kernel_launches(void) { return g_launches.load(); }

void tc_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_enabled.store(on != 0);
}

tc_status tc_profile_read(tc_kernel_time* out, int32_t max, int32_t* count) {
    clear_error();
    if (!count || (max > 0 && !out)) {
        set_error("tc_profile_read: NULL argument");
        return TC_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<tc_kernel_time> agg;
    for (auto& r : g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            set_error("tc_profile_read: event wait failed");
            return TC_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        size_t k = 0;
        for (; k < agg.size(); ++k)
            if (std::strncmp(agg[k].name, r.name, sizeof(agg[k].name)) == 0) break;
        if (k == agg.size()) {
            tc_kernel_time t;
            std::memset(&t, 0, sizeof(t));
            std::strncpy(t.name, r.name, sizeof(t.name) - 1);
            agg.push_back(t);
        }
        agg[k].launches += 1;
        agg[k].total_ms += ms;
    }
    *count = (int32_t)agg.size();
    for (int32_t i = 0; i < max && i < (int32_t)agg.size(); ++i) out[i] = agg[i];
    return TC_OK;
}

}  // extern "C"
