// Batched counting: many preprocessed graphs counted by one persistent
// launch, replayed from a captured CUDA graph, with an autotuner that picks
// the work-unit knobs per degree profile.
//
// The batch lists its graphs by ascending edge count in a device view table;
// the unit lists cover all graphs (heaviest pivots of the largest graph
// first) and each unit adds its hits to its own graph's total.  Counting the
// batch is one cudaGraphLaunch: two memsets and the count kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc_internal.cuh"

struct tc_batch {
    int num = 0;
    std::vector<const tc_graph*> graphs;   // table order: ascending m
    std::vector<int32_t> slot;             // caller's index of each table entry
    tc::Alloc alloc;
    cudaStream_t cap = nullptr;            // private stream the launch is captured on
    void* mem = nullptr;
    size_t mem_bytes = 0;
    GraphView* views = nullptr;            // device, num
    int64_t* vpre = nullptr;               // device, num + 1
    uint64_t* totals = nullptr;            // device, num (caller's order)
    unsigned long long* ctr = nullptr;     // device, CTR_COUNT
    tc::UnitLists units;
    tc_tuning tuning{};
    int64_t V = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace tc {
namespace {

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

void drop_exec(tc_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// (Re)build the unit lists for a tuning and capture the counting launch.
void set_tuning(tc_batch* b, const tc_tuning& t) {
    int64_t m = 0;
    for (const tc_graph* g : b->graphs) m += g->m;
    const tc_tuning tt = clamp_tuning(size_tuning(t, m));
    drop_exec(b);
    if (b->units.mem) {
        b->alloc.put(b->units.mem, b->units.bytes);
        b->units = UnitLists{};
    }
    b->alloc.stream = b->cap;
    b->units = build_unit_lists(b->views, b->vpre, b->num, b->V, tt, b->alloc, b->cap);
    TC_CUDA(cudaStreamSynchronize(b->cap));
    b->tuning = tt;
    const CountLaunch c = prepare_count(b->units, tt, false);
    TC_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemsetAsync(b->ctr, 0, sizeof(unsigned long long) * CTR_COUNT, b->cap);
    cudaError_t e2 = cudaMemsetAsync(b->totals, 0, sizeof(uint64_t) * (size_t)b->num, b->cap);
    bool launched = true;
    try {
        launch_count_raw(c, b->views, b->units, tt, b->ctr, b->cap);
    } catch (const Error&) {
        launched = false;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(b->cap, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || !launched || !g) {
        if (g) cudaGraphDestroy(g);
        TC_FAIL(TC_ECUDA, "batch: capturing the count launch failed (%s)",
                cudaGetErrorString(e3 != cudaSuccess ? e3 : (e1 != cudaSuccess ? e1 : e2)));
    }
    b->graph = g;
    TC_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
}

void batch_release(tc_batch* b) {
    if (!b) return;
    drop_exec(b);
    try {
        if (b->units.mem) b->alloc.put(b->units.mem, b->units.bytes);
        if (b->mem) b->alloc.put(b->mem, b->mem_bytes);
    } catch (const Error&) {
    }
    if (b->cap) {
        cudaStreamSynchronize(b->cap);
        cudaStreamDestroy(b->cap);
    }
    delete b;
}

// Degree-profile signature of a batch: log2 buckets of the graph count, the
// mean edges per graph, the largest pivot row and the mean tail length.
std::string signature(const tc_batch* b) {
    double m = 0, probes = 0, tasks = 0;
    int64_t maxout = 0;
    for (const tc_graph* g : b->graphs) {
        m += (double)g->stats.m;
        probes += (double)g->stats.probes;
        tasks += (double)g->stats.tasks;
        maxout = std::max<int64_t>(maxout, g->stats.max_outdeg);
    }
    auto lb = [](double x) { return (int)std::floor(std::log2(std::max(x, 1.0))); };
    char buf[128];
    snprintf(buf, sizeof(buf), "n%d-m%d-o%d-t%d", lb((double)b->num), lb(m / b->num), lb((double)maxout),
             lb(tasks > 0 ? probes / tasks : 1.0));
    return buf;
}

std::mutex g_tune_mu;
std::map<std::string, tc_tuning> g_tune_cache;

float time_batch(tc_batch* b, int reps, cudaStream_t st) {
    cudaEvent_t e0, e1;
    TC_CUDA(cudaEventCreate(&e0));
    TC_CUDA(cudaEventCreate(&e1));
    TC_CUDA(cudaGraphLaunch(b->exec, st));   // warm
    TC_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) TC_CUDA(cudaGraphLaunch(b->exec, st));
    TC_CUDA(cudaEventRecord(e1, st));
    TC_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / (float)std::max(reps, 1);
}

}  // namespace
}  // namespace tc

using namespace tc;

#define TC_API_BEGIN \
    clear_error();   \
    try {
#define TC_API_END                               \
    }                                            \
    catch (const ::tc::Error& e) {               \
        return e.status;                         \
    }                                            \
    catch (const std::bad_alloc&) {              \
        set_error("host allocation failed");     \
        return TC_ENOMEM;                        \
    }                                            \
    catch (...) {                                \
        set_error("unexpected exception");       \
        return TC_ECUDA;                         \
    }                                            \
    return TC_OK;

extern "C" {

tc_status tc_batch_create(const tc_graph* const* graphs, int32_t num, const tc_tuning* tune,
                          void* stream, tc_batch** out) {
    TC_API_BEGIN
    if (!graphs || num <= 0 || !out) TC_FAIL(TC_EINVAL, "tc_batch_create: need graphs, num > 0, out");
    for (int32_t k = 0; k < num; ++k) {
        if (!graphs[k]) TC_FAIL(TC_EINVAL, "tc_batch_create: graph %d is NULL", k);
        if (graphs[k]->host) TC_FAIL(TC_EINVAL, "tc_batch_create: graph %d was offloaded to host memory", k);
    }
    tc_batch* b = new tc_batch();
    try {
        b->num = num;
        TC_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        b->alloc.stream = b->cap;
        std::vector<int32_t> order(num);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t x, int32_t y) { return graphs[x]->m < graphs[y]->m; });
        for (int32_t k : order) {
            b->graphs.push_back(graphs[k]);
            b->slot.push_back(k);
        }
        const size_t sv = align_up(sizeof(GraphView) * (size_t)num);
        const size_t sp = align_up(sizeof(int64_t) * (size_t)(num + 1));
        const size_t st_ = align_up(sizeof(uint64_t) * (size_t)num);
        const size_t sc = align_up(sizeof(unsigned long long) * CTR_COUNT);
        b->mem_bytes = sv + sp + st_ + sc;
        b->mem = b->alloc.get(b->mem_bytes);
        char* a = static_cast<char*>(b->mem);
        b->views = reinterpret_cast<GraphView*>(a);
        b->vpre = reinterpret_cast<int64_t*>(a + sv);
        b->totals = reinterpret_cast<uint64_t*>(a + sv + sp);
        b->ctr = reinterpret_cast<unsigned long long*>(a + sv + sp + st_);
        std::vector<GraphView> hv(num);
        std::vector<int64_t> hp(num + 1, 0);
        for (int32_t k = 0; k < num; ++k) {
            const tc_graph* g = b->graphs[k];
            GraphView v{};
            v.off = g->off;
            v.adj = g->adj;
            v.loff = g->loff;
            v.tasks = g->tasks;
            v.tnew = nullptr;
            v.total = reinterpret_cast<unsigned long long*>(b->totals + b->slot[k]);
            v.n = g->n;
            v.off64 = g->off64 ? 1 : 0;
            hv[k] = v;
            hp[k + 1] = hp[k] + g->n;
        }
        b->V = hp[num];
        TC_CUDA(cudaMemcpyAsync(b->views, hv.data(), sizeof(GraphView) * num, cudaMemcpyHostToDevice, b->cap));
        TC_CUDA(cudaMemcpyAsync(b->vpre, hp.data(), sizeof(int64_t) * (num + 1), cudaMemcpyHostToDevice, b->cap));
        TC_CUDA(cudaStreamSynchronize(b->cap));
        tc_tuning t;
        tuning_resolve(tune, &t);
        set_tuning(b, t);
    } catch (...) {
        batch_release(b);
        throw;
    }
    (void)stream;
    *out = b;
    TC_API_END
}

tc_status tc_batch_count(tc_batch* b, uint64_t* totals_dev, void* stream) {
    TC_API_BEGIN
    if (!b || !b->exec) TC_FAIL(TC_EINVAL, "tc_batch_count: batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        Prof prof_("k_count_batch", st);
        TC_CUDA(cudaGraphLaunch(b->exec, st));
    }
    if (totals_dev && totals_dev != b->totals)
        TC_CUDA(cudaMemcpyAsync(totals_dev, b->totals, sizeof(uint64_t) * (size_t)b->num,
                                cudaMemcpyDeviceToDevice, st));
    TC_API_END
}

tc_status tc_batch_autotune(tc_batch* b, int32_t reps, tc_tuning* chosen, void* stream) {
    TC_API_BEGIN
    if (!b) TC_FAIL(TC_EINVAL, "tc_batch_autotune: batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::string sig = signature(b);
    tc_tuning best = b->tuning;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(sig);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        float best_ms = 1e30f;
        const int small_max[] = {16, 64};
        const int warp_tasks[] = {64, 512};
        const int cta_tasks[] = {512, 4096};
        const int threads[] = {128, 256};
        const int merge_max[] = {0, 16};   // short pivot rows searched instead of tabled
        for (int a : small_max)
            for (int w : warp_tasks)
                for (int c : cta_tasks)
                    for (int th : threads)
                        for (int mm : merge_max) {
                            tc_tuning cand;
                            tuning_defaults(&cand);
                            cand.small_max_outdeg = a;
                            cand.warp_unit_tasks = w;
                            cand.cta_unit_tasks = c;
                            cand.cta_threads = th;
                            cand.merge_max_outdeg = mm;
                            tc_tuning res;
                            tuning_resolve(&cand, &res);
                            set_tuning(b, res);
                            const float ms = time_batch(b, std::max(reps, 1), st);
                            if (ms < best_ms) {
                                best_ms = ms;
                                best = b->tuning;
                            }
                        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[sig] = best;
    }
    set_tuning(b, best);
    if (chosen) *chosen = b->tuning;
    TC_API_END
}

tc_status tc_batch_get_count_stats(const tc_batch* b, tc_count_stats* out, void* stream) {
    TC_API_BEGIN
    if (!b || !out) TC_FAIL(TC_EINVAL, "tc_batch_get_count_stats: NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long c[CTR_COUNT];
    std::vector<uint64_t> tot(b->num);
    TC_CUDA(cudaMemcpyAsync(c, b->ctr, sizeof(c), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(tot.data(), b->totals, sizeof(uint64_t) * b->num, cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    out->triangles = std::accumulate(tot.begin(), tot.end(), (uint64_t)0);
    for (int k = 0; k < 2; ++k) {
        out->units[k] = c[CTR_UNITS + k];
        out->tasks[k] = c[CTR_TASKS + k];
        out->probes[k] = c[CTR_PROBES + k];
        out->staged[k] = c[CTR_STAGED + k];
    }
    TC_API_END
}

void tc_batch_free(tc_batch* b) { batch_release(b); }

tc_status tc_count_batch(const tc_graph* const* graphs, int32_t num, const tc_tuning* tune,
                         uint64_t* totals_dev, void* stream) {
    TC_API_BEGIN
    if (!totals_dev) TC_FAIL(TC_EINVAL, "tc_count_batch: totals_dev is NULL");
    tc_batch* b = nullptr;
    tc_status s = tc_batch_create(graphs, num, tune, stream, &b);
    if (s != TC_OK) return s;
    s = tc_batch_count(b, totals_dev, stream);
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    batch_release(b);
    if (s != TC_OK) return s;
    TC_API_END
}

}  // extern "C"
