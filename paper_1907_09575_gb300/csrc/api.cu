// C ABI entry points: argument checks, error capture, allocation, ownership.
#include <chrono>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>

#include "common.cuh"
#include "tc_internal.cuh"

namespace tc {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// The library's stream-ordered memory pool of each device.  Freed blocks stay
// reserved for the next call (no release threshold): a graph's arena and its
// preprocessing scratch are tens of GB at the larger workloads, and mapping
// them afresh on every call costs more than the kernels of a small step.
// tc_release_memory hands the unused part back.
constexpr int kMaxDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[kMaxDevices] = {};

static cudaMemPool_t library_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= kMaxDevices) TC_FAIL(TC_EINVAL, "device %d out of range", dev);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        TC_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = ~0ull;
        TC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        // a block freed on another stream is reused only once its free has
        // completed, never by making this stream wait for that one: the
        // serving workers' streams stay independent
        int no = 0;
        TC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no));
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

void* Alloc::get(size_t bytes) {
    void* p = nullptr;
    if (has_user) {
        p = user.alloc(bytes, user.ctx, stream);
        if (!p) TC_FAIL(TC_ENOMEM, "device allocation of %zu bytes failed (caller allocator)", bytes);
        return p;
    }
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, library_pool(dev), stream);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        TC_FAIL(TC_ENOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return p;
}

void release_pool(int dev) {
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (dev >= 0 && dev < kMaxDevices) pool = g_pool[dev];
    }
    if (pool) TC_CUDA(cudaMemPoolTrimTo(pool, 0));
}

void Alloc::put(void* p, size_t bytes) {
    if (!p) return;
    if (has_user)
        user.free(p, bytes, user.ctx, stream);
    else
        cudaFreeAsync(p, stream);
}

void tuning_defaults(tc_tuning* t) {
    std::memset(t, 0, sizeof(*t));
    t->small_max_outdeg = kSmallMaxOutdeg;
    t->warp_unit_tasks = 0;     // chosen by the graph's size (size_tuning)
    t->cta_unit_tasks = 2048;
    t->cta_threads = 256;
    t->slice_max = kMaxSlice;
}

void tuning_resolve(const tc_tuning* in, tc_tuning* out) {
    tuning_defaults(out);
    if (!in) return;
    if (in->small_max_outdeg > 0) out->small_max_outdeg = std::min(in->small_max_outdeg, kSmallMaxOutdeg);
    if (in->warp_unit_tasks > 0) out->warp_unit_tasks = std::min(in->warp_unit_tasks, kMaxUnitTasks);
    if (in->cta_unit_tasks > 0) out->cta_unit_tasks = std::min(in->cta_unit_tasks, kMaxUnitTasks);
    if (in->cta_threads > 0) {
        int th = in->cta_threads;
        th = std::max(64, std::min(256, th));
        out->cta_threads = (th / 32) * 32;
    }
    if (in->slice_max > 0) out->slice_max = std::max(64, std::min(in->slice_max, kMaxSlice));
    out->table_mode = in->table_mode == 1 ? 1 : 0;
    out->merge_max_outdeg = std::max(0, std::min(in->merge_max_outdeg, out->small_max_outdeg));
}

// Warp units of 16 tasks spread a small graph's few units over the SMs
// (RMAT scale 14: 87 -> 48 us per count); from 2^21 edges up 64 are as fast
// or faster (scale 20: 1.87 ms either way; scale 26: 426 against 429 ms).
tc_tuning size_tuning(const tc_tuning& t, int64_t m) {
    tc_tuning out = t;
    if (out.warp_unit_tasks <= 0) out.warp_unit_tasks = m < (1ll << 21) ? 16 : 64;
    return out;
}

bool tuning_equal(const tc_tuning& a, const tc_tuning& b) {
    return std::memcmp(&a, &b, sizeof(tc_tuning)) == 0;
}

// Five timing events per host thread and device, created at the thread's
// first call on that device and kept (never destroyed: they live as long as
// the process).
struct Events {
    cudaEvent_t e[5] = {};
    Events() {
        int dev = 0;
        TC_CUDA(cudaGetDevice(&dev));
        if (dev < 0 || dev >= kMaxDevices) TC_FAIL(TC_EINVAL, "device %d out of range", dev);
        static thread_local cudaEvent_t cache[kMaxDevices][5] = {};
        for (int k = 0; k < 5; ++k) {
            if (!cache[dev][k]) TC_CUDA(cudaEventCreate(&cache[dev][k]));
            e[k] = cache[dev][k];
        }
    }
    double ms(int a, int b) const {
        float v = 0.f;
        return cudaEventElapsedTime(&v, e[a], e[b]) == cudaSuccess ? (double)v : -1.0;
    }
};

bool is_pinned(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

static thread_local tc_triangles_timing g_last_timing{};
static thread_local bool g_have_timing = false;

static void graph_release(tc_graph* g) {
    if (!g) return;
    try {
        if (g->units_mem) g->alloc.put(g->units_mem, g->units_bytes);
        if (g->tlow) g->alloc.put(g->tlow, g->tlow_bytes);
        if (g->arena) g->alloc.put(g->arena, g->arena_bytes);
    } catch (const Error&) {
    }
    host_copy_free(g->host);
    delete g;
}

static void need_device_graph(const tc_graph* g, const char* fn) {
    if (g && g->host) TC_FAIL(TC_EINVAL, "%s: the graph was offloaded to host memory (use tc_count_tiled)", fn);
}

}  // namespace tc

using namespace tc;

#define TC_API_BEGIN \
    clear_error();   \
    try {
#define TC_API_END                                               \
    }                                                            \
    catch (const ::tc::Error& e) {                               \
        return e.status;                                         \
    }                                                            \
    catch (const std::bad_alloc&) {                              \
        set_error("host allocation failed");                     \
        return TC_ENOMEM;                                        \
    }                                                            \
    catch (...) {                                                \
        set_error("unexpected exception");                       \
        return TC_ECUDA;                                         \
    }                                                            \
    return TC_OK;

extern "C" {

const char* tc_last_error(void) { return g_err; }

tc_status tc_tuning_default(tc_tuning* out) {
    TC_API_BEGIN
    if (!out) TC_FAIL(TC_EINVAL, "tc_tuning_default: out is NULL");
    tuning_defaults(out);
    TC_API_END
}

tc_status tc_preprocess(const int32_t* src, const int32_t* dst, int64_t num_pairs, int64_t n,
                        uint32_t flags, const tc_allocator* alloc, void* stream, tc_graph** out) {
    TC_API_BEGIN
    if (!out) TC_FAIL(TC_EINVAL, "tc_preprocess: out is NULL");
    if (num_pairs < 0) TC_FAIL(TC_EINVAL, "tc_preprocess: num_pairs < 0");
    if (n < 0 || n >= (int64_t)0x7fffffff) TC_FAIL(TC_EINVAL, "tc_preprocess: n outside [0, 2^31-1)");
    if (num_pairs > 0 && (!src || !dst)) TC_FAIL(TC_EINVAL, "tc_preprocess: src or dst is NULL");
    if (num_pairs > (int64_t)0x7fffffff) TC_FAIL(TC_EINVAL, "tc_preprocess: num_pairs >= 2^31");
    if ((flags & TC_OFFSETS_32) && (flags & TC_OFFSETS_64))
        TC_FAIL(TC_EINVAL, "tc_preprocess: both offset widths requested");
    if (alloc && (!alloc->alloc || !alloc->free))
        TC_FAIL(TC_EINVAL, "tc_preprocess: allocator without alloc/free");
    tc_graph* g = new tc_graph();
    g->n = n;
    g->num_pairs = num_pairs;
    g->bits = std::max(1, ceil_log2_u64((uint64_t)std::max<int64_t>(n, 1)));
    g->alloc.stream = static_cast<cudaStream_t>(stream);
    if (alloc) {
        g->alloc.user = *alloc;
        g->alloc.has_user = true;
    }
    g->stats.n = n;
    g->stats.num_pairs = num_pairs;
    try {
        preprocess(g, src, dst, num_pairs, flags, static_cast<cudaStream_t>(stream));
    } catch (...) {
        graph_release(g);
        throw;
    }
    *out = g;
    TC_API_END
}

tc_status tc_preprocess_components(const int32_t* src, const int32_t* dst, int64_t num_pairs,
                                   const int64_t* vertex_prefix, int32_t num_comps, uint32_t flags,
                                   const tc_allocator* alloc, void* stream, tc_graph** out) {
    TC_API_BEGIN
    if (!out || !vertex_prefix || num_comps <= 0)
        TC_FAIL(TC_EINVAL, "tc_preprocess_components: need out, vertex_prefix and num_comps > 0");
    if (vertex_prefix[0] != 0) TC_FAIL(TC_EINVAL, "tc_preprocess_components: vertex_prefix[0] != 0");
    for (int32_t c = 0; c < num_comps; ++c)
        if (vertex_prefix[c + 1] < vertex_prefix[c])
            TC_FAIL(TC_EINVAL, "tc_preprocess_components: vertex_prefix decreases at %d", c);
    const int64_t n = vertex_prefix[num_comps];
    if (num_pairs < 0) TC_FAIL(TC_EINVAL, "tc_preprocess_components: num_pairs < 0");
    if (n >= (int64_t)0x7fffffff) TC_FAIL(TC_EINVAL, "tc_preprocess_components: n >= 2^31-1");
    if (num_pairs > 0 && (!src || !dst)) TC_FAIL(TC_EINVAL, "tc_preprocess_components: src or dst is NULL");
    if (num_pairs > (int64_t)0x7fffffff) TC_FAIL(TC_EINVAL, "tc_preprocess_components: num_pairs >= 2^31");
    if ((flags & TC_OFFSETS_32) && (flags & TC_OFFSETS_64))
        TC_FAIL(TC_EINVAL, "tc_preprocess_components: both offset widths requested");
    if (alloc && (!alloc->alloc || !alloc->free))
        TC_FAIL(TC_EINVAL, "tc_preprocess_components: allocator without alloc/free");
    tc_graph* g = new tc_graph();
    g->n = n;
    g->num_pairs = num_pairs;
    g->bits = std::max(1, ceil_log2_u64((uint64_t)std::max<int64_t>(n, 1)));
    g->alloc.stream = static_cast<cudaStream_t>(stream);
    if (alloc) {
        g->alloc.user = *alloc;
        g->alloc.has_user = true;
    }
    g->stats.n = n;
    g->stats.num_pairs = num_pairs;
    try {
        preprocess_with_components(g, src, dst, num_pairs, flags, vertex_prefix, num_comps,
                                   static_cast<cudaStream_t>(stream));
    } catch (...) {
        graph_release(g);
        throw;
    }
    *out = g;
    TC_API_END
}

tc_status tc_count_components(tc_graph* g, const tc_tuning* tune, uint64_t* comp_totals_dev,
                              void* stream) {
    TC_API_BEGIN
    if (!g || !comp_totals_dev) TC_FAIL(TC_EINVAL, "tc_count_components: NULL argument");
    need_device_graph(g, "tc_count_components");
    if (g->num_comps <= 0 || !g->comp)
        TC_FAIL(TC_EINVAL, "tc_count_components: graph was not preprocessed with components");
    tc_tuning t;
    tuning_resolve(tune, &t);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    g->alloc.stream = st;
    count_components(g, t, comp_totals_dev, st);
    TC_API_END
}

tc_status tc_count(tc_graph* g, const tc_tuning* tune, uint64_t* total_host,
                   uint64_t* total_dev, uint64_t* per_vertex_dev, void* stream) {
    TC_API_BEGIN
    if (!g) TC_FAIL(TC_EINVAL, "tc_count: graph is NULL");
    if (!total_host && !total_dev && !per_vertex_dev)
        TC_FAIL(TC_EINVAL, "tc_count: no output requested");
    need_device_graph(g, "tc_count");
    tc_tuning t;
    tuning_resolve(tune, &t);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    g->alloc.stream = st;
    count(g, t, total_dev, per_vertex_dev, st);
    if (total_host) {
        unsigned long long v = 0;
        TC_CUDA(cudaMemcpyAsync(&v, g->counters + CTR_TOTAL, sizeof(v), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        *total_host = v;
    }
    TC_API_END
}

tc_status tc_triangles(const int32_t* src_host, const int32_t* dst_host, int64_t num_pairs,
                       int64_t n, uint32_t flags, void* stream, uint64_t* total_host,
                       uint64_t* per_vertex_host) {
    TC_API_BEGIN
    if (!total_host) TC_FAIL(TC_EINVAL, "tc_triangles: total_host is NULL");
    if (flags & TC_INPUT_ON_DEVICE) TC_FAIL(TC_EINVAL, "tc_triangles: takes host inputs");
    if (num_pairs < 0) TC_FAIL(TC_EINVAL, "tc_triangles: num_pairs < 0");
    if (n < 0 || n >= (int64_t)0x7fffffff) TC_FAIL(TC_EINVAL, "tc_triangles: n outside [0, 2^31-1)");
    if (num_pairs > 0 && (!src_host || !dst_host)) TC_FAIL(TC_EINVAL, "tc_triangles: src or dst is NULL");
    if (num_pairs > (int64_t)0x7fffffff) TC_FAIL(TC_EINVAL, "tc_triangles: num_pairs >= 2^31");
    if ((flags & TC_OFFSETS_32) && (flags & TC_OFFSETS_64))
        TC_FAIL(TC_EINVAL, "tc_triangles: both offset widths requested");
    const auto wall0 = std::chrono::steady_clock::now();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Events ev;
    tc_triangles_timing tm{};
    tm.input_pinned = num_pairs > 0 && is_pinned(src_host) && is_pinned(dst_host);
    tc_graph* g = new tc_graph();
    g->n = n;
    g->num_pairs = num_pairs;
    g->bits = std::max(1, ceil_log2_u64((uint64_t)std::max<int64_t>(n, 1)));
    g->alloc.stream = st;
    g->stats.n = n;
    g->stats.num_pairs = num_pairs;
    g->ev_uploaded = ev.e[1];
    uint64_t* pv = nullptr;
    try {
        TC_CUDA(cudaEventRecord(ev.e[0], st));
        preprocess(g, src_host, dst_host, num_pairs, flags, st);
        TC_CUDA(cudaEventRecord(ev.e[2], st));
        tc_tuning t;
        tuning_resolve(nullptr, &t);
        if (per_vertex_host && n > 0) pv = static_cast<uint64_t*>(g->alloc.get(sizeof(uint64_t) * n));
        count(g, t, nullptr, pv, st);
        TC_CUDA(cudaEventRecord(ev.e[3], st));
        unsigned long long v = 0;
        TC_CUDA(cudaMemcpyAsync(&v, g->counters + CTR_TOTAL, sizeof(v), cudaMemcpyDeviceToHost, st));
        if (pv)
            TC_CUDA(cudaMemcpyAsync(per_vertex_host, pv, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaEventRecord(ev.e[4], st));
        TC_CUDA(cudaStreamSynchronize(st));
        *total_host = v;
    } catch (...) {
        if (pv) g->alloc.put(pv, sizeof(uint64_t) * n);
        g->ev_uploaded = nullptr;
        graph_release(g);
        throw;
    }
    if (pv) g->alloc.put(pv, sizeof(uint64_t) * n);
    tm.h2d_issue_ms = g->upload_issue_ms;
    tm.upload_method = g->upload_method;
    tm.ce_slice_gbs = g->upload_probe_gbs[0];
    tm.sm_slice_gbs = g->upload_probe_gbs[1];
    g->ev_uploaded = nullptr;
    graph_release(g);
    tm.h2d_ms = ev.ms(0, 1);
    tm.preprocess_ms = ev.ms(1, 2);
    tm.count_ms = ev.ms(2, 3);
    tm.d2h_ms = ev.ms(3, 4);
    tm.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    g_last_timing = tm;
    g_have_timing = true;
    TC_API_END
}

tc_status tc_triangles_get_timing(tc_triangles_timing* out) {
    TC_API_BEGIN
    if (!out) TC_FAIL(TC_EINVAL, "tc_triangles_get_timing: out is NULL");
    if (!g_have_timing) TC_FAIL(TC_EINVAL, "tc_triangles_get_timing: no tc_triangles call on this thread yet");
    *out = g_last_timing;
    TC_API_END
}

tc_status tc_graph_get_stats(const tc_graph* g, tc_graph_stats* out) {
    TC_API_BEGIN
    if (!g || !out) TC_FAIL(TC_EINVAL, "tc_graph_get_stats: NULL argument");
    *out = g->stats;
    out->small_units = g->n_small;
    out->large_units = g->n_large;
    out->device_bytes = (int64_t)(g->arena_bytes + g->units_bytes);
    TC_API_END
}

tc_status tc_graph_offload(tc_graph* g, void* stream) {
    TC_API_BEGIN
    if (!g) TC_FAIL(TC_EINVAL, "tc_graph_offload: graph is NULL");
    graph_offload(g, static_cast<cudaStream_t>(stream));
    TC_API_END
}

tc_status tc_count_tiled(const tc_graph* g, int64_t device_budget_bytes, const tc_allocator* alloc,
                         const tc_tuning* tune, uint64_t* total_host, uint64_t* per_vertex_host,
                         tc_tiled_stats* stats, void* stream) {
    TC_API_BEGIN
    if (!g || !total_host) TC_FAIL(TC_EINVAL, "tc_count_tiled: NULL graph or total_host");
    if (!g->host) TC_FAIL(TC_EINVAL, "tc_count_tiled: the graph is on the device (tc_graph_offload first)");
    if (alloc && (!alloc->alloc || !alloc->free))
        TC_FAIL(TC_EINVAL, "tc_count_tiled: allocator without alloc/free");
    tc_tuning t;
    tuning_resolve(tune, &t);
    Alloc al;
    al.stream = static_cast<cudaStream_t>(stream);
    if (alloc) {
        al.user = *alloc;
        al.has_user = true;
    }
    TiledStats ts;
    count_tiled(g, device_budget_bytes, al, t, total_host, per_vertex_host, &ts, al.stream);
    if (stats) {
        stats->pivot_blocks = ts.pivot_blocks;
        stats->row_blocks = ts.row_blocks;
        stats->tiles = ts.tiles;
        stats->tile_tasks = ts.tile_tasks;
        stats->h2d_bytes = ts.h2d_bytes;
        stats->probes = ts.probes;
        stats->split_pivots = ts.split_pivots;
    }
    TC_API_END
}

tc_status tc_count_get_stats(const tc_graph* g, tc_count_stats* out, void* stream) {
    TC_API_BEGIN
    if (!g || !out) TC_FAIL(TC_EINVAL, "tc_count_get_stats: NULL argument");
    need_device_graph(g, "tc_count_get_stats");
    unsigned long long c[CTR_COUNT];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TC_CUDA(cudaMemcpyAsync(c, g->counters, sizeof(c), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    out->triangles = c[CTR_TOTAL];
    for (int k = 0; k < 2; ++k) {
        out->units[k] = c[CTR_UNITS + k];
        out->tasks[k] = c[CTR_TASKS + k];
        out->probes[k] = c[CTR_PROBES + k];
        out->staged[k] = c[CTR_STAGED + k];
    }
    TC_API_END
}

void tc_graph_free(tc_graph* g) { graph_release(g); }

tc_status tc_selftest_wait_timeout(int64_t spin_limit, void* stream) {
    TC_API_BEGIN
    if (spin_limit < 1 || spin_limit > (1 << 20))
        TC_FAIL(TC_EINVAL, "tc_selftest_wait_timeout: spin_limit outside [1, 2^20]");
    Alloc al;
    al.stream = static_cast<cudaStream_t>(stream);
    if (selftest_wait_timeout((long)spin_limit, al, al.stream))
        TC_FAIL(TC_ETIMEOUT, "tc_selftest_wait_timeout: the bounded wait ran out and reported it");
    TC_FAIL(TC_ECUDA, "tc_selftest_wait_timeout: the wait ended without its word being published");
    TC_API_END
}

tc_status tc_memory_get_stats(int device, int32_t reset_high, tc_memory_stats* out) {
    TC_API_BEGIN
    if (!out || device < 0 || device >= kMaxDevices)
        TC_FAIL(TC_EINVAL, "tc_memory_get_stats: NULL out or device %d out of range", device);
    cudaMemPool_t pool = library_pool(device);
    uint64_t v[4] = {0, 0, 0, 0};
    TC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v[0]));
    TC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &v[1]));
    TC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v[2]));
    TC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v[3]));
    out->reserved = (int64_t)v[0];
    out->reserved_high = (int64_t)v[1];
    out->used = (int64_t)v[2];
    out->used_high = (int64_t)v[3];
    if (reset_high) {
        uint64_t zero = 0;
        TC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &zero));
        TC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    TC_API_END
}

tc_status tc_release_memory(int device) {
    TC_API_BEGIN
    if (device >= kMaxDevices) TC_FAIL(TC_EINVAL, "tc_release_memory: device %d out of range", device);
    if (device >= 0) {
        release_pool(device);
    } else {
        for (int d = 0; d < kMaxDevices; ++d) release_pool(d);
    }
    TC_API_END
}

}  // extern "C"
