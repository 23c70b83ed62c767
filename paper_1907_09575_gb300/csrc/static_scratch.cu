// tc_triangles_static: count a small graph without allocating device memory.
//
// Some callers cannot call cudaMalloc at the time they want a count: code
// that runs after start-up has handed all of the device's memory to another
// allocator (a framework's caching pool, a serving runtime with a fixed
// memory budget), or latency-critical loops that must not allocate at steady
// state.  This entry point runs the same preprocessing and counting kernels
// as tc_preprocess + tc_count, but carves every buffer out of one file-scope
// device array of fixed size, so it needs no allocation at all.
//
// The array is a __device__ variable: every GPU that loads the library holds
// it until the process exits.  Its device address is looked up once per
// device (cudaGetSymbolAddress, with that device current) on the first call
// made on that device.  Every call reuses the whole array from its start; the
// kernels clear what must start at zero.  Two calls whose GPU work overlaps
// (different streams, no synchronisation between them) race on the array.
#include <mutex>

#include "common.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

// Worst case for TC_STATIC_MAX_PAIRS pairs and TC_STATIC_MAX_VERTICES
// vertices with every temporary kept (the bump allocator never frees):
// about 22 MiB (the dedup hash table, 2^19 slots = 4 MiB, is the largest
// single temporary); 32 MiB leaves room for alignment.
constexpr size_t kStaticScratchBytes = 32ull << 20;

__device__ __align__(256) unsigned char g_tc_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

struct Bump {
    char* base;
    size_t cap;
    size_t used;
};

void* bump_alloc(size_t bytes, void* ctx, void* /*stream*/) {
    Bump* b = static_cast<Bump*>(ctx);
    const size_t off = (b->used + 255) & ~size_t(255);
    if (off + bytes > b->cap) return nullptr;
    b->used = off + bytes;
    return b->base + off;
}

void bump_free(void* /*ptr*/, size_t /*bytes*/, void* /*ctx*/, void* /*stream*/) {}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" tc_status tc_triangles_static(const int32_t* src_dev, const int32_t* dst_dev,
                                         int64_t num_pairs, int64_t n, uint64_t* total_dev,
                                         uint64_t* per_vertex_dev, void* stream) {
    clear_error();
    if (num_pairs < 0 || n < 0) {
        set_error("tc_triangles_static: negative size");
        return TC_EINVAL;
    }
    if (num_pairs > TC_STATIC_MAX_PAIRS || n > TC_STATIC_MAX_VERTICES) {
        set_error("tc_triangles_static: %lld pairs / %lld vertices exceed the static limits "
                  "(%d pairs, %d vertices); use tc_preprocess + tc_count",
                  (long long)num_pairs, (long long)n, TC_STATIC_MAX_PAIRS, TC_STATIC_MAX_VERTICES);
        return TC_EINVAL;
    }
    if ((num_pairs > 0 && (!src_dev || !dst_dev)) || !total_dev) {
        set_error("tc_triangles_static: NULL src_dev, dst_dev or total_dev");
        return TC_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error("tc_triangles_static: no usable current device (%s)", cudaGetErrorString(e));
        return TC_ECUDA;
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_tc_static_scratch);
            if (e != cudaSuccess || !p) {
                set_error("tc_triangles_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return TC_ECUDA;
            }
            g_static_addr[dev] = p;
        }
        base = g_static_addr[dev];
    }
    Bump bump{static_cast<char*>(base), kStaticScratchBytes, 0};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    try {
        tc_graph g;
        g.n = n;
        g.num_pairs = num_pairs;
        g.bits = std::max(1, ceil_log2_u64((uint64_t)std::max<int64_t>(n, 1)));
        g.alloc.stream = st;
        g.alloc.user = tc_allocator{bump_alloc, bump_free, &bump};
        g.alloc.has_user = true;
        g.stats.n = n;
        g.stats.num_pairs = num_pairs;
        preprocess(&g, src_dev, dst_dev, num_pairs, TC_INPUT_ON_DEVICE | TC_OFFSETS_32, st);
        tc_tuning t;
        tuning_resolve(nullptr, &t);
        count(&g, t, total_dev, per_vertex_dev, st);
    } catch (const Error& err) {
        if (err.status == TC_ENOMEM)
            set_error("tc_triangles_static: static scratch of %zu bytes exhausted", kStaticScratchBytes);
        return err.status;
    } catch (...) {
        set_error("tc_triangles_static: unexpected exception");
        return TC_ECUDA;
    }
    return TC_OK;
}
