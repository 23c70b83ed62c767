// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tc {

// ---------------------------------------------------------------------------
// error reporting: a thread-local message plus a status code
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

struct Error {
    tc_status status;
};

#define TC_FAIL(st, ...)                  \
    do {                                  \
        ::tc::set_error(__VA_ARGS__);     \
        throw ::tc::Error{st};            \
    } while (0)

#define TC_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            TC_FAIL(TC_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                    __FILE__, __LINE__);                                           \
    } while (0)

#define TC_LAUNCH_CHECK() TC_CUDA(cudaGetLastError())

// Scope around one kernel launch: counts it and, when profiling is on,
// brackets it with CUDA events on the launching stream.
class Prof {
public:
    Prof(const char* name, cudaStream_t st);
    ~Prof();
    Prof(const Prof&) = delete;
    Prof& operator=(const Prof&) = delete;

private:
    const char* name_;
    cudaStream_t st_;
    void* a_ = nullptr;
    void* b_ = nullptr;
};

// ---------------------------------------------------------------------------
// device memory through the caller's allocator (or the library's pool)
// ---------------------------------------------------------------------------
struct Alloc {
    tc_allocator user{};
    bool has_user = false;
    cudaStream_t stream = nullptr;

    void* get(size_t bytes);
    void put(void* p, size_t bytes);
};

// RAII scratch buffer on an Alloc.
template <class T>
struct Buf {
    Alloc* a = nullptr;
    T* p = nullptr;
    size_t bytes = 0;
    Buf() = default;
    Buf(Alloc& al, size_t count) : a(&al), bytes(sizeof(T) * (count ? count : 1)) {
        p = static_cast<T*>(al.get(bytes));
    }
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    Buf(Buf&& o) noexcept : a(o.a), p(o.p), bytes(o.bytes) { o.p = nullptr; }
    Buf& operator=(Buf&& o) noexcept {
        release();
        a = o.a; p = o.p; bytes = o.bytes; o.p = nullptr;
        return *this;
    }
    ~Buf() { release(); }
    void release() {
        if (p && a) a->put(p, bytes);
        p = nullptr;
    }
    T* get() const { return p; }
};

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

inline int ceil_log2_u64(uint64_t x) {  // smallest b with 2^b >= x (x >= 1)
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

inline int num_sms() {
    static int s = -1;
    if (s < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        if (s <= 0) s = 1;
    }
    return s;
}

inline unsigned grid_for(int64_t items, int threads, int64_t cap = 0) {
    int64_t g = (items + threads - 1) / threads;
    if (g < 1) g = 1;
    if (cap > 0 && g > cap) g = cap;
    if (g > 0x7fffffff) g = 0x7fffffff;
    return (unsigned)g;
}

// ---------------------------------------------------------------------------
// device-wide primitives (scan.cu, radix.cu)
// ---------------------------------------------------------------------------

// out[i] = sum_{k<i} in[i]; *total_dev (if non-null) = sum of all.  Any of
// (int32, int64) in, int64 out.  in may alias out.
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t count, int64_t* total_dev,
                        Alloc& al, cudaStream_t st);
void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t count,
                               int64_t* total_dev, Alloc& al, cudaStream_t st);
// two int32 arrays of the same length (one launch when they are short)
void exclusive_scan2_i32_to_i64(const int32_t* in0, int64_t* out0, int64_t* total0, const int32_t* in1,
                                int64_t* out1, int64_t* total1, int64_t count, Alloc& al, cudaStream_t st);

// Stable LSD radix sort of 64-bit keys on bits [lo, hi).  Sorted keys end up
// in *keys (the two buffers may be swapped).  count <= 2^31 - 1.  With
// err_dev, a look-back timeout ORs 4 into *err_dev and the call returns
// without synchronising; without it, the call synchronises and throws
// TC_ETIMEOUT itself.
void radix_sort_u64(uint64_t** keys, uint64_t** alt, int64_t count, int lo, int hi,
                    Alloc& al, cudaStream_t st, int* err_dev = nullptr);
// One warp waits, with the radix look-back's bounded wait, on a word nothing
// publishes; true when the bound ran out and was reported (synchronises).
bool selftest_wait_timeout(long limit, Alloc& al, cudaStream_t st);

}  // namespace tc

// The graph object behind the opaque handle.
struct tc_graph {
    int64_t n = 0, m = 0, num_pairs = 0;
    int bits = 1;               // ceil(log2(n)), >= 1
    bool off64 = false;
    tc::Alloc alloc;
    void* arena = nullptr;
    size_t arena_bytes = 0;

    // device views into the arena
    void* off = nullptr;        // U offsets, n+1 (int32 or int64)
    int32_t* adj = nullptr;     // U columns, m, rows ascending
    int32_t* perm = nullptr;    // old id -> new label, n
    int64_t* loff = nullptr;    // task list offsets per pivot j, n+1
    struct Task* tasks = nullptr;   // <j,i,k> tasks grouped by pivot j
    struct Unit* small_units = nullptr;
    struct Unit* large_units = nullptr;
    unsigned long long* counters = nullptr;  // queue heads and totals (device)
    struct GraphView* view = nullptr;        // device copy of this graph's view
    struct GraphView* view_comp = nullptr;   // same, hits credited per component
    int32_t* comp = nullptr;                 // component of each new label (or null)
    unsigned long long* comp_totals = nullptr;
    int32_t num_comps = 0;
    uint64_t* tnew = nullptr;   // per-vertex accumulator in new labels, n
    unsigned* tlow = nullptr;   // 32-bit per-task shares (per-vertex counts), n, on demand
    size_t tlow_bytes = 0;

    // instrumentation of a host-input preprocessing (set by tc_triangles):
    // an event recorded on the stream once the pairs are uploaded, and the
    // host time spent issuing the upload (long when the source is pageable)
    cudaEvent_t ev_uploaded = nullptr;
    double upload_issue_ms = 0.0;
    int upload_method = 0;      // 1 copy engine, 2 SM loads of page-locked memory
    double upload_probe_gbs[2] = {0.0, 0.0};   // the timed slices: copy engine, SM loads

    // after tc_graph_offload: the count's arrays in page-locked host memory
    // (and no device arena)
    struct HostCopy* host = nullptr;

    int64_t n_tasks = 0, n_small = 0, n_large = 0;
    void* units_mem = nullptr;      // small units, then large units
    size_t units_bytes = 0;
    tc_tuning units_tuning{};       // tuning the unit lists were built for
    tc_graph_stats stats{};
};

// Page-locked host copies of a graph's count arrays (tc_graph_offload).
struct HostCopy {
    void* off = nullptr;        // n+1, int32 or int64 as tc_graph::off64
    int32_t* adj = nullptr;     // m
    int64_t* loff = nullptr;    // n+1
    struct Task* tasks = nullptr;   // n_tasks
    int32_t* perm = nullptr;    // n
};

// A <j,i,k> task: edge (i,j) of U with the part of U_i after j nonempty.
struct Task {
    int64_t start;   // index in adj of the first entry of U_i after j
    int32_t len;     // number of entries of U_i after j (> 0)
    int32_t i;       // row (new label), for per-vertex credit
};

// A work unit: graph g (index into the view table), pivot j, a slice of U_j
// (for pivots larger than one table) and a contiguous range of j's tasks.
struct Unit {
    int32_t j;
    int32_t slice;      // slice index of U_j (entries [slice*S, slice*S+S))
    int32_t g;
    int32_t pad;
    int64_t t0;         // first task (index into tasks)
    int64_t t1;         // one past the last task
};

// What the count kernel needs of one graph.
struct GraphView {
    const void* off;              // U offsets (int32 or int64)
    const int32_t* adj;           // U columns
    const int64_t* loff;          // task offsets per pivot
    const Task* tasks;
    unsigned long long* tnew;     // per-vertex accumulator (new labels), or null
    unsigned long long* total;    // where this graph's hits are added
    const int32_t* comp;          // component of each new label, or null
    unsigned long long* comp_totals;   // per-component totals (with comp)
    int64_t n;
    int32_t off64;
    int32_t jbase;                // label of local pivot 0 (tiles of a host-resident
                                  // graph index pivots from their block's start)
    int32_t i0, i1;               // tiles: the rows counted by this launch ...
    int64_t tail_shift;           // ... whose entries start this far into adj
};

// Device counters of one count: queue heads, the total, and work done by the
// warp kernel (index 0) and the CTA kernel (index 1).
enum : int {
    CTR_SMALL_HEAD = 0,
    CTR_LARGE_HEAD = 1,
    CTR_TOTAL = 2,
    CTR_UNITS = 3,    // +0 warp, +1 CTA
    CTR_TASKS = 5,
    CTR_PROBES = 7,
    CTR_STAGED = 9,
    CTR_COUNT = 16
};
