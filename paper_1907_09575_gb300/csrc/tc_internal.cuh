// Declarations shared between the preprocessing, counting and API units.
#pragma once
#include "common.cuh"

namespace tc {

constexpr int kSmallTable = 128;     // hash slots of a warp unit's table
constexpr int kSmallMaxOutdeg = 64;  // largest pivot row a warp unit takes
constexpr int kMaxSlice = 4096;      // largest pivot slice a CTA unit tables
constexpr int kMaxUnitTasks = 8192;  // 16-bit hit counters; a shared long-task queue

// One RMAT request expanded on the device (same stream as tc_generate_rmat),
// its ids shifted by vbase.
struct RmatJob {
    uint64_t key, A, B, C;
    int64_t n, vbase;
    int32_t scale;
    uint32_t t1, t2, t3;
};
RmatJob make_rmat_job(uint64_t seed, int scale, int64_t n, uint32_t t1, uint32_t t2, uint32_t t3,
                      int64_t vbase);
void generate_rmat_multi(const RmatJob* jobs_dev, const int64_t* ppre_dev, int nreq, int64_t total,
                         int32_t* src, int32_t* dst, cudaStream_t st);

void tuning_defaults(tc_tuning* t);
// Fills the knobs left to the graph's size (m edges, or the batch's total).
tc_tuning size_tuning(const tc_tuning& t, int64_t m);
void tuning_resolve(const tc_tuning* in, tc_tuning* out);  // fills zeros, clamps
bool tuning_equal(const tc_tuning& a, const tc_tuning& b);

void preprocess(tc_graph* g, const int32_t* src, const int32_t* dst, int64_t P, uint32_t flags,
                cudaStream_t st);
// Same, with optional components (vpre_host: num_comps + 1 prefix of vertex
// counts) checked and attached to the graph.
void preprocess_with_components(tc_graph* g, const int32_t* src, const int32_t* dst, int64_t P,
                                uint32_t flags, const int64_t* vpre_host, int32_t num_comps,
                                cudaStream_t st);
// Unit lists over the graphs of a view table (one graph, or a batch).
struct UnitLists {
    void* mem = nullptr;
    size_t bytes = 0;
    Unit* large = nullptr;
    Unit* small = nullptr;
    int64_t nlarge = 0, nsmall = 0;
};

// Unit building in two phases: plan_units launches the counting kernels and
// scans (the list sizes land at ps[V], pl[V] on the device); once the host
// knows them, fill_units allocates and fills the lists.
struct UnitPlan {
    Buf<int32_t> cs, cl;
    Buf<int64_t> ps, pl;
    int64_t V = 0;
    int num = 0;
    const GraphView* views = nullptr;
    const int64_t* vpre = nullptr;
    tc_tuning t{};
};
void plan_units(UnitPlan& P, const GraphView* views_dev, const int64_t* vpre_dev, int num, int64_t V,
                const tc_tuning& t, Alloc& al, cudaStream_t st);
UnitLists fill_units(UnitPlan& P, int64_t ns, int64_t nl, Alloc& al, cudaStream_t st);
void adopt_units(tc_graph* g, const UnitLists& L, const tc_tuning& tt);

tc_tuning clamp_tuning(const tc_tuning& t);
UnitLists build_unit_lists(const GraphView* views_dev, const int64_t* vpre_dev, int num, int64_t V,
                           const tc_tuning& t, Alloc& al, cudaStream_t st);
size_t count_smem_bytes(bool pv, int threads, int unit_tasks);
struct CountLaunch {
    unsigned grid = 1;
    int threads = 256;
    size_t smem = 0;
    bool pv = false;
    bool merge = false;   // the instance with the search path for short pivot rows
    bool win = false;     // the instance that counts one tile (a window of rows)
    bool buckets = false; // the instance that puts every CTA slice in 4-slot buckets (table_mode 1)
};
// Sets the kernel's shared-memory attribute and sizes the persistent grid
// (not a stream operation: call it outside stream capture).
CountLaunch prepare_count(const UnitLists& L, const tc_tuning& t, bool pv, bool win = false);
// tlow (per-vertex counts of one graph only): zeroed 32-bit counters that
// receive each task's share, or null to add it to the 64-bit accumulator.
void launch_count_raw(const CountLaunch& c, const GraphView* views_dev, const UnitLists& L,
                      const tc_tuning& t, unsigned long long* ctr, cudaStream_t st,
                      unsigned* tlow = nullptr);
// Launches the count kernel; ctr holds the queue heads and work counters.
// win: the tile instance, reading the row window (i0, i1, tail_shift) of the view
void launch_count(const GraphView* views_dev, const UnitLists& L, const tc_tuning& t, bool pv,
                  unsigned long long* ctr, cudaStream_t st, bool profile, unsigned* tlow = nullptr,
                  bool win = false);
void build_units(tc_graph* g, const tc_tuning& t, cudaStream_t st);
void count(tc_graph* g, const tc_tuning& t, uint64_t* total_dev, uint64_t* per_vertex_dev,
           cudaStream_t st);
// Per-component totals of a graph preprocessed with components.
void count_components(tc_graph* g, const tc_tuning& t, uint64_t* comp_totals_dev,
                      cudaStream_t st);
// Marks the graph's vertices with components [vpre[c], vpre[c+1]) -> c and
// checks that every pair stays inside one component (TC_EINVAL otherwise).
void attach_components(tc_graph* g, const int32_t* src_dev, const int32_t* dst_dev, int64_t P,
                       const int64_t* vpre_host, int32_t num_comps, cudaStream_t st);

// Out-of-core count (tiled.cu).  graph_offload moves the count's arrays to
// page-locked host memory and frees the device arena; count_tiled counts
// such a graph within `budget` bytes of device memory taken from `al`.
struct TiledStats {
    int64_t pivot_blocks = 0, row_blocks = 0, tiles = 0, tile_tasks = 0, h2d_bytes = 0, split_pivots = 0;
    uint64_t probes = 0;
};
void graph_offload(tc_graph* g, cudaStream_t st);
void host_copy_free(HostCopy* h);
void count_tiled(const tc_graph* g, int64_t budget, Alloc& al, const tc_tuning& t, uint64_t* total_host,
                 uint64_t* per_vertex_host, TiledStats* ts, cudaStream_t st);

}  // namespace tc
