/*
 * tc.h -- C ABI of the GB300 exact triangle counter.
 *
 * The library counts the triangles of a simple undirected graph exactly, by
 * the method of Tom and Karypis, "A 2D Parallel Triangle Counting Algorithm
 * for Distributed-Memory Architectures" (ICPP 2019):
 *
 *   - the graph is made simple and undirected (Section 2, Section 6.1),
 *   - vertices are relabelled in non-decreasing degree (Section 3.1,
 *     Section 5.3 "Reorder vertices based on non-decreasing degree"),
 *   - each edge is kept once, in the upper triangular part U (Section 5.3
 *     "Create the upper and the lower triangular portion"), rows sorted,
 *   - every edge (i,j) of U contributes c_ij = sum_{k>j} u_ik u_jk (Eq. 1),
 *     the total being the sum of c_ij over U (Eq. 2); equivalently the
 *     entries of UL at the nonzeros of U (Eq. 6, Eq. 7), summed.
 *
 * Counting follows the paper's <j,i,k> map-based enumeration (Section 3.1,
 * Section 5.1 last paragraph): for each vertex j the row U_j is hashed once
 * and probed by the part after j of every row U_i with i in column j.
 *
 * All entry points return a tc_status and never abort or throw.  On failure
 * tc_last_error() gives a message (per host thread) and no output is written.
 * All device pointers are CUDA device (or managed) memory of the current
 * device; `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Entry points that must read a size back from the device
 * synchronise the stream; each says so.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TC_API __attribute__((visibility("default")))
#else
#define TC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TC_OK = 0,
    TC_EINVAL = 1,     /* bad argument: NULL pointer, negative size, id outside [0,n) */
    TC_ENOMEM = 2,     /* device allocation failed (including an injected failure) */
    TC_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    TC_ETIMEOUT = 4,   /* a bounded device wait ran out (serving queue) */
    TC_EBUSY = 5,      /* over the admission budget (serving) */
    TC_EUNSUPPORTED = 6
} tc_status;

/* Opaque preprocessed graph.  Owns one device arena (the single-blob layout
 * of Section 5.2, last paragraph) holding the degree-ordered U in CSR, the
 * <j,i,k> task lists, the work units and the relabelling. */
typedef struct tc_graph tc_graph;

/* Caller-supplied device allocator; NULL selects the library's own
 * stream-ordered memory pool on the current device, allocated and freed on
 * the call's stream.  That pool keeps freed memory reserved for later calls
 * (tc_release_memory returns it).  alloc returns NULL on failure.  free
 * receives the size that was allocated. */
typedef struct {
    void* (*alloc)(size_t bytes, void* ctx, void* stream);
    void (*free)(void* ptr, size_t bytes, void* ctx, void* stream);
    void* ctx;
} tc_allocator;

/* tc_preprocess flags */
#define TC_INPUT_ON_DEVICE 0x1u  /* src/dst are device pointers (else host) */
#define TC_OFFSETS_32      0x2u  /* force 32-bit CSR offsets (EINVAL if m >= 2^31) */
#define TC_OFFSETS_64      0x4u  /* force 64-bit CSR offsets */
/* With neither offset flag, 32-bit offsets are used when m < 2^31. */

/* Counting knobs.  Zero in any field selects its default (some defaults
 * depend on the graph's size; tc_tuning_default leaves those at zero).  The
 * count never depends on them; only speed does. */
typedef struct {
    int32_t small_max_outdeg;  /* pivots with |U_j| <= this go to warp units (<= 64) */
    int32_t warp_unit_tasks;   /* tasks per warp unit (<= 8192); 0: 16 for graphs of
                                  fewer than 2^21 edges, else 64 */
    int32_t cta_unit_tasks;    /* tasks per CTA unit (<= 8192) */
    int32_t cta_threads;       /* threads per CTA of the large-pivot kernel (64..256) */
    int32_t slice_max;         /* pivot entries tabled at once by one CTA (64..4096) */
    int32_t table_mode;        /* 0: a bitmap when the pivot's label span fits (the
                                  direct-index case of Section 5.2), else an exact
                                  tag table (a hash that is a bijection of the
                                  label); 1: the AND-hash of Section 5.2 in 4-slot
                                  buckets for every pivot (the hashed-pivot
                                  ablation; merge_max_outdeg is then not used) */
    int32_t merge_max_outdeg;  /* warp-unit pivots with |U_j| <= this build no table:
                                  each lane searches the sorted row (the list-based
                                  traversal of Section 3.1); 0 = never (<= 64) */
    int32_t reserved;
} tc_tuning;

/* Graph facts, computed during preprocessing. */
typedef struct {
    int64_t n;              /* vertices */
    int64_t num_pairs;      /* input pairs */
    int64_t m;              /* simple undirected edges = nnz(U) */
    int64_t max_deg;        /* max d(v) */
    int64_t max_outdeg;     /* max |U_v| */
    int64_t tasks;          /* edges (i,j) of U with a nonempty part of U_i after j */
    uint64_t probes;        /* sum over tasks of |{k in U_i : k > j}| = sum_i C(|U_i|,2) */
    int64_t small_units;    /* work units of the warp kernel */
    int64_t large_units;    /* work units of the CTA kernel */
    int64_t device_bytes;   /* bytes held by the graph's arena */
    int32_t offset_bytes;   /* 4 or 8 */
    int32_t pad;
    uint64_t probes_ijk;    /* the probes of the <i,j,k> order (Section 3.1):
                               sum over (i,j) in U of |U_j| = sum_j d-(j) d+(j) */
} tc_graph_stats;

/*
 * tc_preprocess -- Section 5.3 on one device: simple-graph conversion, degree
 * counting, relabelling in non-decreasing (degree, id) order, orientation into
 * U, CSR build with sorted rows, the <j,i,k> task lists (Section 5.1, last
 * paragraph) and degree-binned work units (the doubly sparse list of
 * Section 5.2 becomes the unit list: empty rows get no unit).
 *
 *   src, dst   num_pairs vertex ids each (int32, in [0, n)); pair e is the
 *              undirected edge {src[e], dst[e]}.  Self-loops are dropped and
 *              duplicates (either direction) merged.  Host pointers unless
 *              flags has TC_INPUT_ON_DEVICE.  Read only; the caller keeps
 *              ownership and may free them once the call returns.
 *   num_pairs  >= 0.          n  number of vertices, 0 <= n < 2^31.
 *   flags      TC_INPUT_ON_DEVICE, TC_OFFSETS_32, TC_OFFSETS_64.
 *   alloc      device allocator, or NULL for the library's pool.
 *   stream     cudaStream_t as void*.  The call synchronises it.
 *   out        receives the new graph (owned by the caller until
 *              tc_graph_free); untouched on failure.
 *
 * Errors: TC_EINVAL for NULL src/dst with num_pairs > 0, NULL out, negative
 * sizes, n >= 2^31, or any id outside [0, n); TC_ENOMEM; TC_ECUDA.
 */
TC_API tc_status tc_preprocess(const int32_t* src, const int32_t* dst, int64_t num_pairs,
                        int64_t n, uint32_t flags, const tc_allocator* alloc,
                        void* stream, tc_graph** out);

/*
 * tc_count -- Eq. 1 and Eq. 2 over the graph: the exact number of triangles,
 * and optionally the number of triangles through each vertex.
 *
 *   g            a graph from tc_preprocess.  Its adjacency is not changed,
 *                but the call updates what the graph caches for counting:
 *                the work units (rebuilt when the tuning differs from the
 *                last count's), the 32-bit per-task counters of per-vertex
 *                counts, and the stream its allocations are ordered on.  So
 *                one count at a time per graph; counts of different graphs
 *                may run concurrently.
 *   tune         NULL for defaults.
 *   total_host   if non-NULL, receives the total; the call then synchronises
 *                the stream.
 *   total_dev    if non-NULL, device uint64 that receives the total
 *                (stream ordered, no synchronisation needed).
 *   per_vertex_dev  NULL, or device array of n uint64 that receives, for each
 *                ORIGINAL vertex id v, the triangles containing v
 *                (overwritten; their sum is 3 x total).
 *   stream       cudaStream_t as void*.
 *
 * Errors: TC_EINVAL for NULL g, or both totals NULL and per_vertex_dev NULL;
 * TC_ECUDA.
 */
TC_API tc_status tc_count(tc_graph* g, const tc_tuning* tune, uint64_t* total_host,
                   uint64_t* total_dev, uint64_t* per_vertex_dev, void* stream);

/*
 * tc_preprocess_components -- tc_preprocess of a disjoint union of graphs
 * whose vertex ranges are [vertex_prefix[c], vertex_prefix[c+1]) for
 * components c = 0..num_comps-1.  Any total order of the vertices orients U
 * correctly (Section 3.1 only asks for degree order to save work), so the
 * union is relabelled by degree as one graph; every triangle lies inside one
 * component, and tc_count_components credits each to its component.
 *
 *   vertex_prefix  host array of num_comps + 1 int64, vertex_prefix[0] = 0,
 *                  non-decreasing; n = vertex_prefix[num_comps].
 *   num_comps      >= 1.
 *   Other arguments as tc_preprocess.  Every pair must join two vertices of
 *   one component (checked on the device).
 * Errors: as tc_preprocess, plus TC_EINVAL for a bad prefix or a pair that
 * joins two components.  Synchronises the stream.
 */
TC_API tc_status tc_preprocess_components(const int32_t* src, const int32_t* dst, int64_t num_pairs,
                                          const int64_t* vertex_prefix, int32_t num_comps,
                                          uint32_t flags, const tc_allocator* alloc, void* stream,
                                          tc_graph** out);

/*
 * tc_count_components -- Eq. 1 / Eq. 2 per component of a graph from
 * tc_preprocess_components: comp_totals_dev (device, num_comps uint64)
 * receives each component's triangle count.  Stream ordered.  Updates the
 * graph's counting caches as tc_count does (one count at a time per graph).
 * Errors: TC_EINVAL for NULL arguments or a graph without components.
 */
TC_API tc_status tc_count_components(tc_graph* g, const tc_tuning* tune,
                                     uint64_t* comp_totals_dev, void* stream);

/*
 * tc_triangles -- one call from host pair lists to host results: H2D copy,
 * tc_preprocess, tc_count, D2H copy, release.  Same arguments and errors as
 * the two calls it makes; total_host must be non-NULL, per_vertex_host is
 * NULL or n host uint64.  Synchronises the stream.
 */
TC_API tc_status tc_triangles(const int32_t* src_host, const int32_t* dst_host, int64_t num_pairs,
                       int64_t n, uint32_t flags, void* stream, uint64_t* total_host,
                       uint64_t* per_vertex_host);

/* Where the time of the calling thread's last tc_triangles went.  Device
 * phases come from CUDA events recorded on the call's stream; wall_ms is the
 * host time of the whole call.  Not part of the paper's method.
 *   wall_ms          host time from entry to return
 *   h2d_ms           device time of the upload of both pair arrays
 *   preprocess_ms    device time from the end of the upload to the end of
 *                    tc_preprocess's work (host synchronisations included)
 *   count_ms         device time of the count (and per-vertex gather)
 *   d2h_ms           device time of the copies of the results to the host
 *   h2d_issue_ms     host time spent issuing the upload (as long as the copy
 *                    itself when the pairs are pageable host memory)
 *   input_pinned     1 if both pair arrays are page-locked host memory
 *   upload_method    1: the copy engine; 2: SM loads over the CPU-GPU link
 *                    (page-locked input only).  Uploads of 2^27 pairs or more
 *                    time a 128 MB slice each way and send the rest by the
 *                    faster; smaller ones use SM loads.
 *   ce_slice_gbs, sm_slice_gbs  the rates of those two timed slices (0 when
 *                    no slice was timed)
 * TC_EINVAL on NULL out or when this thread made no successful call. */
typedef struct {
    double wall_ms, h2d_ms, preprocess_ms, count_ms, d2h_ms, h2d_issue_ms;
    int32_t input_pinned;
    int32_t upload_method;
    double ce_slice_gbs, sm_slice_gbs;
} tc_triangles_timing;
TC_API tc_status tc_triangles_get_timing(tc_triangles_timing* out);

/*
 * Graphs larger than the device budget (Section 5.1, Eq. 4 and Eq. 5: the
 * paper's blocks of U and L with their shifts, as tiles streamed through
 * device memory on one GPU).
 *
 * tc_graph_offload -- moves the graph's count arrays (U in CSR, the <j,i,k>
 *   tasks, the relabelling) into page-locked host memory and frees its
 *   device arena.  Afterwards only tc_count_tiled, tc_graph_get_stats and
 *   tc_graph_free accept the graph (tc_count and the batch calls return
 *   TC_EINVAL).  A second call does nothing.  Synchronises the stream.
 *   Errors: TC_EINVAL for NULL g or a graph with components; TC_ENOMEM when
 *   host memory cannot be page-locked (the graph is then unchanged); TC_ECUDA.
 *
 * tc_count_tiled -- Eq. 1 / Eq. 2 on an offloaded graph using at most
 *   device_budget_bytes of device memory, all of it taken from `alloc`
 *   (NULL: the library's pool) on `stream` and given back before return.
 *   Pivots are split into blocks whose rows and tasks fit, rows into blocks
 *   whose entries fit two buffers; each (row block, pivot block) tile is
 *   counted by the ordinary count kernel while the next row block uploads
 *   on a second stream.  The budget must hold 8 B per vertex when per-vertex
 *   counts are asked for, and the largest row (several times over).
 *     total_host       receives the total (required).
 *     per_vertex_host  NULL, or n host uint64 receiving, per ORIGINAL vertex,
 *                      the triangles through it.
 *     stats            NULL, or receives the tiling's figures.
 *   Synchronises the stream.  Errors: TC_EINVAL for NULL g or total_host or
 *   a graph not offloaded; TC_ENOMEM when the budget is too small (message
 *   says why) or an allocation fails; TC_ECUDA.
 */
typedef struct {
    int64_t pivot_blocks;   /* blocks of pivots (a pivot with many tasks may span several) */
    int64_t row_blocks;     /* blocks of rows whose tails the tasks probe */
    int64_t tiles;          /* (row block, pivot block) pairs counted */
    int64_t tile_tasks;     /* tasks counted over all tiles (= the graph's tasks) */
    int64_t h2d_bytes;      /* bytes uploaded */
    uint64_t probes;        /* tail entries probed (= tc_graph_stats.probes) */
    int64_t split_pivots;   /* pivots whose tasks were spread over several pivot blocks */
} tc_tiled_stats;
TC_API tc_status tc_graph_offload(tc_graph* g, void* stream);
TC_API tc_status tc_count_tiled(const tc_graph* g, int64_t device_budget_bytes, const tc_allocator* alloc,
                                const tc_tuning* tune, uint64_t* total_host, uint64_t* per_vertex_host,
                                tc_tiled_stats* stats, void* stream);

/* Work done by the last tc_count on a graph, read from device counters:
 * index 0 is the warp kernel (pivots with |U_j| <= small_max_outdeg), index 1
 * the CTA kernel.  probes = entries of the rows U_i read and looked up. */
typedef struct {
    uint64_t triangles;
    uint64_t units[2];    /* work units processed */
    uint64_t tasks[2];    /* <j,i,k> tasks processed */
    uint64_t probes[2];   /* table lookups (tail entries read) */
    uint64_t staged[2];   /* pivot entries inserted into tables */
} tc_count_stats;

/* Reads the counters of the graph's last tc_count (synchronises the
 * stream).  TC_EINVAL on NULL arguments; TC_ECUDA. */
TC_API tc_status tc_count_get_stats(const tc_graph* g, tc_count_stats* out, void* stream);

/* Fills *out with the graph's facts.  TC_EINVAL on NULL arguments. */
TC_API tc_status tc_graph_get_stats(const tc_graph* g, tc_graph_stats* out);

/* Releases the graph's arena on the stream given at preprocessing.
 * NULL is accepted and ignored. */
TC_API void tc_graph_free(tc_graph* g);

/* Returns to the device the memory that the library's pool of `device`
 * holds but no graph, batch or server uses (device < 0: every device).  The
 * pool keeps freed memory so that repeated calls reuse it rather than map it
 * again; a caller that needs the memory elsewhere calls this after the
 * streams that freed library memory have completed.  Not part of the paper's
 * method.  TC_EINVAL for a device index above the library's limit (64);
 * TC_ECUDA. */
TC_API tc_status tc_release_memory(int device);

/* Device memory of the library's own pool on `device` (not part of the
 * paper's method): bytes reserved from the device, bytes in live
 * allocations, and the high-water marks of both since the pool was created
 * or since the last call with reset_high != 0 (which zeroes them after
 * reading).  Allocations through a caller's tc_allocator are not seen.
 * TC_EINVAL for NULL out or a device outside [0, 64); TC_ECUDA. */
typedef struct {
    int64_t reserved, reserved_high;
    int64_t used, used_high;
} tc_memory_stats;
TC_API tc_status tc_memory_get_stats(int device, int32_t reset_high, tc_memory_stats* out);

/* Self-test of the device's bounded waits (not part of the paper's method).
 * One warp waits, with the wait the radix sort's look-back uses, for a
 * device word that nothing ever publishes, polling at most spin_limit times
 * (1 <= spin_limit <= 2^20, a few ms at most); the wait runs out, the kernel
 * records it and returns, and the call reports it.  Returns TC_ETIMEOUT --
 * the expected result -- and leaves the context usable; TC_EINVAL for a
 * limit out of range; TC_ECUDA.  Synchronises the stream. */
TC_API tc_status tc_selftest_wait_timeout(int64_t spin_limit, void* stream);

/* Defaults for every tc_tuning field.  TC_EINVAL on NULL. */
TC_API tc_status tc_tuning_default(tc_tuning* out);

/* Last error message of the calling host thread ("" if none). */
TC_API const char* tc_last_error(void);

/*
 * tc_generate_rmat -- device copy of the seeded RMAT input generator (not
 * part of the paper's method; it produces synthetic inputs on the device so
 * that large workloads need no host generation or upload).  Writes pairs
 * [e0, e0+count) of the stream of (seed, scale, n) to src_dev / dst_dev
 * (device int32, count entries each).  t1 < t2 < t3 are the cumulative a,
 * a+b, a+b+c probabilities scaled to 2^32.  The stream is, bit for bit, the
 * one of the host generator: splitmix64 draws, one 32-bit half per level,
 * a seeded bijective id scramble on [0, 2^scale), rejection of ids >= n.
 * Errors: TC_EINVAL for scale outside [1,31], n outside [1, 2^scale],
 * negative e0/count, NULL outputs with count > 0; TC_ECUDA.
 */
TC_API tc_status tc_generate_rmat(uint64_t seed, int32_t scale, int64_t n, int64_t e0,
                           int64_t count, uint32_t t1, uint32_t t2, uint32_t t3,
                           int32_t* src_dev, int32_t* dst_dev, void* stream);

/*
 * Batched counting (no counterpart in the paper: many independent graphs
 * counted by one persistent launch).  A batch references its graphs' arenas:
 * they must stay alive, unchanged, until tc_batch_free.  The batch owns a
 * view table, merged work units over all graphs and a captured CUDA graph
 * (two memsets and the count kernel), replayed by tc_batch_count.
 *
 * tc_batch_create: graphs = num graph handles (num >= 1); tune NULL for
 *   defaults; stream unused (the batch works on a private stream and
 *   synchronises it).  *out receives the batch.  TC_EINVAL on NULL or
 *   num <= 0; TC_ENOMEM; TC_ECUDA.
 * tc_batch_count: one graph launch on `stream`; if totals_dev is non-NULL it
 *   receives num device uint64 totals, in the order the graphs were given.
 *   Stream ordered; one count at a time per batch.
 * tc_batch_autotune: times candidate tunings (reps replays each: warp/CTA
 *   bin boundary, tasks per warp and per CTA unit, CTA threads, and the
 *   merge threshold below which short pivot rows are searched rather than
 *   tabled) and keeps the fastest; the choice is cached per degree profile (graph count, mean
 *   edges, largest pivot row, mean tail length) for later batches in the
 *   process.  *chosen (may be NULL) receives it.  Synchronises `stream`.
 * tc_batch_get_count_stats: work counters of the last tc_batch_count;
 *   triangles = sum of the totals.  Synchronises `stream`.
 * tc_count_batch: create, count into totals_dev (required), free.
 */
typedef struct tc_batch tc_batch;
TC_API tc_status tc_batch_create(const tc_graph* const* graphs, int32_t num, const tc_tuning* tune,
                                 void* stream, tc_batch** out);
TC_API tc_status tc_batch_count(tc_batch* b, uint64_t* totals_dev, void* stream);
TC_API tc_status tc_batch_autotune(tc_batch* b, int32_t reps, tc_tuning* chosen, void* stream);
TC_API tc_status tc_batch_get_count_stats(const tc_batch* b, tc_count_stats* out, void* stream);
TC_API void tc_batch_free(tc_batch* b);
TC_API tc_status tc_count_batch(const tc_graph* const* graphs, int32_t num, const tc_tuning* tune,
                                uint64_t* totals_dev, void* stream);

/*
 * Serving (no counterpart in the paper).  A server takes count requests --
 * seeded RMAT specs, expanded on the device -- in arrival order and runs
 * them in ticks: worker threads (one CUDA stream each) take requests from
 * the head of the queue while the tick stays within max_batch requests and
 * max_tick_pairs pairs and the device bytes of all ticks in flight stay
 * within hbm_budget_bytes (each request's footprint is estimated as
 * 64 B per pair + 48 B per vertex); a tick's requests are preprocessed as one
 * disjoint union and counted per component (tc_preprocess_components /
 * tc_count_components).  Ticks on different workers overlap on the device.
 * Results carry the caller-given arrival time and the server-clock times of
 * admission and completion (tc_server_now: seconds since creation).
 *
 * tc_server_create: cfg may be NULL (all defaults); zero or negative size
 *   fields take defaults (16 GiB budget, 2 workers, 512 requests and 2^27
 *   pairs per tick); device -1 (or NULL cfg) uses the current device.
 * tc_server_submit_rmat: queue one request; *ticket (may be NULL) gets its
 *   id.  TC_EINVAL for a bad spec; TC_EBUSY if the request alone exceeds the
 *   budget (it is dropped).
 * tc_server_submit_rmat_many: queue count requests at once, in order, under
 *   one lock (a worker that wakes sees all of them); t_arrival[k] and
 *   tickets[k] (tickets may be NULL) as above.  All or nothing: if any spec
 *   is bad (TC_EINVAL) or over the budget (TC_EBUSY), none is queued.
 * tc_server_poll: move up to max finished results to out (waiting up to
 *   wait_ms for the first); *count gets how many.
 * tc_server_drain: wait until every submitted request is done; TC_ETIMEOUT
 *   after timeout_ms (the requests stay queued), else the first error any
 *   tick met (TC_OK if none).
 * tc_server_free: finishes the ticks in flight and the queued requests that
 *   fit, stops the workers, frees the server.
 */
typedef struct tc_server tc_server;
typedef struct {
    int64_t hbm_budget_bytes;
    int32_t workers;
    int32_t max_batch;
    int64_t max_tick_pairs;
    int32_t device;        /* CUDA device; -1 for the calling thread's current one */
    int32_t pad;
} tc_server_config;
typedef struct {
    uint64_t seed;
    int32_t scale;         /* ids drawn on [0, 2^scale), those >= n redrawn */
    int32_t pad;
    int64_t n;             /* vertices, 1 <= n <= 2^scale */
    int64_t num_pairs;     /* generated pairs */
    uint32_t t1, t2, t3;   /* cumulative a, a+b, a+b+c scaled to 2^32 */
    uint32_t pad2;
} tc_rmat_spec;
typedef struct {
    int64_t ticket;
    uint64_t triangles;
    double t_arrival, t_admit, t_done;
    int32_t status;        /* TC_OK, or the error of the request's tick */
    int32_t tick_requests; /* requests counted in the same tick */
    int64_t tick_pairs;    /* pairs of all requests of that tick */
    double t_dev_start, t_dev_end;   /* device time span of the tick (seconds
                                        from server creation; -1 if unknown) */
} tc_server_result;
typedef struct {
    int64_t submitted, completed, failed, pending, ticks;
    int64_t bytes_in_flight, peak_bytes_in_flight, busy_workers;
    double device_busy_s;     /* device time covered by at least one tick's span */
    double device_overlap_s;  /* device time covered by two or more ticks' spans */
} tc_server_stats;

TC_API tc_status tc_server_create(const tc_server_config* cfg, tc_server** out);
TC_API double tc_server_now(const tc_server* s);
TC_API tc_status tc_server_submit_rmat(tc_server* s, const tc_rmat_spec* spec, double t_arrival,
                                       int64_t* ticket);
TC_API tc_status tc_server_submit_rmat_many(tc_server* s, const tc_rmat_spec* specs, int32_t count,
                                            const double* t_arrival, int64_t* tickets);
TC_API tc_status tc_server_poll(tc_server* s, tc_server_result* out, int32_t max, int32_t* count,
                                int32_t wait_ms);
TC_API tc_status tc_server_drain(tc_server* s, int32_t timeout_ms);
TC_API tc_status tc_server_get_stats(tc_server* s, tc_server_stats* out);
TC_API void tc_server_free(tc_server* s);

/*
 * tc_triangles_static -- tc_preprocess + tc_count for a small graph with no
 * device allocation.  (The paper has no counterpart: this serves callers
 * that cannot call cudaMalloc when they need a count, e.g. code running
 * after start-up has given all device memory to another allocator, such as
 * a framework's caching pool or a serving runtime with a fixed budget, or
 * latency-critical loops that must not allocate at steady state.)
 *
 * Every buffer comes from one file-scope device array of 32 MiB that each
 * GPU loading the library holds until the process exits.  The first call on
 * a device looks up that array's address (cudaGetSymbolAddress, with the
 * device current); make that first call before any stream capture.  Each
 * call reuses the whole array; calls whose GPU work overlaps race on it, so
 * issue them on one stream or synchronise between them.
 *
 *   src_dev, dst_dev  num_pairs device int32 ids in [0, n) (read only).
 *   num_pairs  0 .. TC_STATIC_MAX_PAIRS.   n  0 .. TC_STATIC_MAX_VERTICES.
 *   total_dev  device uint64 receiving the total (required).
 *   per_vertex_dev  NULL or n device uint64 (original ids), as tc_count.
 *   stream     cudaStream_t as void*; the call synchronises it while
 *              preprocessing; the count itself is stream ordered.
 *
 * Errors: TC_EINVAL for sizes beyond the limits (with a message naming
 * them), negative sizes, NULL required pointers or ids outside [0, n);
 * TC_ECUDA.  Allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine is called.
 */
#define TC_STATIC_MAX_PAIRS 262144
#define TC_STATIC_MAX_VERTICES 65536
TC_API tc_status tc_triangles_static(const int32_t* src_dev, const int32_t* dst_dev,
                                     int64_t num_pairs, int64_t n, uint64_t* total_dev,
                                     uint64_t* per_vertex_dev, void* stream);

/*
 * Kernel accounting (not part of the paper's method; measurement support).
 *
 * tc_kernel_launches: number of kernels this library has launched since it
 * was loaded (all threads).
 * tc_profile_enable: on != 0 clears the records and starts bracketing every
 * launch with CUDA events recorded on the launching stream; 0 stops.
 * tc_profile_read: waits for the recorded events and writes, per kernel
 * name, the launches and summed device time since profiling was enabled.
 * Fills at most max entries; *count receives the number of names.
 * TC_EINVAL on NULL count (or NULL out with max > 0); TC_ECUDA.
 */
typedef struct {
    char name[40];
    int64_t launches;
    double total_ms;
} tc_kernel_time;

TC_API long long tc_kernel_launches(void);
TC_API void tc_profile_enable(int32_t on);
TC_API tc_status tc_profile_read(tc_kernel_time* out, int32_t max, int32_t* count);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
