// tc_count: Eq. 1 / Eq. 2 by the paper's <j,i,k> map-based enumeration.
//
// For a pivot j the row U_j (the labels k > j adjacent to j) is put in a
// shared-memory table once; every task (i,j) of j -- an edge of U whose row
// U_i continues after j -- then probes the table with each entry of U_i
// after j.  Each hit k is one triangle {i, j, k} counted at edge (i, j)
// (Eq. 1 sums exactly the k > j with u_ik = u_jk = 1).
//
// Tables (Section 5.2, "Modifying the hashing routine for sparser vertices"):
// when the label span of U_j fits the table, slot = k - min(U_j) (direct, no
// probing); otherwise slot = k AND (size-1) with linear probing, size >= 2|U_j|.
// Probes outside [min U_j, max U_j] are rejected before the lookup, the
// per-probe form of the early exit of Section 5.2.
//
// Work: units (pivot, slice of U_j, range of tasks) in two lists.  Pivots
// with |U_j| <= 64 are handled by one warp each (a 128-slot table per warp);
// larger pivots by one CTA with a table of up to 2 x 8192 slots, split into
// slices beyond that.  Persistent CTAs pop units from atomic queue heads.
// Inside a unit, a warp takes 32 tasks at a time and walks the concatenation
// of their tails 32 probes per step (the owning task of each probe is found
// by a 5-step shuffle binary search over the warp's prefix sums), so loads of
// a tail are contiguous across lanes whatever the tail lengths.
//
// Per-vertex counts (t[v] = triangles through v): each hit credits k through
// a shared counter per table slot, i through a per-task shared counter, and j
// once per unit; all flushed with one global atomic per nonzero counter.
#include <algorithm>

#include "common.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int kSmallWarps = 8;
constexpr int kSmallThreads = kSmallWarps * 32;
constexpr int kGrab = 4;   // warp units popped per queue access
constexpr int kEmpty = -1;

__device__ __forceinline__ int64_t shfl64(int64_t v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
}

__device__ __forceinline__ int warp_incl_scan_i32(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ __forceinline__ void table_insert(int* tab, unsigned mask, bool direct, int lo, int k) {
    if (direct) {
        tab[k - lo] = k;
        return;
    }
    unsigned s = (unsigned)k & mask;
    while (true) {
        int old = atomicCAS(&tab[s], kEmpty, k);
        if (old == kEmpty) return;
        s = (s + 1) & mask;
    }
}

// slot holding k, or -1
__device__ __forceinline__ int table_find(const int* tab, unsigned mask, bool direct, int lo,
                                          int hi, int k) {
    if (k < lo || k > hi) return -1;
    if (direct) return (tab[k - lo] == k) ? (k - lo) : -1;
    unsigned s = (unsigned)k & mask;
    while (true) {
        int v = tab[s];
        if (v == k) return (int)s;
        if (v == kEmpty) return -1;
        s = (s + 1) & mask;
    }
}

// One warp walks tasks [t0, t1) against the table.  Returns this lane's hits.
// With PV, per-task hits go to tnew[i] and per-slot hits to slot_hits.
template <bool PV>
__device__ __forceinline__ uint64_t warp_probe_tasks(const Task* __restrict__ tasks, int64_t t0,
                                                     int64_t t1, int64_t tstride,
                                                     const int32_t* __restrict__ adj,
                                                     const int* tab, unsigned mask, bool direct,
                                                     int lo, int hi, unsigned* slot_hits,
                                                     unsigned* task_hits,
                                                     unsigned long long* tnew) {
    const int lane = threadIdx.x & 31;
    uint64_t hits = 0;
    for (int64_t tb = t0; tb < t1; tb += tstride) {
        const int64_t t = tb + lane;
        const bool valid = t < t1;
        int64_t start = 0;
        int len = 0, i = 0;
        if (valid) {
            const Task T = tasks[t];
            start = T.start;
            len = T.len;
            i = T.i;
        }
        const int incl = warp_incl_scan_i32(len);
        const int excl = incl - len;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (PV) {
            task_hits[lane] = 0;
            __syncwarp();
        }
        for (int q0 = 0; q0 < total; q0 += 32) {
            const int q = q0 + lane;
            // largest lane o with excl_o <= q (zero-length tasks are skipped
            // because the next task shares their prefix)
            int o = 0;
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                int c = o + step;
                if (__shfl_sync(0xffffffffu, excl, c) <= q) o = c;
            }
            const int ex_o = __shfl_sync(0xffffffffu, excl, o);
            const int64_t st_o = shfl64(start, o);
            if (q < total) {
                const int k = __ldg(&adj[st_o + (q - ex_o)]);
                const int s = table_find(tab, mask, direct, lo, hi, k);
                if (s >= 0) {
                    ++hits;
                    if (PV) {
                        atomicAdd(&slot_hits[s], 1u);
                        atomicAdd(&task_hits[o], 1u);
                    }
                }
            }
        }
        if (PV) {
            __syncwarp();
            const unsigned h = task_hits[lane];
            if (valid && h) atomicAdd(&tnew[i], (unsigned long long)h);
            __syncwarp();
        }
    }
    return hits;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class OffT, bool PV>
__global__ void __launch_bounds__(kSmallThreads)
    k_count_small(const Unit* __restrict__ units, int64_t nunits, const Task* __restrict__ tasks,
                  const OffT* __restrict__ off, const int32_t* __restrict__ adj,
                  unsigned long long* __restrict__ ctr, unsigned long long* __restrict__ tnew) {
    __shared__ int tab_s[kSmallWarps][kSmallTable];
    __shared__ unsigned slot_s[kSmallWarps][PV ? kSmallTable : 1];
    __shared__ unsigned task_s[kSmallWarps][PV ? 32 : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* tab = tab_s[w];
    unsigned* slot_hits = slot_s[w];
    unsigned* task_hits = task_s[w];
    uint64_t hits = 0;
    while (true) {
        long long u0 = 0;
        if (lane == 0) u0 = (long long)atomicAdd(&ctr[CTR_SMALL_HEAD], (unsigned long long)kGrab);
        u0 = __shfl_sync(0xffffffffu, u0, 0);
        if (u0 >= nunits) break;
        const int64_t u1 = min64(u0 + kGrab, nunits);
        for (int64_t u = u0; u < u1; ++u) {
            const Unit U = units[u];
            const int64_t rb = (int64_t)off[U.j], re = (int64_t)off[U.j + 1];
            const int dp = (int)(re - rb);
            const int lo = adj[rb], hi = adj[re - 1];
            const bool direct = (int64_t)hi - lo < kSmallTable;
            const unsigned mask = kSmallTable - 1;
#pragma unroll
            for (int s = lane; s < kSmallTable; s += 32) {
                tab[s] = kEmpty;
                if (PV) slot_hits[s] = 0;
            }
            __syncwarp();
            for (int q = lane; q < dp; q += 32) table_insert(tab, mask, direct, lo, adj[rb + q]);
            __syncwarp();
            uint64_t uh = warp_probe_tasks<PV>(tasks, U.t0, U.t1, 32, adj, tab, mask, direct, lo, hi,
                                               slot_hits, task_hits, tnew);
            hits += uh;
            if (PV) {
                __syncwarp();
#pragma unroll
                for (int s = lane; s < kSmallTable; s += 32) {
                    const unsigned c = slot_hits[s];
                    if (c) atomicAdd(&tnew[tab[s]], (unsigned long long)c);
                }
                uh = warp_sum_u64(uh);
                if (lane == 0 && uh) atomicAdd(&tnew[U.j], (unsigned long long)uh);
            }
            __syncwarp();
        }
    }
    hits = warp_sum_u64(hits);
    if (lane == 0 && hits) atomicAdd(&ctr[CTR_TOTAL], (unsigned long long)hits);
}

template <class OffT, bool PV>
__global__ void k_count_large(const Unit* __restrict__ units, int64_t nunits,
                              const Task* __restrict__ tasks, const OffT* __restrict__ off,
                              const int32_t* __restrict__ adj, int slice_max,
                              unsigned long long* __restrict__ ctr,
                              unsigned long long* __restrict__ tnew) {
    extern __shared__ int smem[];
    __shared__ long long s_unit;
    __shared__ unsigned task_s[32][PV ? 32 : 1];
    __shared__ unsigned long long s_red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int* tab = smem;
    uint64_t hits = 0;
    while (true) {
        if (threadIdx.x == 0) s_unit = (long long)atomicAdd(&ctr[CTR_LARGE_HEAD], 1ull);
        __syncthreads();
        const long long u = s_unit;
        if (u >= nunits) break;
        const Unit U = units[u];
        const int64_t row_b = (int64_t)off[U.j], row_e = (int64_t)off[U.j + 1];
        const int64_t rb = row_b + (int64_t)U.slice * slice_max;
        const int64_t re = min64(row_e, rb + slice_max);
        const int dp = (int)(re - rb);
        int size = 256;
        while (size < 2 * dp) size <<= 1;
        const unsigned mask = (unsigned)size - 1u;
        const int lo = adj[rb], hi = adj[re - 1];
        const bool direct = (int64_t)hi - lo < size;
        unsigned* slot_hits = reinterpret_cast<unsigned*>(smem + size);
        for (int s = threadIdx.x; s < size; s += blockDim.x) {
            tab[s] = kEmpty;
            if (PV) slot_hits[s] = 0;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < dp; q += blockDim.x) table_insert(tab, mask, direct, lo, adj[rb + q]);
        __syncthreads();
        uint64_t uh = warp_probe_tasks<PV>(tasks, U.t0 + (int64_t)w * 32, U.t1, (int64_t)nw * 32, adj,
                                           tab, mask, direct, lo, hi, slot_hits, task_s[w], tnew);
        hits += uh;
        __syncthreads();
        if (PV) {
            for (int s = threadIdx.x; s < size; s += blockDim.x) {
                const unsigned c = slot_hits[s];
                if (c) atomicAdd(&tnew[tab[s]], (unsigned long long)c);
            }
            uh = warp_sum_u64(uh);
            if (lane == 0) s_red[w] = uh;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned long long tot = 0;
                for (int q = 0; q < nw; ++q) tot += s_red[q];
                if (tot) atomicAdd(&tnew[U.j], tot);
            }
            __syncthreads();
        }
    }
    hits = warp_sum_u64(hits);
    if (lane == 0 && hits) atomicAdd(&ctr[CTR_TOTAL], (unsigned long long)hits);
}

__global__ void k_gather_pv(const unsigned long long* __restrict__ tnew,
                            const int32_t* __restrict__ perm, int64_t n,
                            uint64_t* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        out[v] = tnew[perm[v]];
}

__global__ void k_copy_total(const unsigned long long* __restrict__ ctr, uint64_t* __restrict__ out) {
    *out = ctr[CTR_TOTAL];
}

// ---------------------------------------------------------------------------
// work units
// ---------------------------------------------------------------------------
template <class OffT>
__global__ void k_unit_counts(const OffT* __restrict__ off, const int64_t* __restrict__ loff,
                              int64_t n, int small_max, int tw, int tcta, int slice,
                              int32_t* __restrict__ cs, int32_t* __restrict__ cl) {
    for (int64_t jj = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; jj < n;
         jj += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = n - 1 - jj;   // heavy pivots (high labels) first
        const int64_t dp = (int64_t)off[j + 1] - (int64_t)off[j];
        const int64_t nt = loff[j + 1] - loff[j];
        int32_t a = 0, b = 0;
        if (dp > 0 && nt > 0) {
            if (dp <= small_max) {
                a = (int32_t)((nt + tw - 1) / tw);
            } else {
                const int64_t slices = (dp + slice - 1) / slice;
                b = (int32_t)(slices * ((nt + tcta - 1) / tcta));
            }
        }
        cs[jj] = a;
        cl[jj] = b;
    }
}

template <class OffT>
__global__ void k_unit_fill(const OffT* __restrict__ off, const int64_t* __restrict__ loff,
                            int64_t n, int small_max, int tw, int tcta, int slice,
                            const int64_t* __restrict__ ps, const int64_t* __restrict__ pl,
                            Unit* __restrict__ us, Unit* __restrict__ ul) {
    for (int64_t jj = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; jj < n;
         jj += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = n - 1 - jj;
        const int64_t dp = (int64_t)off[j + 1] - (int64_t)off[j];
        const int64_t a = loff[j], b = loff[j + 1];
        if (dp <= 0 || b <= a) continue;
        if (dp <= small_max) {
            int64_t p = ps[jj];
            for (int64_t t = a; t < b; t += tw) us[p++] = Unit{(int32_t)j, 0, t, min64(t + tw, b)};
        } else {
            const int64_t slices = (dp + slice - 1) / slice;
            int64_t p = pl[jj];
            for (int64_t t = a; t < b; t += tcta)
                for (int64_t s = 0; s < slices; ++s)
                    ul[p++] = Unit{(int32_t)j, (int32_t)s, t, min64(t + tcta, b)};
        }
    }
}

template <class OffT>
void build_units_t(tc_graph* g, const tc_tuning& t, cudaStream_t st) {
    Alloc& al = g->alloc;
    const int64_t n = g->n;
    const OffT* off = static_cast<const OffT*>(g->off);
    const unsigned G = (unsigned)(num_sms() * 8);
    Buf<int32_t> cs(al, (size_t)std::max<int64_t>(n, 1)), cl(al, (size_t)std::max<int64_t>(n, 1));
    Buf<int64_t> ps(al, (size_t)(n + 1)), pl(al, (size_t)(n + 1));
    if (n > 0) {
        {
            Prof prof_("k_unit_counts", st);
            k_unit_counts<OffT><<<grid_for(n, 256, G), 256, 0, st>>>(
            off, g->loff, n, t.small_max_outdeg, t.warp_unit_tasks, t.cta_unit_tasks, t.slice_max,
            cs.get(), cl.get());
        }
        TC_LAUNCH_CHECK();
    }
    exclusive_scan_i32_to_i64(cs.get(), ps.get(), n, ps.get() + n, al, st);
    exclusive_scan_i32_to_i64(cl.get(), pl.get(), n, pl.get() + n, al, st);
    int64_t ns = 0, nl = 0;
    TC_CUDA(cudaMemcpyAsync(&ns, ps.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&nl, pl.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (g->units_mem) {
        al.put(g->units_mem, g->units_bytes);
        g->units_mem = nullptr;
    }
    g->units_bytes = sizeof(Unit) * (size_t)std::max<int64_t>(ns + nl, 1);
    g->units_mem = al.get(g->units_bytes);
    g->small_units = static_cast<Unit*>(g->units_mem);
    g->large_units = g->small_units + ns;
    if (n > 0) {
        {
            Prof prof_("k_unit_fill", st);
            k_unit_fill<OffT><<<grid_for(n, 256, G), 256, 0, st>>>(
            off, g->loff, n, t.small_max_outdeg, t.warp_unit_tasks, t.cta_unit_tasks, t.slice_max,
            ps.get(), pl.get(), g->small_units, g->large_units);
        }
        TC_LAUNCH_CHECK();
    }
    g->n_small = ns;
    g->n_large = nl;
    int size = 256;
    const int64_t need = min64(g->stats.max_outdeg, t.slice_max);
    while (size < 2 * need) size <<= 1;
    g->large_table = size;
    g->units_tuning = t;
    g->stats.small_units = ns;
    g->stats.large_units = nl;
}

template <class OffT, bool PV>
void count_t(const tc_graph* g, const tc_tuning& t, cudaStream_t st) {
    const OffT* off = static_cast<const OffT*>(g->off);
    unsigned long long* tnew = reinterpret_cast<unsigned long long*>(g->tnew);
    const int sms = num_sms();
    if (g->n_small > 0) {
        int per_sm = 0;
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_small<OffT, PV>,
                                                              kSmallThreads, 0));
        per_sm = std::max(per_sm, 1);
        int64_t need = (g->n_small + kGrab * kSmallWarps - 1) / (kGrab * kSmallWarps);
        unsigned grid = (unsigned)std::max<int64_t>(1, min64((int64_t)sms * per_sm, need));
        {
            Prof prof_("k_count_small", st);
            k_count_small<OffT, PV><<<grid, kSmallThreads, 0, st>>>(g->small_units, g->n_small, g->tasks,
                                                               off, g->adj, g->counters, tnew);
        }
        TC_LAUNCH_CHECK();
    }
    if (g->n_large > 0) {
        const int threads = t.cta_threads;
        const size_t smem = sizeof(int) * (size_t)g->large_table * (PV ? 2 : 1);
        auto kern = k_count_large<OffT, PV>;
        TC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        per_sm = std::max(per_sm, 1);
        unsigned grid = (unsigned)std::max<int64_t>(1, min64((int64_t)sms * per_sm, g->n_large));
        {
            Prof prof_("k_count_large", st);
            kern<<<grid, threads, smem, st>>>(g->large_units, g->n_large, g->tasks, off, g->adj,
                                          t.slice_max, g->counters, tnew);
        }
        TC_LAUNCH_CHECK();
    }
}

}  // namespace

void build_units(tc_graph* g, const tc_tuning& t, cudaStream_t st) {
    if (g->off64)
        build_units_t<int64_t>(g, t, st);
    else
        build_units_t<int32_t>(g, t, st);
}

void count(const tc_graph* gc, const tc_tuning& t, uint64_t* total_dev, uint64_t* per_vertex_dev,
           cudaStream_t st) {
    tc_graph* g = const_cast<tc_graph*>(gc);   // unit lists are a cache of the tuning
    if (!tuning_equal(t, g->units_tuning)) build_units(g, t, st);
    const bool pv = per_vertex_dev != nullptr;
    TC_CUDA(cudaMemsetAsync(g->counters, 0, sizeof(unsigned long long) * CTR_COUNT, st));
    if (pv && g->n > 0) TC_CUDA(cudaMemsetAsync(g->tnew, 0, sizeof(uint64_t) * (size_t)g->n, st));
    if (g->off64) {
        if (pv) count_t<int64_t, true>(g, t, st); else count_t<int64_t, false>(g, t, st);
    } else {
        if (pv) count_t<int32_t, true>(g, t, st); else count_t<int32_t, false>(g, t, st);
    }
    if (pv && g->n > 0) {
        {
            Prof prof_("k_gather_pv", st);
            k_gather_pv<<<grid_for(g->n, 256, num_sms() * 8), 256, 0, st>>>(
            reinterpret_cast<const unsigned long long*>(g->tnew), g->perm, g->n, per_vertex_dev);
        }
        TC_LAUNCH_CHECK();
    }
    if (total_dev) {
        {
            Prof prof_("k_copy_total", st);
            k_copy_total<<<1, 1, 0, st>>>(g->counters, total_dev);
        }
        TC_LAUNCH_CHECK();
    }
}

}  // namespace tc
