// tc_preprocess: Section 5.3 of the paper on one device.
//
//   a1 canonicalise   pairs -> key (min << b | max); self-loops dropped
//   a2 unique         up to 2^26 pairs: keys inserted into a device hash set
//                     (open addressing, load <= 1/2) whose compacted slots
//                     are E, in no particular order (a5 sorts them).  Larger
//                     inputs: LSD radix sort, first of each run kept -- the
//                     set's random atomics into a table of 2^31 slots ran
//                     slower than the sort's passes (measured at 2^30 pairs).
//   a3 degrees        d(v) counted when a key enters the set / from the
//                     unique runs
//   a4 relabel        rank by (d(v), v): the counting sort of Section 5.3 as
//                     one stable pass on the degree clipped at 255 (nearly
//                     every vertex), the vertices at or above it then sorted
//                     on their full degree; the rank is the new label
//   a5 orient + CSR   (min, max) of the new labels, sorted -> U rows ascending
//   a6 tasks + units  <j,i,k> tasks grouped by pivot j, then work units
//
// b = ceil(log2 n) bits per id, so keys use 2b <= 62 bits.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "common.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int kT = 256;

#ifndef TC_DEGREE_COUNTING
#define TC_DEGREE_COUNTING 1   // a4: 1 counting pass + heavy tail (Section 5.3); 0 radix on the degree bits
#endif
// below this many vertices the radix form takes fewer launches (the heavy
// tail's own sort costs more than the passes it saves)
constexpr int64_t kCountingMinVertices = 1ll << 20;
constexpr int kHeavy = 255;    // degrees clipped here by the counting pass

constexpr uint64_t kEmptyKey = ~0ull;   // no key: keys use 2b <= 62 bits
constexpr int64_t kHashDedupMaxPairs = 1ll << 26;   // table of at most 2^27 slots (1 GB)

// a bijective 64-bit mixer (the finaliser of splitmix64, Steele, Lea and
// Flood 2014) spreading the keys over the table
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

// a1 + a2 + a3: pair -> canonical key -> hash set; the pair that inserts a
// key counts it in the degrees of both ends.  Ids outside [0, n) set error
// bit 1 and are skipped.  The table (capacity cmask + 1 >= 2 * pairs) never
// fills, so a probe sequence always ends; it is bounded all the same.
__global__ void k_dedup_insert(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                               int64_t P, int64_t n, int bits, unsigned long long* __restrict__ table,
                               uint64_t cmask, int32_t* __restrict__ deg, int* __restrict__ err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || b < 0 || (int64_t)a >= n || (int64_t)b >= n) {
            atomicOr(err, 1);
            continue;
        }
        if (a == b) continue;
        const int32_t lo = min(a, b), hi = max(a, b);
        const unsigned long long key = ((unsigned long long)lo << bits) | (unsigned long long)hi;
        uint64_t h = mix64(key) & cmask;
        for (uint64_t probe = 0; probe <= cmask; ++probe) {
            const unsigned long long prev = atomicCAS(&table[h], kEmptyKey, key);
            if (prev == kEmptyKey) {
                atomicAdd(&deg[lo], 1);
                atomicAdd(&deg[hi], 1);
                break;
            }
            if (prev == key) break;
            h = (h + 1) & cmask;
        }
    }
}

// The occupied slots of the table -> E.  Each CTA takes chunks of
// kCompactItems * blockDim slots, ranks its keys with a block scan and
// reserves their places in E with one atomic on the count.
constexpr int kCompactItems = 16;

__global__ void __launch_bounds__(256) k_table_compact(const unsigned long long* __restrict__ table,
                                                       int64_t cap, uint64_t* __restrict__ E,
                                                       unsigned long long* __restrict__ count) {
    __shared__ unsigned wsum[8];
    __shared__ unsigned long long s_base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t chunk = (int64_t)kCompactItems * blockDim.x;
    for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < cap; c0 += (int64_t)gridDim.x * chunk) {
        unsigned long long k[kCompactItems];
        unsigned mine = 0;
#pragma unroll
        for (int u = 0; u < kCompactItems; ++u) {
            const int64_t s = c0 + (int64_t)u * blockDim.x + threadIdx.x;
            k[u] = s < cap ? table[s] : kEmptyKey;
            mine += k[u] != kEmptyKey;
        }
        unsigned inc = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        unsigned before = 0, total = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            if (q < w) before += wsum[q];
            total += wsum[q];
        }
        if (threadIdx.x == 0) s_base = total ? atomicAdd(count, (unsigned long long)total) : 0ull;
        __syncthreads();
        unsigned long long at = s_base + before + inc - mine;
#pragma unroll
        for (int u = 0; u < kCompactItems; ++u)
            if (k[u] != kEmptyKey) E[at++] = k[u];
        __syncthreads();   // wsum and s_base are rewritten by the next chunk
    }
}

// counter[v] += 1 for the active lanes, whose v are non-decreasing across the
// warp: one atomic per run of equal v among neighbouring active lanes (an
// inactive lane splits a run; both parts are added).  All 32 lanes call it.
__device__ __forceinline__ void warp_add_sorted(int32_t* counter, int32_t v, bool active) {
    const int lane = threadIdx.x & 31;
    const int32_t pv = __shfl_up_sync(0xffffffffu, v, 1);
    const bool pa = __shfl_up_sync(0xffffffffu, active, 1);
    const bool cont = active && lane > 0 && pa && pv == v;
    const unsigned C = __ballot_sync(0xffffffffu, cont);   // lanes continuing a run
    if (active && !cont) {
        // run length: 1 + the continuation lanes right after this one
        const unsigned rest = lane == 31 ? 0u : (C >> (lane + 1));
        atomicAdd(&counter[v], 1 + __ffs(~rest) - 1);
    }
}

__global__ void k_canon(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                        int64_t P, int64_t n, int bits, uint64_t sentinel,
                        uint64_t* __restrict__ keys, int* __restrict__ err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[e], b = dst[e];
        uint64_t k = sentinel;
        if (a < 0 || b < 0 || (int64_t)a >= n || (int64_t)b >= n) {
            atomicOr(err, 1);
        } else if (a != b) {
            uint64_t lo = (uint64_t)min(a, b), hi = (uint64_t)max(a, b);
            k = (lo << bits) | hi;
        }
        keys[e] = k;
    }
}

__global__ void k_unique_flags(const uint64_t* __restrict__ keys, int64_t P, uint64_t sentinel,
                               int32_t* __restrict__ flags) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[e];
        flags[e] = (k != sentinel && (e == 0 || keys[e - 1] != k)) ? 1 : 0;
    }
}

// Adds c to counter[v] once per group of lanes holding the same v.
__global__ void k_unique_compact(const uint64_t* __restrict__ keys, const int32_t* __restrict__ flags,
                                 const int64_t* __restrict__ pos, int64_t P, int bits,
                                 uint64_t* __restrict__ E, int32_t* __restrict__ deg) {
    const uint64_t mask = (1ull << bits) - 1ull;
    // grid-stride with whole-warp iterations so the warp intrinsics see full warps
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < P; base += stride) {
        int64_t e = base + threadIdx.x;
        bool keep = e < P && flags[e];
        uint64_t k = keep ? keys[e] : 0;
        if (keep) E[pos[e]] = k;
        warp_add_sorted(deg, (int32_t)(k >> bits), keep);   // keys sorted: min ids in runs
        if (keep) atomicAdd(&deg[(int32_t)(k & mask)], 1);
    }
}

// out[0] = max of x; out[2] += the entries >= kHeavy
__global__ void k_max_i32(const int32_t* __restrict__ x, int64_t n, int* __restrict__ out) {
    int mx = 0, heavy = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        mx = max(mx, x[v]);
        heavy += x[v] >= kHeavy;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        heavy += __shfl_xor_sync(0xffffffffu, heavy, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, mx);
        if (heavy) atomicAdd(out + 2, heavy);
    }
}

// the counting pass's keys: degree clipped to kHeavy, then the id
__global__ void k_degree_keys_clipped(const int32_t* __restrict__ deg, int64_t n, int bits,
                                      uint64_t* __restrict__ keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = ((uint64_t)(uint32_t)min(deg[v], kHeavy) << bits) | (uint64_t)v;
}

// the heavy tail (the last h keys of the counting pass, ids in order) with
// their full degrees
__global__ void k_heavy_keys(const uint64_t* __restrict__ sorted, int64_t n, int64_t h, int bits,
                             const int32_t* __restrict__ deg, uint64_t* __restrict__ out) {
    const uint64_t mask = (1ull << bits) - 1ull;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < h;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = sorted[n - h + q] & mask;
        out[q] = ((uint64_t)(uint32_t)deg[v] << bits) | v;
    }
}

__global__ void k_degree_keys(const int32_t* __restrict__ deg, int64_t n, int bits,
                              uint64_t* __restrict__ keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = ((uint64_t)(uint32_t)deg[v] << bits) | (uint64_t)v;
}

// perm[old id] = rank; degn[rank] = degree (the key's high bits)
__global__ void k_perm(const uint64_t* __restrict__ sorted, int64_t n, int bits,
                       int32_t* __restrict__ perm, int32_t* __restrict__ degn) {
    const uint64_t mask = (1ull << bits) - 1ull;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = sorted[r];
        perm[k & mask] = (int32_t)r;
        degn[r] = (int32_t)(k >> bits);
    }
}

// the same for sorted keys whose ranks start at r0
__global__ void k_perm_at(const uint64_t* __restrict__ sorted, int64_t count, int64_t r0, int bits,
                          int32_t* __restrict__ perm, int32_t* __restrict__ degn) {
    const uint64_t mask = (1ull << bits) - 1ull;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = sorted[q];
        perm[k & mask] = (int32_t)(r0 + q);
        degn[r0 + q] = (int32_t)(k >> bits);
    }
}

__global__ void k_orient(const uint64_t* __restrict__ E, int64_t m, int bits,
                         const int32_t* __restrict__ perm, uint64_t* __restrict__ keys) {
    const uint64_t mask = (1ull << bits) - 1ull;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = E[e];
        uint32_t u = (uint32_t)perm[k >> bits], v = (uint32_t)perm[k & mask];
        uint64_t lo = min(u, v), hi = max(u, v);
        keys[e] = (lo << bits) | hi;
    }
}

// adj[e] = column; dplus[row] += 1 (rows are sorted, so lanes agree a lot)
__global__ void k_adj_rows(const uint64_t* __restrict__ keys, int64_t m, int bits,
                           int32_t* __restrict__ adj, int32_t* __restrict__ dplus) {
    const uint64_t mask = (1ull << bits) - 1ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < m; base += stride) {
        int64_t e = base + threadIdx.x;
        bool ok = e < m;
        uint64_t k = ok ? keys[e] : 0;
        if (ok) adj[e] = (int32_t)(k & mask);
        warp_add_sorted(dplus, (int32_t)(k >> bits), ok);
    }
}

// a5 by counting, for graphs small enough that no row of U can pass
// kRowSortMax entries (in degree order a row of d entries has d neighbours
// of degree >= d, so d^2 <= 2m): the oriented pairs are counted per row,
// scattered into their row's slots, and each row is sorted where it lies.
#ifndef TC_ORIENT_COUNT_MAX
#define TC_ORIENT_COUNT_MAX (1ll << 24)
#endif
constexpr int64_t kOrientCountMaxM = TC_ORIENT_COUNT_MAX;
constexpr int kRowSortMax = 8192;   // sqrt(2 * 2^25)
static_assert(kOrientCountMaxM <= (int64_t)kRowSortMax * kRowSortMax / 2, "rows fit the row sort");
constexpr int kRowSortThreads = 256;

__global__ void k_orient_count(const uint64_t* __restrict__ E, int64_t m, int bits,
                               const int32_t* __restrict__ perm, uint64_t* __restrict__ keys,
                               int32_t* __restrict__ dplus) {
    const uint64_t mask = (1ull << bits) - 1ull;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = E[e];
        const uint32_t u = (uint32_t)perm[k >> bits], v = (uint32_t)perm[k & mask];
        const uint64_t lo = min(u, v), hi = max(u, v);
        keys[e] = (lo << bits) | hi;
        atomicAdd(&dplus[lo], 1);
    }
}

// out[off[u] + (u's arrival order)] = the pair; cur counts arrivals per row
__global__ void k_orient_scatter(const uint64_t* __restrict__ keys, int64_t m, int bits,
                                 const int64_t* __restrict__ off, int32_t* __restrict__ cur,
                                 uint64_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[e];
        const int64_t u = (int64_t)(k >> bits);
        out[off[u] + atomicAdd(&cur[u], 1)] = k;
    }
}

// Bitonic sort of a warp's 32*E columns, lane l holding entries l*E ..
// l*E + E - 1: exchanges at distances below E stay in a lane's registers,
// longer ones pair lanes by a shuffle.
template <int E>
__device__ __forceinline__ void warp_bitonic(uint32_t (&x)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int r = 0; r < E; ++r)
                    if ((r & j) == 0) {
                        const bool up = ((lane * E + r) & k) == 0;
                        const uint32_t a = x[r], c = x[r | j];
                        x[r] = up ? min(a, c) : max(a, c);
                        x[r | j] = up ? max(a, c) : min(a, c);
                    }
            } else {
                const int lj = j / E;
                const bool low = (lane & lj) == 0;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const uint32_t y = __shfl_xor_sync(0xffffffffu, x[r], lj);
                    const bool up = ((lane * E + r) & k) == 0;
                    x[r] = (low == up) ? min(x[r], y) : max(x[r], y);
                }
            }
        }
}

template <int E>
__device__ __forceinline__ void warp_sort_row(uint64_t* __restrict__ keys, int32_t* __restrict__ adj,
                                              int64_t rb, int d, uint64_t row, uint64_t mask) {
    const int lane = threadIdx.x & 31;
    uint32_t x[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int q = lane * E + r;
        x[r] = q < d ? (uint32_t)(keys[rb + q] & mask) : 0xffffffffu;
    }
    warp_bitonic<E>(x);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int q = lane * E + r;
        if (q < d) {
            keys[rb + q] = row | x[r];
            adj[rb + q] = (int32_t)x[r];
        }
    }
}

// Rows of at most kWarpRowMax entries: one warp each, sorted in registers.
// Longer rows are listed for k_row_sort_long.  adj = the columns.
constexpr int kWarpRowMax = 256;
__global__ void k_row_sort_short(uint64_t* __restrict__ keys, const int64_t* __restrict__ off, int64_t n,
                                 int bits, int32_t* __restrict__ adj, int32_t* __restrict__ longrows,
                                 int* __restrict__ nlong) {
    const uint64_t mask = (1ull << bits) - 1ull;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int64_t rb = off[r];
        const int64_t d = off[r + 1] - rb;
        const uint64_t row = (uint64_t)r << bits;
        if (d > kWarpRowMax) {
            if (lane == 0) longrows[atomicAdd(nlong, 1)] = (int32_t)r;
        } else if (d > 128) {
            warp_sort_row<kWarpRowMax / 32>(keys, adj, rb, (int)d, row, mask);
        } else if (d > 64) {
            warp_sort_row<4>(keys, adj, rb, (int)d, row, mask);
        } else if (d > 32) {
            warp_sort_row<2>(keys, adj, rb, (int)d, row, mask);
        } else if (d > 1) {
            warp_sort_row<1>(keys, adj, rb, (int)d, row, mask);
        } else if (d == 1 && lane == 0) {
            adj[rb] = (int32_t)(keys[rb] & mask);
        }
    }
}

// Rows of kWarpRowMax+1 .. kRowSortMax entries: one block each, a bitonic
// sort of the columns in shared memory (a row's keys share their row bits).
// A longer row (impossible within kOrientCountMaxM) sets error bit 8 and is
// skipped.
__global__ void __launch_bounds__(kRowSortThreads) k_row_sort_long(
        uint64_t* __restrict__ keys, const int64_t* __restrict__ off, int bits, int32_t* __restrict__ adj,
        const int32_t* __restrict__ longrows, const int* __restrict__ nlong, int* __restrict__ err) {
    __shared__ uint32_t v[kRowSortMax];
    const uint64_t mask = (1ull << bits) - 1ull;
    const int nl = *nlong;
    for (int x = blockIdx.x; x < nl; x += gridDim.x) {
        const int64_t r = longrows[x];
        const int64_t rb = off[r];
        const int d = (int)(off[r + 1] - rb);
        if (d > kRowSortMax) {
            if (threadIdx.x == 0) atomicOr(err, 8);
            continue;
        }
        int P = 2 * kWarpRowMax;
        while (P < d) P <<= 1;
        for (int q = threadIdx.x; q < P; q += blockDim.x)
            v[q] = q < d ? (uint32_t)(keys[rb + q] & mask) : 0xffffffffu;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int q = threadIdx.x; q < P; q += blockDim.x) {
                    const int l = q ^ j;
                    if (l > q) {
                        const uint32_t a = v[q], b = v[l];
                        const bool up = (q & k) == 0;
                        if ((a > b) == up) {
                            v[q] = b;
                            v[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
        const uint64_t row = (uint64_t)r << bits;
        for (int q = threadIdx.x; q < d; q += blockDim.x) {
            keys[rb + q] = row | v[q];
            adj[rb + q] = (int32_t)v[q];
        }
        __syncthreads();   // v is rewritten by the next row
    }
}

template <class OffT>
__global__ void k_store_offsets(const int64_t* __restrict__ off64, int64_t count,
                                OffT* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < count;
         v += (int64_t)gridDim.x * blockDim.x)
        out[v] = (OffT)off64[v];
}

// Task (i,j): edge e of U, row i, column j, with len = entries of U_i after j
// (> 0).  The tasks of pivot j are the edges of U that end at j -- its
// in-degree d-(j) = deg(j) - d+(j) -- less the rows whose last entry is j.
// Also sums the probes the <i,j,k> order would make, sum_j d-(j) d+(j).
template <class OffT>
__global__ void k_task_count_in(const int32_t* __restrict__ degn, const OffT* __restrict__ off,
                                int64_t n, int32_t* __restrict__ tcount,
                                unsigned long long* __restrict__ probes_ijk) {
    unsigned long long my = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t dp = (int32_t)(off[v + 1] - off[v]);
        const int32_t din = degn[v] - dp;
        tcount[v] = din;
        my += (unsigned long long)din * (unsigned long long)dp;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) my += __shfl_xor_sync(0xffffffffu, my, o);
    if ((threadIdx.x & 31) == 0 && my) atomicAdd(probes_ijk, my);
}

// ... and drop each row's last entry; probes = sum over rows of C(d+(i), 2)
template <class OffT>
__global__ void k_task_count_last(const OffT* __restrict__ off, const int32_t* __restrict__ adj,
                                  int64_t n, int32_t* __restrict__ tcount,
                                  unsigned long long* __restrict__ probes) {
    unsigned long long my = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t re = (int64_t)off[i + 1];
        const int64_t d = re - (int64_t)off[i];
        if (d > 0) {
            atomicSub(&tcount[adj[re - 1]], 1);
            my += (unsigned long long)(d * (d - 1) / 2);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) my += __shfl_xor_sync(0xffffffffu, my, o);
    if ((threadIdx.x & 31) == 0 && my) atomicAdd(probes, my);
}

// fill[j] starts at the first task slot of pivot j and is advanced
// atomically; each thread keeps kFillILP edges' atomics in flight at once.
#ifndef TC_FILL_ILP
#define TC_FILL_ILP 4
#endif
constexpr int kFillILP = TC_FILL_ILP;

template <class OffT>
__global__ void k_task_fill(const uint64_t* __restrict__ keys, int64_t m, int bits,
                            const OffT* __restrict__ off, unsigned long long* __restrict__ fill,
                            Task* __restrict__ tasks) {
    const uint64_t mask = (1ull << bits) - 1ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < m; e0 += stride * kFillILP) {
        int64_t i[kFillILP], len[kFillILP];
        int32_t j[kFillILP];
#pragma unroll
        for (int u = 0; u < kFillILP; ++u) {
            const int64_t e = e0 + u * stride;
            len[u] = 0;
            if (e < m) {
                const uint64_t k = keys[e];
                i[u] = (int64_t)(k >> bits);
                j[u] = (int32_t)(k & mask);
                len[u] = (int64_t)off[i[u] + 1] - e - 1;
            }
        }
        unsigned long long slot[kFillILP];
#pragma unroll
        for (int u = 0; u < kFillILP; ++u)
            if (len[u] > 0) slot[u] = atomicAdd(&fill[j[u]], 1ull);
#pragma unroll
        for (int u = 0; u < kFillILP; ++u)
            if (len[u] > 0) {
                Task t;
                t.start = e0 + u * stride + 1;
                t.len = (int32_t)len[u];
                t.i = (int32_t)i[u];
                tasks[slot[u]] = t;
            }
    }
}

template <class OffT>
__global__ void k_max_outdeg(const OffT* __restrict__ off, int64_t n, int* __restrict__ out) {
    int mx = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, (int)(off[v + 1] - off[v]));
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Host pairs into device memory by SM loads over the CPU-GPU link, for page-
// locked host memory the device can address.  On Grace-Blackwell these loads
// hold the link's rate where the copy engine's rate from the same buffer
// varies several-fold.  16-byte vectors when both ends allow them.
__global__ void k_upload_i32(const int32_t* __restrict__ src, int32_t* __restrict__ dst, int64_t count) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
        const int64_t n4 = count >> 2;
        const int4* s4 = reinterpret_cast<const int4*>(src);
        int4* d4 = reinterpret_cast<int4*>(dst);
        for (int64_t i = tid; i < n4; i += stride) d4[i] = s4[i];
        done = n4 << 2;
    }
    for (int64_t i = done + tid; i < count; i += stride) dst[i] = src[i];
}

// Uploads n int32 from host memory to dst on st by method 1 (copy engine)
// or 2 (SM loads from the device address dsrc of page-locked memory).
void upload_i32(const int32_t* hsrc, const int32_t* dsrc, int32_t* dst, int64_t n, int method,
                cudaStream_t st) {
    if (n <= 0) return;
    if (method == 2) {
        Prof prof_("k_upload_i32", st);
        k_upload_i32<<<(unsigned)(num_sms() * 8), 512, 0, st>>>(dsrc, dst, n);
    } else {
        TC_CUDA(cudaMemcpyAsync(dst, hsrc, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st));
    }
    TC_LAUNCH_CHECK();
}

// The device address of page-locked host memory (null for pageable memory
// or memory this device cannot address).
const int32_t* mapped_host(const int32_t* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<const int32_t*>(a.devicePointer);
}

// component of vertex v: largest c with vpre[c] <= v
__device__ __forceinline__ int comp_of(const int64_t* __restrict__ vpre, int num, int64_t v) {
    int lo = 0, hi = num - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vpre[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_check_comp(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                             int64_t P, const int64_t* __restrict__ vpre, int num,
                             int* __restrict__ err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P;
         e += (int64_t)gridDim.x * blockDim.x)
        if (comp_of(vpre, num, src[e]) != comp_of(vpre, num, dst[e])) atomicOr(err, 2);
}

__global__ void k_comp_new(const int32_t* __restrict__ perm, int64_t n, const int64_t* __restrict__ vpre,
                           int num, int32_t* __restrict__ comp) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        comp[perm[v]] = comp_of(vpre, num, v);
}

}  // namespace

void preprocess(tc_graph* g, const int32_t* src_in, const int32_t* dst_in, int64_t P,
                uint32_t flags, cudaStream_t st) {
    preprocess_with_components(g, src_in, dst_in, P, flags, nullptr, 0, st);
}

void preprocess_with_components(tc_graph* g, const int32_t* src_in, const int32_t* dst_in, int64_t P,
                                uint32_t flags, const int64_t* vpre_host, int32_t num_comps,
                                cudaStream_t st) {
    Alloc& al = g->alloc;
    const int64_t n = g->n;
    const int bits = g->bits;
    const unsigned G = (unsigned)(num_sms() * 8);

    // input on the device
    const int32_t* src = src_in;
    const int32_t* dst = dst_in;
    Buf<int32_t> hsrc, hdst;
    if (!(flags & TC_INPUT_ON_DEVICE) && P > 0) {
        hsrc = Buf<int32_t>(al, (size_t)P);
        hdst = Buf<int32_t>(al, (size_t)P);
        const auto t0 = std::chrono::steady_clock::now();
        const int32_t* ms = mapped_host(src_in);
        const int32_t* md = mapped_host(dst_in);
        if (ms && md) {
            // Page-locked pairs: the copy engine and SM loads over the link
            // reach different rates on different boxes (memory placement,
            // other traffic on the host side), and together no more than
            // the link gives (measured: running both at once, split by their
            // rates, was slower than the faster alone).  A large upload times
            // one slice each way and sends the rest by the faster.  The
            // slices are parts of the upload.
            constexpr int64_t kSlice = 32ll << 20;   // int32: 128 MB
            if (P >= 4 * kSlice) {
                cudaEvent_t e[3] = {};
                auto cleanup = [&]() {
                    for (auto& x : e)
                        if (x) cudaEventDestroy(x);
                };
                try {
                    for (auto& x : e) TC_CUDA(cudaEventCreate(&x));
                    TC_CUDA(cudaEventRecord(e[0], st));
                    upload_i32(src_in, ms, hsrc.get(), kSlice, 1, st);
                    TC_CUDA(cudaEventRecord(e[1], st));
                    upload_i32(src_in + kSlice, ms + kSlice, hsrc.get() + kSlice, kSlice, 2, st);
                    TC_CUDA(cudaEventRecord(e[2], st));
                    float ce = 0.f, sm = 0.f;
                    TC_CUDA(cudaEventSynchronize(e[2]));
                    TC_CUDA(cudaEventElapsedTime(&ce, e[0], e[1]));
                    TC_CUDA(cudaEventElapsedTime(&sm, e[1], e[2]));
                    g->upload_probe_gbs[0] = 4.0 * kSlice / (std::max(ce, 1e-6f) * 1e6);
                    g->upload_probe_gbs[1] = 4.0 * kSlice / (std::max(sm, 1e-6f) * 1e6);
                    const int method = ce < sm ? 1 : 2;
                    upload_i32(src_in + 2 * kSlice, ms + 2 * kSlice, hsrc.get() + 2 * kSlice, P - 2 * kSlice,
                               method, st);
                    upload_i32(dst_in, md, hdst.get(), P, method, st);
                    g->upload_method = method;
                } catch (...) {
                    cleanup();
                    throw;
                }
                cleanup();
            } else {
                upload_i32(src_in, ms, hsrc.get(), P, 2, st);
                upload_i32(dst_in, md, hdst.get(), P, 2, st);
                g->upload_method = 2;
            }
        } else {
            TC_CUDA(cudaMemcpyAsync(hsrc.get(), src_in, sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
            TC_CUDA(cudaMemcpyAsync(hdst.get(), dst_in, sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
            g->upload_method = 1;
        }
        g->upload_issue_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        src = hsrc.get();
        dst = hdst.get();
    }
    if (g->ev_uploaded) TC_CUDA(cudaEventRecord(g->ev_uploaded, st));

    Buf<int> scal(al, 8);   // [0] err, [1] max degree, [2] max out-degree, [3] heavy vertices
    TC_CUDA(cudaMemsetAsync(scal.get(), 0, 8 * sizeof(int), st));
    Buf<int64_t> vpre;
    if (num_comps > 0) {
        vpre = Buf<int64_t>(al, (size_t)num_comps + 1);
        // pageable source: the copy is staged before the call returns
        TC_CUDA(cudaMemcpyAsync(vpre.get(), vpre_host, sizeof(int64_t) * (size_t)(num_comps + 1),
                                cudaMemcpyHostToDevice, st));
    }
    Buf<int64_t> tot(al, 4);  // [0] m, [1] tasks

    // a1 + a2 + a3
    Buf<uint64_t> kb(al, (size_t)std::max<int64_t>(P, 1));
    uint64_t* keys = kb.get();
    Buf<uint64_t> ab;            // second key buffer: the sort's, or allocated for a5
    uint64_t* alt = nullptr;
    int64_t m = 0;
    Buf<int32_t> deg(al, (size_t)std::max<int64_t>(n, 1));
    TC_CUDA(cudaMemsetAsync(deg.get(), 0, sizeof(int32_t) * std::max<int64_t>(n, 1), st));
    TC_CUDA(cudaMemsetAsync(tot.get(), 0, sizeof(int64_t), st));
    if (P > 0 && P <= kHashDedupMaxPairs) {
        // canonical keys into a hash set, degrees on first insert, the set
        // compacted into E
        int64_t cap = 1024;
        while (cap < 2 * P) cap <<= 1;
        Buf<unsigned long long> table(al, (size_t)cap);
        TC_CUDA(cudaMemsetAsync(table.get(), 0xff, sizeof(unsigned long long) * (size_t)cap, st));
        {
            Prof prof_("k_dedup_insert", st);
            k_dedup_insert<<<grid_for(P, kT, G), kT, 0, st>>>(src, dst, P, n, bits, table.get(),
                                                              (uint64_t)(cap - 1), deg.get(), scal.get());
        }
        TC_LAUNCH_CHECK();
        if (num_comps > 0) {
            Prof prof_("k_check_comp", st);
            k_check_comp<<<grid_for(P, kT, G), kT, 0, st>>>(src, dst, P, vpre.get(), num_comps, scal.get());
        }
        TC_LAUNCH_CHECK();
        hsrc.release();
        hdst.release();
        {
            Prof prof_("k_table_compact", st);
            k_table_compact<<<grid_for(cap, kT * kCompactItems, G), kT, 0, st>>>(
                table.get(), cap, keys, reinterpret_cast<unsigned long long*>(tot.get()));
        }
        TC_LAUNCH_CHECK();
    } else if (P > 0) {
        // canonical keys, radix sorted, first of each run kept (making the
        // keys inside the sort's digit count and first pass, from the two
        // pair arrays, was slower: 19 ms against 14 for this pass, a key
        // pass and its share of the digit count)
        const uint64_t sentinel = (bits * 2 >= 64) ? ~0ull : ((1ull << (2 * bits)) - 1ull);
        ab = Buf<uint64_t>(al, (size_t)P);
        alt = ab.get();
        {
            Prof prof_("k_canon", st);
            k_canon<<<grid_for(P, kT, G), kT, 0, st>>>(src, dst, P, n, bits, sentinel, keys, scal.get());
        }
        TC_LAUNCH_CHECK();
        if (num_comps > 0) {
            Prof prof_("k_check_comp", st);
            k_check_comp<<<grid_for(P, kT, G), kT, 0, st>>>(src, dst, P, vpre.get(), num_comps, scal.get());
        }
        TC_LAUNCH_CHECK();
        hsrc.release();
        hdst.release();
        // ids outside [0, n) became sentinels; the error is read at the next sync
        radix_sort_u64(&keys, &alt, P, 0, 2 * bits, al, st, scal.get());
        {
            Buf<int32_t> fl(al, (size_t)P);
            Buf<int64_t> pos(al, (size_t)P);
            {
                Prof prof_("k_unique_flags", st);
                k_unique_flags<<<grid_for(P, kT, G), kT, 0, st>>>(keys, P, sentinel, fl.get());
            }
            TC_LAUNCH_CHECK();
            exclusive_scan_i32_to_i64(fl.get(), pos.get(), P, tot.get(), al, st);
            {
                Prof prof_("k_unique_compact", st);
                k_unique_compact<<<grid_for(P, kT, G), kT, 0, st>>>(keys, fl.get(), pos.get(), P, bits,
                                                                alt, deg.get());
            }
            TC_LAUNCH_CHECK();
        }
        std::swap(keys, alt);  // E now in `keys`
    }
    // one synchronisation for: errors so far, m, max degree, heavy vertices
    int maxdeg = 0, nheavy = 0;
    {
        if (n > 0) {
            Prof prof_("k_max_i32", st);
            k_max_i32<<<grid_for(n, kT, G), kT, 0, st>>>(deg.get(), n, scal.get() + 1);   // [1], [3]
        }
        TC_LAUNCH_CHECK();
        int hs[4] = {0, 0, 0, 0};
        TC_CUDA(cudaMemcpyAsync(hs, scal.get(), 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (P > 0) TC_CUDA(cudaMemcpyAsync(&m, tot.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        if (hs[0] & 1) TC_FAIL(TC_EINVAL, "tc_preprocess: a vertex id lies outside [0, n)");
        if (hs[0] & 2) TC_FAIL(TC_EINVAL, "tc_preprocess_components: a pair joins two components");
        if (hs[0] & 4) TC_FAIL(TC_ETIMEOUT, "tc_preprocess: a sort look-back wait ran past its bound");
        maxdeg = hs[1];
        nheavy = hs[3];
    }
    g->m = m;
    g->stats.m = m;
    if ((flags & TC_OFFSETS_32) && m >= (int64_t)0x7fffffff)
        TC_FAIL(TC_EINVAL, "tc_preprocess: 32-bit offsets requested but m = %lld", (long long)m);
    g->off64 = (flags & TC_OFFSETS_64) ? true : (flags & TC_OFFSETS_32) ? false
                                                                         : (m >= (int64_t)0x7fffffff);
    const size_t ob = g->off64 ? 8 : 4;

    // arena: off, adj, perm, loff, tasks (capacity m), counters, tnew
    size_t sz_off = align_up(ob * (size_t)(n + 1)), sz_adj = align_up(4 * (size_t)std::max<int64_t>(m, 1));
    size_t sz_perm = align_up(4 * (size_t)std::max<int64_t>(n, 1));
    size_t sz_loff = align_up(8 * (size_t)(n + 1));
    size_t sz_tasks = align_up(sizeof(Task) * (size_t)std::max<int64_t>(m, 1));
    size_t sz_ctr = align_up(sizeof(unsigned long long) * CTR_COUNT) + align_up(sizeof(GraphView));
    size_t sz_tnew = align_up(8 * (size_t)std::max<int64_t>(n, 1));
    size_t sz_comp = num_comps > 0 ? align_up(4 * (size_t)std::max<int64_t>(n, 1)) : 0;
    size_t sz_ctot = num_comps > 0 ? align_up(8 * (size_t)num_comps) : 0;
    sz_ctr += align_up(sizeof(GraphView));
    g->arena_bytes = sz_off + sz_adj + sz_perm + sz_loff + sz_tasks + sz_ctr + sz_tnew + sz_comp + sz_ctot;
    g->arena = al.get(g->arena_bytes);
    char* a = static_cast<char*>(g->arena);
    g->off = a; a += sz_off;
    g->adj = reinterpret_cast<int32_t*>(a); a += sz_adj;
    g->perm = reinterpret_cast<int32_t*>(a); a += sz_perm;
    g->loff = reinterpret_cast<int64_t*>(a); a += sz_loff;
    g->tasks = reinterpret_cast<Task*>(a); a += sz_tasks;
    g->counters = reinterpret_cast<unsigned long long*>(a);
    g->view = reinterpret_cast<GraphView*>(a + align_up(sizeof(unsigned long long) * CTR_COUNT));
    g->view_comp = reinterpret_cast<GraphView*>(a + align_up(sizeof(unsigned long long) * CTR_COUNT) +
                                                align_up(sizeof(GraphView)));
    a += sz_ctr;
    g->tnew = reinterpret_cast<uint64_t*>(a);
    a += sz_tnew;
    if (num_comps > 0) {
        g->comp = reinterpret_cast<int32_t*>(a);
        a += sz_comp;
        g->comp_totals = reinterpret_cast<unsigned long long*>(a);
        g->num_comps = num_comps;
    }

    // a4 relabel
    if (n > 0) {
        Buf<uint64_t> dk(al, (size_t)n), da(al, (size_t)n);
        uint64_t* dkeys = dk.get();
        uint64_t* dalt = da.get();
        if (TC_DEGREE_COUNTING && n >= kCountingMinVertices) {
            // the counting sort of Section 5.3 for degrees below kHeavy (one
            // stable pass), the heavy tail sorted on its full degrees
            {
                Prof prof_("k_degree_keys", st);
                k_degree_keys_clipped<<<grid_for(n, kT, G), kT, 0, st>>>(deg.get(), n, bits, dkeys);
            }
            TC_LAUNCH_CHECK();
            radix_sort_u64(&dkeys, &dalt, n, bits, bits + 8, al, st, scal.get());
            // the heavy tail's keys are read (degrees by original id) before
            // k_perm overwrites deg with the degrees in rank order
            Buf<uint64_t> hk, ha;
            uint64_t* hkeys = nullptr;
            uint64_t* halt = nullptr;
            if (nheavy > 0) {
                hk = Buf<uint64_t>(al, (size_t)nheavy);
                ha = Buf<uint64_t>(al, (size_t)nheavy);
                hkeys = hk.get();
                halt = ha.get();
                {
                    Prof prof_("k_heavy_keys", st);
                    k_heavy_keys<<<grid_for(nheavy, kT, G), kT, 0, st>>>(dkeys, n, nheavy, bits, deg.get(), hkeys);
                }
                TC_LAUNCH_CHECK();
            }
            {
                Prof prof_("k_perm", st);
                k_perm<<<grid_for(n - nheavy, kT, G), kT, 0, st>>>(dkeys, n - nheavy, bits, g->perm, deg.get());
            }
            TC_LAUNCH_CHECK();
            if (nheavy > 0) {
                const int dbits = ceil_log2_u64((uint64_t)maxdeg + 1);
                radix_sort_u64(&hkeys, &halt, nheavy, bits, bits + dbits, al, st, scal.get());
                {
                    Prof prof_("k_perm", st);
                    k_perm_at<<<grid_for(nheavy, kT, G), kT, 0, st>>>(hkeys, nheavy, n - nheavy, bits, g->perm,
                                                                      deg.get());
                }
                TC_LAUNCH_CHECK();
            }
        } else {
            {
                Prof prof_("k_degree_keys", st);
                k_degree_keys<<<grid_for(n, kT, G), kT, 0, st>>>(deg.get(), n, bits, dkeys);
            }
            TC_LAUNCH_CHECK();
            int dbits = ceil_log2_u64((uint64_t)maxdeg + 1);
            radix_sort_u64(&dkeys, &dalt, n, bits, bits + dbits, al, st, scal.get());
            {
                Prof prof_("k_perm", st);
                k_perm<<<grid_for(n, kT, G), kT, 0, st>>>(dkeys, n, bits, g->perm, deg.get());
            }
            TC_LAUNCH_CHECK();
        }
    }
    g->stats.max_deg = maxdeg;
    if (num_comps > 0 && n > 0) {
        Prof prof_("k_comp_new", st);
        k_comp_new<<<grid_for(n, kT, G), kT, 0, st>>>(g->perm, n, vpre.get(), num_comps, g->comp);
    }
    TC_LAUNCH_CHECK();

    // a5 orient and build U
    Buf<int32_t> dplus(al, (size_t)std::max<int64_t>(n, 1));
    TC_CUDA(cudaMemsetAsync(dplus.get(), 0, sizeof(int32_t) * std::max<int64_t>(n, 1), st));
    Buf<int64_t> off64(al, (size_t)(n + 1));
    if (!alt) {
        ab = Buf<uint64_t>(al, (size_t)std::max<int64_t>(m, 1));
        alt = ab.get();
    }
    if (m > 0 && m <= kOrientCountMaxM) {
        {
            Prof prof_("k_orient_count", st);
            k_orient_count<<<grid_for(m, kT, G), kT, 0, st>>>(keys, m, bits, g->perm, alt, dplus.get());
        }
        TC_LAUNCH_CHECK();
        // off = exclusive scan of dplus, with off[n] = m
        exclusive_scan_i32_to_i64(dplus.get(), off64.get(), n, off64.get() + n, al, st);
        TC_CUDA(cudaMemsetAsync(dplus.get(), 0, sizeof(int32_t) * (size_t)n, st));
        {
            Prof prof_("k_orient_scatter", st);
            k_orient_scatter<<<grid_for(m, kT, G), kT, 0, st>>>(alt, m, bits, off64.get(), dplus.get(), keys);
        }
        TC_LAUNCH_CHECK();
        Buf<int32_t> longrows(al, (size_t)(m / (kWarpRowMax + 1) + 1));
        {
            Prof prof_("k_row_sort_short", st);
            k_row_sort_short<<<grid_for(32 * n, kT, G), kT, 0, st>>>(keys, off64.get(), n, bits, g->adj,
                                                                    longrows.get(), scal.get() + 4);
        }
        TC_LAUNCH_CHECK();
        {
            Prof prof_("k_row_sort_long", st);
            k_row_sort_long<<<(unsigned)std::min<int64_t>(m / (kWarpRowMax + 1) + 1, 4 * (int64_t)num_sms()),
                              kRowSortThreads, 0, st>>>(keys, off64.get(), bits, g->adj, longrows.get(),
                                                        scal.get() + 4, scal.get());
        }
        TC_LAUNCH_CHECK();
    } else {
        if (m > 0) {
            {
                Prof prof_("k_orient", st);
                k_orient<<<grid_for(m, kT, G), kT, 0, st>>>(keys, m, bits, g->perm, alt);
            }
            TC_LAUNCH_CHECK();
            std::swap(keys, alt);
            radix_sort_u64(&keys, &alt, m, 0, 2 * bits, al, st, scal.get());
            {
                Prof prof_("k_adj_rows", st);
                k_adj_rows<<<grid_for(m, kT, G), kT, 0, st>>>(keys, m, bits, g->adj, dplus.get());
            }
            TC_LAUNCH_CHECK();
        }
        // off = exclusive scan of dplus, with off[n] = m
        exclusive_scan_i32_to_i64(dplus.get(), off64.get(), n, off64.get() + n, al, st);
    }
    if (g->off64) {
        TC_CUDA(cudaMemcpyAsync(g->off, off64.get(), 8 * (size_t)(n + 1), cudaMemcpyDeviceToDevice, st));
    } else {
        {
            Prof prof_("k_store_offsets", st);
            k_store_offsets<int32_t><<<grid_for(n + 1, kT, G), kT, 0, st>>>(
            off64.get(), n + 1, static_cast<int32_t*>(g->off));
        }
        TC_LAUNCH_CHECK();
    }

    // a6 tasks grouped by pivot j
    Buf<unsigned long long> probes(al, 2);   // [0] <j,i,k> probes, [1] <i,j,k> probes
    TC_CUDA(cudaMemsetAsync(probes.get(), 0, 2 * sizeof(unsigned long long), st));
    int32_t* tcount = dplus.get();  // reuse
    if (n > 0) {
        {
            Prof prof_("k_task_count_in", st);
            if (g->off64)
                k_task_count_in<int64_t><<<grid_for(n, kT, G), kT, 0, st>>>(
                    deg.get(), static_cast<const int64_t*>(g->off), n, tcount, probes.get() + 1);
            else
                k_task_count_in<int32_t><<<grid_for(n, kT, G), kT, 0, st>>>(
                    deg.get(), static_cast<const int32_t*>(g->off), n, tcount, probes.get() + 1);
        }
        TC_LAUNCH_CHECK();
        {
            Prof prof_("k_task_count_last", st);
            if (g->off64)
                k_task_count_last<int64_t><<<grid_for(n, kT, G), kT, 0, st>>>(
                    static_cast<const int64_t*>(g->off), g->adj, n, tcount, probes.get());
            else
                k_task_count_last<int32_t><<<grid_for(n, kT, G), kT, 0, st>>>(
                    static_cast<const int32_t*>(g->off), g->adj, n, tcount, probes.get());
        }
        TC_LAUNCH_CHECK();
    }
    deg.release();
    exclusive_scan_i32_to_i64(tcount, g->loff, n, g->loff + n, al, st);
    if (m > 0) {
        Buf<unsigned long long> fill(al, (size_t)std::max<int64_t>(n, 1));
        TC_CUDA(cudaMemcpyAsync(fill.get(), g->loff, sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1),
                                cudaMemcpyDeviceToDevice, st));
        {
            Prof prof_("k_task_fill", st);
            if (g->off64)
                k_task_fill<int64_t><<<grid_for(m, kT, G), kT, 0, st>>>(
                    keys, m, bits, static_cast<const int64_t*>(g->off), fill.get(), g->tasks);
            else
                k_task_fill<int32_t><<<grid_for(m, kT, G), kT, 0, st>>>(
                    keys, m, bits, static_cast<const int32_t*>(g->off), fill.get(), g->tasks);
        }
        TC_LAUNCH_CHECK();
    }
    int maxout = 0;
    if (n > 0) {
        if (g->off64)
            {
                Prof prof_("k_max_outdeg", st);
                k_max_outdeg<int64_t><<<grid_for(n, kT, G), kT, 0, st>>>(
                static_cast<const int64_t*>(g->off), n, scal.get() + 2);
            }
        else
            {
                Prof prof_("k_max_outdeg", st);
                k_max_outdeg<int32_t><<<grid_for(n, kT, G), kT, 0, st>>>(
                static_cast<const int32_t*>(g->off), n, scal.get() + 2);
            }
        TC_LAUNCH_CHECK();
    }
    // the device view the count kernel reads (pageable sources: staged on return)
    {
        GraphView v{};
        v.off = g->off;
        v.adj = g->adj;
        v.loff = g->loff;
        v.tasks = g->tasks;
        v.tnew = reinterpret_cast<unsigned long long*>(g->tnew);
        v.total = g->counters + CTR_TOTAL;
        v.n = n;
        v.off64 = g->off64 ? 1 : 0;
        TC_CUDA(cudaMemcpyAsync(g->view, &v, sizeof(v), cudaMemcpyHostToDevice, st));
        GraphView vc = v;
        vc.tnew = nullptr;
        vc.comp = g->comp;
        vc.comp_totals = g->comp_totals;
        TC_CUDA(cudaMemcpyAsync(g->view_comp, &vc, sizeof(vc), cudaMemcpyHostToDevice, st));
    }

    // a6 work units for the default tuning, sized at the same synchronisation
    // as the task statistics
    tc_tuning def;
    tuning_defaults(&def);
    def = clamp_tuning(size_tuning(def, m));
    Buf<int64_t> gvpre(al, 2);
    const int64_t hv[2] = {0, n};
    TC_CUDA(cudaMemcpyAsync(gvpre.get(), hv, sizeof(hv), cudaMemcpyHostToDevice, st));
    UnitPlan plan;
    plan_units(plan, g->view, gvpre.get(), 1, n, def, al, st);
    unsigned long long hprobes[2] = {0, 0};
    int64_t ntasks = 0, ns = 0, nl = 0;
    int herr = 0;
    TC_CUDA(cudaMemcpyAsync(&maxout, scal.get() + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&herr, scal.get(), sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(hprobes, probes.get(), sizeof(hprobes), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&ntasks, g->loff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&ns, plan.ps.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&nl, plan.pl.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (herr & 4) TC_FAIL(TC_ETIMEOUT, "tc_preprocess: a sort look-back wait ran past its bound");
    if (herr & 8) TC_FAIL(TC_EUNSUPPORTED, "tc_preprocess: a row of U exceeds the row sort's bound");
    g->n_tasks = ntasks;
    g->stats.max_outdeg = maxout;
    g->stats.tasks = ntasks;
    g->stats.probes = hprobes[0];
    g->stats.probes_ijk = hprobes[1];
    g->stats.offset_bytes = (int32_t)ob;
    UnitLists L = fill_units(plan, ns, nl, al, st);
    adopt_units(g, L, def);
    g->stats.device_bytes = (int64_t)(g->arena_bytes + g->units_bytes);
}

}  // namespace tc
