// Stable LSD radix sort of 64-bit keys on a bit range, 8-bit digits.
//
// Per digit: (1) every tile of kTile keys histograms its digits (warp peers
// found with __match_any_sync, so equal digits cost one shared atomic per
// warp), written digit-major; (2) one exclusive scan over that table gives
// each (digit, tile) its global output offset; (3) every tile ranks its keys
// stably (warp w owns a contiguous segment, ranks come from match_any peer
// masks plus a running per-warp counter), permutes them into digit order in
// shared memory and writes each digit run out contiguously.
#include "common.cuh"

namespace tc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                 // keys per thread
constexpr int kTile = kThreads * kItems;   // 4096 keys per tile
constexpr int kSeg = kTile / kWarps;       // 512 keys per warp segment
constexpr int kRounds = kSeg / 32;         // 16 rounds of 32 keys
constexpr int kRadix = 256;

__device__ __forceinline__ unsigned digit_of(uint64_t k, int shift, unsigned mask) {
    return (unsigned)(k >> shift) & mask;
}

__global__ void __launch_bounds__(kThreads) k_hist(const uint64_t* __restrict__ keys, int64_t count,
                                                   int shift, unsigned mask,
                                                   int64_t* __restrict__ H, int64_t nblocks) {
    __shared__ unsigned hist[kWarps][kRadix];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)w * kSeg;
#pragma unroll 4
    for (int r = 0; r < kRounds; ++r) {
        int64_t idx = base + r * 32 + lane;
        bool valid = idx < count;
        unsigned d = valid ? digit_of(keys[idx], shift, mask) : (kRadix + lane);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) hist[w][d] += __popc(peers);
    }
    __syncthreads();
    for (int d = threadIdx.x; d <= (int)mask; d += kThreads) {
        unsigned s = 0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) s += hist[q][d];
        H[(int64_t)d * nblocks + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads) k_scatter(const uint64_t* __restrict__ in,
                                                      uint64_t* __restrict__ out, int64_t count,
                                                      int shift, unsigned mask,
                                                      const int64_t* __restrict__ H,
                                                      int64_t nblocks) {
    __shared__ uint64_t stage[kTile];
    __shared__ unsigned wcnt[kWarps][kRadix];   // counts, then per-warp exclusive prefix
    __shared__ unsigned dstart[kRadix];         // tile-local start of each digit run
    __shared__ unsigned wsum[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();

    const int64_t tbase = (int64_t)blockIdx.x * kTile;
    const int64_t base = tbase + (int64_t)w * kSeg;
    uint64_t key[kRounds];
    unsigned rank[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        int64_t idx = base + r * 32 + lane;
        bool valid = idx < count;
        key[r] = valid ? in[idx] : 0;
        unsigned d = valid ? digit_of(key[r], shift, mask) : (kRadix + lane);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned prior = valid ? wcnt[w][d] : 0;
        __syncwarp();
        rank[r] = prior + __popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = prior + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per-warp exclusive prefix per digit, and digit totals
    unsigned tot = 0;
    if (threadIdx.x < kRadix) {
        const int d = threadIdx.x;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) {
            unsigned c = wcnt[q][d];
            wcnt[q][d] = tot;
            tot += c;
        }
    }
    // exclusive scan of the 256 digit totals (one per thread)
    unsigned inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    unsigned before = 0;
    for (int q = 0; q < w; ++q) before += wsum[q];
    if (threadIdx.x < kRadix) dstart[threadIdx.x] = before + inc - tot;
    __syncthreads();
    // permute into digit order inside the tile
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        int64_t idx = base + r * 32 + lane;
        if (idx < count) {
            unsigned d = digit_of(key[r], shift, mask);
            stage[dstart[d] + wcnt[w][d] + rank[r]] = key[r];
        }
    }
    __syncthreads();
    const int valid_in_tile = (int)min64((int64_t)kTile, count - tbase);
    for (int p = threadIdx.x; p < valid_in_tile; p += kThreads) {
        uint64_t k = stage[p];
        unsigned d = digit_of(k, shift, mask);
        int64_t g = H[(int64_t)d * nblocks + blockIdx.x] + (p - (int)dstart[d]);
        out[g] = k;
    }
}

}  // namespace

void radix_sort_u64(uint64_t** keys, uint64_t** alt, int64_t count, int lo, int hi, Alloc& al,
                    cudaStream_t st) {
    if (count <= 1 || hi <= lo) return;
    const int64_t nblocks = (count + kTile - 1) / kTile;
    Buf<int64_t> H(al, (size_t)(kRadix * nblocks));
    for (int shift = lo; shift < hi; shift += 8) {
        const int nbits = min(8, hi - shift);
        const unsigned mask = (1u << nbits) - 1u;
        const int64_t rows = (int64_t)(mask + 1) * nblocks;
        {
            Prof prof_("k_hist", st);
            k_hist<<<(unsigned)nblocks, kThreads, 0, st>>>(*keys, count, shift, mask, H.get(), nblocks);
        }
        TC_LAUNCH_CHECK();
        exclusive_scan_i64(H.get(), H.get(), rows, nullptr, al, st);
        {
            Prof prof_("k_scatter", st);
            k_scatter<<<(unsigned)nblocks, kThreads, 0, st>>>(*keys, *alt, count, shift, mask, H.get(),
                                                          nblocks);
        }
        TC_LAUNCH_CHECK();
        uint64_t* t = *keys;
        *keys = *alt;
        *alt = t;
    }
}

}  // namespace tc
