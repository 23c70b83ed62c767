// Stable LSD radix sort of 64-bit keys on a bit range, 8-bit digits.
//
// Per digit: (1) every tile of kTile keys counts its digits into per-warp
// shared histograms (plain shared atomics; a warp whose keys all share one
// digit adds once), written digit-major to the (digit, tile) table; (2) one
// exclusive scan of that table gives each (digit, tile) its output offset;
// (3) every tile loads its keys into shared memory, ranks them stably (warp w
// owns a contiguous segment; the lanes holding the same digit are found with
// one ballot per digit bit, and a running per-warp counter orders the
// rounds), permutes them into digit order in shared memory and writes each
// digit run out contiguously.
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
    uint64_t k[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t idx = base + r * 32 + lane;
        k[r] = idx < count ? keys[idx] : 0;
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const bool valid = base + r * 32 + lane < count;
        const unsigned d = digit_of(k[r], shift, mask);
        const unsigned d0 = __shfl_sync(0xffffffffu, d, 0);
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (__all_sync(0xffffffffu, !valid || d == d0)) {
            if (lane == 0 && vm) atomicAdd(&hist[w][d0], (unsigned)__popc(vm));
        } else if (valid) {
            atomicAdd(&hist[w][d], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d <= (int)mask; d += kThreads) {
        unsigned s = 0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) s += hist[q][d];
        H[(int64_t)d * nblocks + blockIdx.x] = s;
    }
}

// Lanes of the warp whose digit equals this lane's (one ballot per digit bit).
__device__ __forceinline__ unsigned digit_peers(unsigned d, int nbits, unsigned valid_mask) {
    unsigned peers = valid_mask;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (b < nbits) {
            const bool bit = (d >> b) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
    }
    return peers;
}

__global__ void __launch_bounds__(kThreads, 4) k_scatter(const uint64_t* __restrict__ in,
                                                         uint64_t* __restrict__ out, int64_t count,
                                                         int shift, int nbits,
                                                         const int64_t* __restrict__ H,
                                                         int64_t nblocks) {
    __shared__ uint64_t stage[kTile];
    __shared__ unsigned short rank_s[kTile];
    __shared__ unsigned short wcnt[kWarps][kRadix];   // counts, then per-warp exclusive prefix
    __shared__ unsigned dstart[kRadix];               // tile-local start of each digit run
    __shared__ unsigned wsum[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned mask = (1u << nbits) - 1u;
    const int64_t tbase = (int64_t)blockIdx.x * kTile;
    const int valid_in_tile = (int)min64((int64_t)kTile, count - tbase);

    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int p = k * kThreads + threadIdx.x;
        if (p < valid_in_tile) stage[p] = in[tbase + p];
    }
    __syncthreads();

    // stable ranks within each warp's segment
    const int seg = w * kSeg;
#pragma unroll 4
    for (int r = 0; r < kRounds; ++r) {
        const int p = seg + r * 32 + lane;
        const bool valid = p < valid_in_tile;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        const unsigned d = valid ? digit_of(stage[p], shift, mask) : 0u;
        const unsigned peers = digit_peers(d, nbits, vm);
        const unsigned prior = valid ? wcnt[w][d] : 0u;
        __syncwarp();
        if (valid) {
            rank_s[p] = (unsigned short)(prior + __popc(peers & lt));
            if (lane == __ffs(peers) - 1) wcnt[w][d] = (unsigned short)(prior + __popc(peers));
        }
        __syncwarp();
    }
    __syncthreads();
    // per-warp exclusive prefix per digit, and digit totals
    unsigned tot = 0;
    {
        const int d = threadIdx.x;   // kThreads == kRadix
#pragma unroll
        for (int q = 0; q < kWarps; ++q) {
            const unsigned c = wcnt[q][d];
            wcnt[q][d] = (unsigned short)tot;
            tot += c;
        }
    }
    unsigned inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    unsigned before = 0;
    for (int q = 0; q < w; ++q) before += wsum[q];
    dstart[threadIdx.x] = before + inc - tot;
    __syncthreads();
    // permute into digit order inside the tile
    uint64_t key[kItems];
    unsigned pos[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int p = k * kThreads + threadIdx.x;
        if (p < valid_in_tile) {
            key[k] = stage[p];
            const unsigned d = digit_of(key[k], shift, mask);
            pos[k] = dstart[d] + wcnt[p / kSeg][d] + rank_s[p];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int p = k * kThreads + threadIdx.x;
        if (p < valid_in_tile) stage[pos[k]] = key[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int p = k * kThreads + threadIdx.x;
        if (p < valid_in_tile) {
            const uint64_t kk = stage[p];
            const unsigned d = digit_of(kk, shift, mask);
            out[H[(int64_t)d * nblocks + blockIdx.x] + (p - (int)dstart[d])] = kk;
        }
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
            k_scatter<<<(unsigned)nblocks, kThreads, 0, st>>>(*keys, *alt, count, shift, nbits, H.get(),
                                                              nblocks);
        }
        TC_LAUNCH_CHECK();
        uint64_t* t = *keys;
        *keys = *alt;
        *alt = t;
    }
}

}  // namespace tc
