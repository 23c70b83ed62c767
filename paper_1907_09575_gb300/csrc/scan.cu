// Device-wide exclusive prefix sums (reduce-then-scan, recursive over tiles).
#include "common.cuh"

namespace tc {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; returns the
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t s = (lane < kThreads / 32) ? warp_sums[lane] : 0;
        s = warp_incl_scan(s);
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    int64_t before = (w > 0) ? warp_sums[w - 1] : 0;
    *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

template <class Tin>
__global__ void __launch_bounds__(kThreads) k_tile_reduce(const Tin* __restrict__ in, int64_t count,
                                                          int64_t* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t idx = base + (int64_t)k * kThreads + threadIdx.x;
        if (idx < count) s += (int64_t)in[idx];
    }
    int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// offsets: per-tile exclusive offsets (or null for a single tile).  When
// total is non-null the last tile writes the grand total there.
template <class Tin>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const Tin* in, int64_t* out, int64_t count,
                                                        const int64_t* __restrict__ offsets,
                                                        int64_t* total) {
    __shared__ int64_t tile[kTile];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    // coalesced load into shared memory
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int idx = k * kThreads + threadIdx.x;
        int64_t g = base + idx;
        tile[idx] = (g < count) ? (int64_t)in[g] : 0;
    }
    __syncthreads();
    int64_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = tile[threadIdx.x * kItems + k];
        s += v[k];
    }
    int64_t tot;
    int64_t run = block_excl_scan(s, &tot) + (offsets ? offsets[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        tile[threadIdx.x * kItems + k] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int idx = k * kThreads + threadIdx.x;
        int64_t g = base + idx;
        if (g < count) out[g] = tile[idx];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kThreads - 1)
        *total = run;  // the last thread's running sum after its items = grand total
}

// Arrays of up to kBlockMax entries in one launch: one block streams the
// array through shared memory in chunks of kChunk entries (coalesced loads
// and stores; each thread scans kPer contiguous entries of the chunk), the
// running total carried from chunk to chunk.
constexpr int kBlockThreads = 1024;
constexpr int kPer = 4;
constexpr int kChunk = kBlockThreads * kPer;
constexpr int64_t kBlockMax = 16ll * kChunk;

template <class Tin>
__global__ void __launch_bounds__(kBlockThreads) k_block_scan(const Tin* in, int64_t* out, int64_t count,
                                                              int64_t* total) {
    __shared__ int64_t buf[kChunk];
    __shared__ int64_t warp_sums[kBlockThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < count; c0 += kChunk) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int idx = k * kBlockThreads + threadIdx.x;
            buf[idx] = (c0 + idx < count) ? (int64_t)in[c0 + idx] : 0;
        }
        __syncthreads();
        int64_t v[kPer], sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            v[k] = buf[threadIdx.x * kPer + k];
            sum += v[k];
        }
        const int64_t inc = warp_incl_scan(sum);
        if (lane == 31) warp_sums[w] = inc;
        __syncthreads();
        if (w == 0) warp_sums[lane] = warp_incl_scan(warp_sums[lane]);
        __syncthreads();
        int64_t run = carry + (w > 0 ? warp_sums[w - 1] : 0) + inc - sum;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            buf[threadIdx.x * kPer + k] = run;
            run += v[k];
        }
        carry += warp_sums[kBlockThreads / 32 - 1];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int idx = k * kBlockThreads + threadIdx.x;
            if (c0 + idx < count) out[c0 + idx] = buf[idx];
        }
        __syncthreads();   // buf and warp_sums are rewritten by the next chunk
    }
    if (total && threadIdx.x == 0) *total = carry;
}

template <class Tin>
void scan_impl(const Tin* in, int64_t* out, int64_t count, int64_t* total_dev, Alloc& al,
               cudaStream_t st) {
    if (count <= 0) {
        if (total_dev) TC_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), st));
        return;
    }
    int64_t tiles = (count + kTile - 1) / kTile;
    if (tiles > 1 && count <= kBlockMax) {
        {
            Prof prof_("k_block_scan", st);
            k_block_scan<Tin><<<1, kBlockThreads, 0, st>>>(in, out, count, total_dev);
        }
        TC_LAUNCH_CHECK();
        return;
    }
    if (tiles == 1) {
        {
            Prof prof_("k_tile_scan", st);
            k_tile_scan<Tin><<<1, kThreads, 0, st>>>(in, out, count, nullptr, total_dev);
        }
        TC_LAUNCH_CHECK();
        return;
    }
    Buf<int64_t> sums(al, (size_t)tiles);
    {
        Prof prof_("k_tile_reduce", st);
        k_tile_reduce<Tin><<<(unsigned)tiles, kThreads, 0, st>>>(in, count, sums.get());
    }
    TC_LAUNCH_CHECK();
    scan_impl<int64_t>(sums.get(), sums.get(), tiles, nullptr, al, st);
    {
        Prof prof_("k_tile_scan", st);
        k_tile_scan<Tin><<<(unsigned)tiles, kThreads, 0, st>>>(in, out, count, sums.get(), total_dev);
    }
    TC_LAUNCH_CHECK();
}

}  // namespace

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t count, int64_t* total_dev,
                        Alloc& al, cudaStream_t st) {
    scan_impl<int64_t>(in, out, count, total_dev, al, st);
}

void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t count,
                               int64_t* total_dev, Alloc& al, cudaStream_t st) {
    scan_impl<int32_t>(in, out, count, total_dev, al, st);
}

}  // namespace tc
