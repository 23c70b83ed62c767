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

// Arrays of up to kBlockMax entries in one launch.  Warp w owns the
// contiguous segment [w * 32 * per, (w + 1) * 32 * per), read a row of 32
// entries at a time (lane l takes entry l of each row: coalesced).  Pass 1
// sums each warp's segment; the warp sums are scanned across the block;
// pass 2 re-reads the rows (now from cache) and scans each across the warp,
// carrying the running sum from row to row.  in may equal out: each entry is
// read by the lane that writes it, before it writes it.
constexpr int kBlockThreads = 1024;
constexpr int64_t kBlockMax = 65536;
constexpr int kRowBatch = 8;

// Block b scans array b: two arrays of the same length in one launch.
template <class Tin>
__global__ void __launch_bounds__(kBlockThreads) k_block_scan(const Tin* in, int64_t* out, int64_t count,
                                                              int64_t* total, const Tin* in1, int64_t* out1,
                                                              int64_t* total1) {
    if (blockIdx.x == 1) {
        in = in1;
        out = out1;
        total = total1;
    }
    __shared__ int64_t warp_sums[kBlockThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = (count + kBlockThreads - 1) / kBlockThreads;   // rows per warp
    const int64_t seg = (int64_t)w * 32 * per;
    int64_t sum = 0;
    for (int64_t r0 = 0; r0 < per; r0 += kRowBatch) {
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
            const int64_t q = seg + (r0 + u) * 32 + lane;
            sum += (r0 + u < per && q < count) ? (int64_t)in[q] : 0;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) warp_sums[w] = sum;
    __syncthreads();
    if (w == 0) warp_sums[lane] = warp_incl_scan(warp_sums[lane]);
    __syncthreads();
    int64_t carry = (w > 0) ? warp_sums[w - 1] : 0;
    for (int64_t r0 = 0; r0 < per; r0 += kRowBatch) {
        int64_t v[kRowBatch];
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
            const int64_t q = seg + (r0 + u) * 32 + lane;
            v[u] = (r0 + u < per && q < count) ? (int64_t)in[q] : 0;
        }
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
            const int64_t q = seg + (r0 + u) * 32 + lane;
            const int64_t inc = warp_incl_scan(v[u]);
            if (r0 + u < per && q < count) out[q] = carry + inc - v[u];
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    if (total && threadIdx.x == 0) *total = warp_sums[kBlockThreads / 32 - 1];
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
            k_block_scan<Tin><<<1, kBlockThreads, 0, st>>>(in, out, count, total_dev, nullptr, nullptr,
                                                            nullptr);
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

void exclusive_scan2_i32_to_i64(const int32_t* in0, int64_t* out0, int64_t* total0, const int32_t* in1,
                                int64_t* out1, int64_t* total1, int64_t count, Alloc& al, cudaStream_t st) {
    if (count <= 0 || count > kBlockMax) {
        scan_impl<int32_t>(in0, out0, count, total0, al, st);
        scan_impl<int32_t>(in1, out1, count, total1, al, st);
        return;
    }
    {
        Prof prof_("k_block_scan", st);
        k_block_scan<int32_t><<<2, kBlockThreads, 0, st>>>(in0, out0, count, total0, in1, out1, total1);
    }
    TC_LAUNCH_CHECK();
}

}  // namespace tc
