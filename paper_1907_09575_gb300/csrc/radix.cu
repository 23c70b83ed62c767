// Stable LSD radix sort of 64-bit keys on a bit range, 8-bit digits.
//
// One kernel first counts every digit position of every key (LSD passes only
// permute keys, so all passes' global digit counts are known up front).  Then
// each pass is one kernel: a tile of kTile keys, taken in launch order from a
// tile counter, is staged in shared memory and ranked stably (warp w owns a
// contiguous segment; the lanes holding the same digit are found with one
// ballot per digit bit, and a running per-warp counter orders the rounds);
// the tile publishes its digit counts and finds, per digit, how many keys
// earlier tiles hold by looking back over their published counts (decoupled
// look-back: a tile that has its inclusive prefix publishes it, so the walk
// stops there); it then permutes its keys into digit order in shared memory
// and writes each digit run out contiguously.  Look-back waits are bounded:
// past the bound the pass records an error and the sort reports TC_ETIMEOUT.
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

constexpr int kMaxPasses = 8;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1ull;
constexpr long kSpinLimit = 1l << 24;

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Waits until the status word *q carries a flag (top two bits), at most
// `limit` polls; true with the word in v, false when the bound ran out.
__device__ __forceinline__ bool wait_published(const unsigned long long* q, unsigned long long& v,
                                               long limit) {
    v = ld_relaxed(q);
    long spins = 0;
    while ((v >> 62) == 0) {
        if (++spins > limit) return false;
        __nanosleep(32);
        v = ld_relaxed(q);
    }
    return true;
}

// One warp waits, bounded, on a word nothing publishes: the look-back's wait
// running out, error bit 4 set, the kernel returning.
__global__ void k_wait_selftest(const unsigned long long* word, long limit, int* err) {
    unsigned long long v;
    if (!wait_published(word, v, limit) && threadIdx.x == 0) atomicOr(err, 4);
}

// Global digit counts of every pass: hist[pass][digit], bits [lo, hi).
__global__ void __launch_bounds__(kThreads) k_digit_hist(const uint64_t* __restrict__ keys,
                                                         int64_t count, int lo, int npass, int hi,
                                                         unsigned long long* __restrict__ hist) {
    __shared__ unsigned h[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += kThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t base = blockIdx.x * (int64_t)kThreads; base < count; base += (int64_t)gridDim.x * kThreads) {
        const int64_t idx = base + threadIdx.x;
        const bool valid = idx < count;
        const uint64_t k = valid ? keys[idx] : 0;
        for (int p = 0; p < npass; ++p) {
            const int shift = lo + 8 * p;
            const unsigned mask = (1u << min(8, hi - shift)) - 1u;
            const unsigned d = digit_of(k, shift, mask);
            const unsigned d0 = __shfl_sync(0xffffffffu, d, 0);
            const unsigned vm = __ballot_sync(0xffffffffu, valid);
            if (__all_sync(0xffffffffu, !valid || d == d0)) {
                if ((threadIdx.x & 31) == 0 && vm) atomicAdd(&h[p][d0], (unsigned)__popc(vm));
            } else if (valid) {
                atomicAdd(&h[p][d], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * kRadix; i += kThreads) {
        const unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], (unsigned long long)c);
    }
}

// hist[pass][digit] -> exclusive prefix over digits, per pass: one block of
// kRadix threads per pass, a thread per digit.
__global__ void __launch_bounds__(kRadix) k_digit_offsets(unsigned long long* __restrict__ hist, int npass) {
    __shared__ unsigned long long wsum[kRadix / 32];
    const int p = blockIdx.x;
    if (p >= npass) return;
    unsigned long long* h = hist + (size_t)p * kRadix;
    const int d = threadIdx.x, lane = d & 31, w = d >> 5;
    const unsigned long long c = h[d];
    unsigned long long inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    unsigned long long before = 0;
    for (int q = 0; q < w; ++q) before += wsum[q];
    h[d] = before + inc - c;
}

__global__ void __launch_bounds__(kThreads, 4) k_onesweep(const uint64_t* __restrict__ in,
                                                          uint64_t* __restrict__ out, int64_t count,
                                                          int shift, int nbits,
                                                          const unsigned long long* __restrict__ goff,
                                                          unsigned long long* status,
                                                          unsigned* tile_ctr, int* err) {
    __shared__ uint64_t stage[kTile];
    __shared__ unsigned short rank_s[kTile];
    __shared__ unsigned short wcnt[kWarps][kRadix];
    __shared__ unsigned dstart[kRadix];
    __shared__ unsigned wsum[kWarps];
    __shared__ unsigned long long s_goff[kRadix];
    __shared__ int s_tile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned mask = (1u << nbits) - 1u;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int64_t tbase = (int64_t)tile * kTile;
    const int valid_in_tile = (int)min64((int64_t)kTile, count - tbase);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int p = k * kThreads + threadIdx.x;
        if (p < valid_in_tile) stage[p] = in[tbase + p];
    }
    __syncthreads();
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
    unsigned tot = 0;
    {
        const int d = threadIdx.x;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) {
            const unsigned c = wcnt[q][d];
            wcnt[q][d] = (unsigned short)tot;
            tot += c;
        }
    }
    // publish this tile's count of digit d and look back for the keys of
    // digit d in earlier tiles
    {
        const int d = threadIdx.x;
        unsigned long long* my = status + (size_t)tile * kRadix + d;
        unsigned long long excl = 0;
        if (tile == 0) {
            st_relaxed(my, kFlagPre | (unsigned long long)tot);
        } else {
            st_relaxed(my, kFlagAgg | (unsigned long long)tot);
            for (int p = tile - 1; p >= 0; --p) {
                unsigned long long v;
                if (!wait_published(status + (size_t)p * kRadix + d, v, kSpinLimit)) {
                    atomicOr(err, 4);
                    break;
                }
                excl += v & kValMask;
                if ((v >> 62) == 2) break;
            }
            st_relaxed(my, kFlagPre | (excl + tot));
        }
        s_goff[d] = goff[d] + excl;
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
            out[s_goff[d] + (uint64_t)(p - (int)dstart[d])] = kk;
        }
    }
}

}  // namespace

void radix_sort_u64(uint64_t** keys, uint64_t** alt, int64_t count, int lo, int hi, Alloc& al,
                    cudaStream_t st, int* err_dev) {
    if (count <= 1 || hi <= lo) return;
    const int64_t ntiles = (count + kTile - 1) / kTile;
    const int npass = (hi - lo + 7) / 8;
    // [hist: kMaxPasses x 256 u64][tile counters: kMaxPasses u32][error flag]
    Buf<unsigned long long> hist(al, (size_t)kMaxPasses * kRadix + 8);
    Buf<unsigned long long> status(al, (size_t)ntiles * kRadix);
    unsigned* ctrs = reinterpret_cast<unsigned*>(hist.get() + (size_t)kMaxPasses * kRadix);
    int* err = err_dev ? err_dev : reinterpret_cast<int*>(ctrs + kMaxPasses);
    TC_CUDA(cudaMemsetAsync(hist.get(), 0, sizeof(unsigned long long) * ((size_t)kMaxPasses * kRadix + 8), st));
    {
        Prof prof_("k_digit_hist", st);
        k_digit_hist<<<grid_for(count, kThreads, (int64_t)num_sms() * 8), kThreads, 0, st>>>(
            *keys, count, lo, npass, hi, hist.get());
    }
    TC_LAUNCH_CHECK();
    {
        Prof prof_("k_digit_offsets", st);
        k_digit_offsets<<<npass, kRadix, 0, st>>>(hist.get(), npass);
    }
    TC_LAUNCH_CHECK();
    for (int p = 0; p < npass; ++p) {
        const int shift = lo + 8 * p;
        const int nbits = min(8, hi - shift);
        TC_CUDA(cudaMemsetAsync(status.get(), 0, sizeof(unsigned long long) * (size_t)ntiles * kRadix, st));
        {
            Prof prof_("k_onesweep", st);
            k_onesweep<<<(unsigned)ntiles, kThreads, 0, st>>>(*keys, *alt, count, shift, nbits,
                                                              hist.get() + (size_t)p * kRadix,
                                                              status.get(), ctrs + p, err);
        }
        TC_LAUNCH_CHECK();
        uint64_t* t = *keys;
        *keys = *alt;
        *alt = t;
    }
    if (err_dev) return;   // the caller reads the flag at its next synchronisation
    int herr = 0;
    TC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (herr) TC_FAIL(TC_ETIMEOUT, "radix sort: a look-back wait ran past its bound");
}

}  // namespace tc

namespace tc {

bool selftest_wait_timeout(long limit, Alloc& al, cudaStream_t st) {
    Buf<unsigned long long> w(al, 2);   // [0] the word nothing publishes, [1] error flag
    TC_CUDA(cudaMemsetAsync(w.get(), 0, 2 * sizeof(unsigned long long), st));
    k_wait_selftest<<<1, 32, 0, st>>>(w.get(), limit, reinterpret_cast<int*>(w.get() + 1));
    TC_LAUNCH_CHECK();
    int err = 0;
    TC_CUDA(cudaMemcpyAsync(&err, w.get() + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    return (err & 4) != 0;
}

}  // namespace tc
