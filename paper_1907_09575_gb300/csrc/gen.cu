// Device RMAT input generator (synthetic inputs only; not the counting method).
//
// An independent implementation of the integer RMAT stream defined by the
// host generator: counter-based splitmix64 draws (Steele, Lea and Flood,
// OOPSLA 2014), one 32-bit half per recursion level against the cumulative
// a, a+b, a+b+c thresholds, a seeded bijective scramble x -> ((x*A mod 2^s)
// xor B) * C mod 2^s, and rejection of ids >= n (64 attempts, then the
// self-loop (0,0)).  Equal output for equal (seed, scale, n, pair index).
#include "common.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kTagPairs = 0x524D4154ull;  // "RMAT"
constexpr uint64_t kTagScramble = 0x5343524Dull;  // "SCRM"
constexpr int kAttempts = 64;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t ctr) {
    return mix64(key + (ctr + 1ull) * kGamma);
}

__global__ void k_rmat(uint64_t key, int scale, uint64_t n, int64_t e0, int64_t count,
                       uint32_t t1, uint32_t t2, uint32_t t3, uint64_t A, uint64_t B, uint64_t C,
                       int32_t* __restrict__ src, int32_t* __restrict__ dst) {
    const uint64_t mask = (1ull << scale) - 1ull;
    const uint64_t hpa = (uint64_t)((scale + 1) / 2);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = (uint64_t)(e0 + i);
        int32_t su = 0, sv = 0;
        for (int a = 0; a < kAttempts; ++a) {
            const uint64_t base = (e * kAttempts + (uint64_t)a) * hpa;
            uint64_t u = 0, v = 0, h = 0;
            for (int l = 0; l < scale; ++l) {
                if ((l & 1) == 0) h = draw(key, base + (uint64_t)(l >> 1));
                const uint32_t r = (l & 1) ? (uint32_t)(h >> 32) : (uint32_t)h;
                const uint64_t bu = (r >= t2) ? 1ull : 0ull;
                const uint64_t bv = (r >= t1 && r < t2) || (r >= t3) ? 1ull : 0ull;
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            u = ((((u * A) & mask) ^ B) * C) & mask;
            v = ((((v * A) & mask) ^ B) * C) & mask;
            if (u < n && v < n) {
                su = (int32_t)u;
                sv = (int32_t)v;
                break;
            }
        }
        src[i] = su;
        dst[i] = sv;
    }
}

// Many RMAT requests at once: pair x of the concatenation belongs to the
// request r with ppre[r] <= x < ppre[r+1]; its ids are offset by vpre[r].
__global__ void k_rmat_multi(const RmatJob* __restrict__ jobs, const int64_t* __restrict__ ppre,
                             int nreq, int64_t total, int32_t* __restrict__ src,
                             int32_t* __restrict__ dst) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nreq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ppre[mid] <= x) lo = mid; else hi = mid - 1;
        }
        const RmatJob& J = jobs[lo];
        const uint64_t e = (uint64_t)(x - ppre[lo]);
        const uint64_t mask = (1ull << J.scale) - 1ull;
        const uint64_t hpa = (uint64_t)((J.scale + 1) / 2);
        int64_t su = 0, sv = 0;
        for (int a = 0; a < kAttempts; ++a) {
            const uint64_t base = (e * kAttempts + (uint64_t)a) * hpa;
            uint64_t u = 0, v = 0, h = 0;
            for (int l = 0; l < J.scale; ++l) {
                if ((l & 1) == 0) h = draw(J.key, base + (uint64_t)(l >> 1));
                const uint32_t r = (l & 1) ? (uint32_t)(h >> 32) : (uint32_t)h;
                const uint64_t bu = (r >= J.t2) ? 1ull : 0ull;
                const uint64_t bv = (r >= J.t1 && r < J.t2) || (r >= J.t3) ? 1ull : 0ull;
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            u = ((((u * J.A) & mask) ^ J.B) * J.C) & mask;
            v = ((((v * J.A) & mask) ^ J.B) * J.C) & mask;
            if (u < (uint64_t)J.n && v < (uint64_t)J.n) {
                su = (int64_t)u;
                sv = (int64_t)v;
                break;
            }
        }
        src[x] = (int32_t)(J.vbase + su);
        dst[x] = (int32_t)(J.vbase + sv);
    }
}

}  // namespace

RmatJob make_rmat_job(uint64_t seed, int scale, int64_t n, uint32_t t1, uint32_t t2, uint32_t t3,
                      int64_t vbase) {
    RmatJob J;
    J.key = mix64(seed * kGamma + kTagPairs);
    const uint64_t ks = mix64(seed * kGamma + kTagScramble);
    const uint64_t mask = (1ull << scale) - 1ull;
    J.A = (draw(ks, 0) | 1ull) & mask;
    J.B = draw(ks, 1) & mask;
    J.C = (draw(ks, 2) | 1ull) & mask;
    J.n = n;
    J.vbase = vbase;
    J.scale = scale;
    J.t1 = t1;
    J.t2 = t2;
    J.t3 = t3;
    return J;
}

void generate_rmat_multi(const RmatJob* jobs_dev, const int64_t* ppre_dev, int nreq, int64_t total,
                         int32_t* src, int32_t* dst, cudaStream_t st) {
    if (total <= 0) return;
    {
        Prof prof_("k_rmat_multi", st);
        k_rmat_multi<<<grid_for(total, 256, (int64_t)num_sms() * 16), 256, 0, st>>>(
            jobs_dev, ppre_dev, nreq, total, src, dst);
    }
    TC_LAUNCH_CHECK();
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_generate_rmat(uint64_t seed, int32_t scale, int64_t n, int64_t e0,
                                      int64_t count, uint32_t t1, uint32_t t2, uint32_t t3,
                                      int32_t* src_dev, int32_t* dst_dev, void* stream) {
    clear_error();
    if (scale < 1 || scale > 31) {
        set_error("tc_generate_rmat: scale outside [1, 31]");
        return TC_EINVAL;
    }
    if (n < 1 || n > (1ll << scale) || e0 < 0 || count < 0 || (count > 0 && (!src_dev || !dst_dev))) {
        set_error("tc_generate_rmat: bad n, e0, count or output pointer");
        return TC_EINVAL;
    }
    if (!(t1 <= t2 && t2 <= t3)) {
        set_error("tc_generate_rmat: thresholds must be non-decreasing");
        return TC_EINVAL;
    }
    if (count == 0) return TC_OK;
    const uint64_t key = mix64(seed * kGamma + kTagPairs);
    const uint64_t ks = mix64(seed * kGamma + kTagScramble);
    const uint64_t mask = (1ull << scale) - 1ull;
    const uint64_t A = (draw(ks, 0) | 1ull) & mask;
    const uint64_t B = draw(ks, 1) & mask;
    const uint64_t C = (draw(ks, 2) | 1ull) & mask;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        Prof prof_("k_rmat", st);
        k_rmat<<<grid_for(count, 256, (int64_t)num_sms() * 16), 256, 0, st>>>(
        key, scale, (uint64_t)n, e0, count, t1, t2, t3, A, B, C, src_dev, dst_dev);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("tc_generate_rmat: launch failed: %s", cudaGetErrorString(e));
        return TC_ECUDA;
    }
    return TC_OK;
}
