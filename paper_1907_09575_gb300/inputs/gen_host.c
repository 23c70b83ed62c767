/*
 * Seeded synthetic graph generators (host side).
 *
 * These produce the raw, directed, possibly duplicated pair lists that the
 * triangle counter ingests.  They hold none of the counting method's
 * arithmetic: no canonicalisation, ordering, orientation or intersection.
 * Both the CPU oracle and the GPU path are fed from here, so that the two
 * see the very same input bytes.
 *
 * Randomness is counter based: draw(key, ctr) is the splitmix64 finaliser
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014; constants as in Vigna's public-domain splitmix64.c) applied to
 * key + (ctr + 1) * golden-gamma.  Every pair is a pure function of
 * (seed, pair index), so generation parallelises without changing output and
 * an independent device implementation can reproduce it bit for bit.
 *
 * Graph models:
 *   RMAT (Chakrabarti, Zhan, Faloutsos 2004) with a/b/c/d given as 32-bit
 *     integer thresholds, no noise, a seeded bijective id scramble on
 *     [0, 2^scale) and rejection of ids >= n (at most 64 attempts, after which
 *     the pair is emitted as the self-loop (0,0), which ingestion drops).
 *   Chung-Lu: both endpoints drawn independently in proportion to integer
 *     weights given as an inclusive prefix-sum table (inverse CDF by binary
 *     search; the uniform in [0,total) is the high 64 bits of draw*total).
 *   G(n,p): Batagelj-Brandes geometric skipping over the lower triangle
 *     (host only: it takes a floating point logarithm).
 *
 * Compiled with -ffp-contract=off; the integer generators are exact on any
 * host.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t tcgen_key(uint64_t seed, uint64_t tag)
{
    return sm64_mix(seed * GAMMA + tag);
}

uint64_t tcgen_draw(uint64_t key, uint64_t ctr)
{
    return sm64_mix(key + (ctr + 1ULL) * GAMMA);
}

/* Stream tags: distinct sub-streams of one seed. */
#define TAG_RMAT_PAIRS 0x524D4154ULL   /* "RMAT" */
#define TAG_RMAT_SCRAM 0x5343524DULL   /* "SCRM" */
#define TAG_CL_PAIRS   0x43484C55ULL   /* "CHLU" */
#define TAG_GNP        0x474E5020ULL   /* "GNP " */

#define RMAT_MAX_ATTEMPTS 64

static inline uint64_t scramble(uint64_t x, uint64_t A, uint64_t B, uint64_t C,
                                uint64_t mask)
{
    x = (x * A) & mask;
    x ^= B;
    return (x * C) & mask;
}

/* Scramble parameters: A, C odd multipliers and B an xor mask, all reduced
 * mod 2^scale so that the map is a bijection on [0, 2^scale). */
void tcgen_rmat_scramble_params(uint64_t seed, int scale, uint64_t out[3])
{
    uint64_t k = tcgen_key(seed, TAG_RMAT_SCRAM);
    uint64_t mask = (scale >= 64) ? ~0ULL : ((1ULL << scale) - 1ULL);
    out[0] = (tcgen_draw(k, 0) | 1ULL) & mask;
    out[1] = tcgen_draw(k, 1) & mask;
    out[2] = (tcgen_draw(k, 2) | 1ULL) & mask;
    if (scale == 0) { out[0] = out[2] = 0; out[1] = 0; }
}

/* One RMAT pair.  t1 < t2 < t3 are the cumulative a, a+b, a+b+c thresholds
 * scaled to 2^32.  Level l consumes 32 bits: the low half of hash l/2 for
 * even l, the high half for odd l; the first level decides the top bit. */
static inline void rmat_one(uint64_t key, uint64_t e, int scale, uint64_t n,
                            uint32_t t1, uint32_t t2, uint32_t t3,
                            const uint64_t sp[3], int32_t* su, int32_t* sv)
{
    const uint64_t mask = (scale >= 64) ? ~0ULL : ((1ULL << scale) - 1ULL);
    const uint64_t hpa = (uint64_t)((scale + 1) / 2);
    for (int a = 0; a < RMAT_MAX_ATTEMPTS; ++a) {
        uint64_t base = (e * RMAT_MAX_ATTEMPTS + (uint64_t)a) * hpa;
        uint64_t u = 0, v = 0, h = 0;
        for (int l = 0; l < scale; ++l) {
            if ((l & 1) == 0) h = tcgen_draw(key, base + (uint64_t)(l >> 1));
            uint32_t r = (l & 1) ? (uint32_t)(h >> 32) : (uint32_t)h;
            uint64_t bu, bv;
            if (r < t1)      { bu = 0; bv = 0; }
            else if (r < t2) { bu = 0; bv = 1; }
            else if (r < t3) { bu = 1; bv = 0; }
            else             { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        u = scramble(u, sp[0], sp[1], sp[2], mask);
        v = scramble(v, sp[0], sp[1], sp[2], mask);
        if (u < n && v < n) { *su = (int32_t)u; *sv = (int32_t)v; return; }
    }
    *su = 0; *sv = 0;
}

/* Pairs [e0, e0+count) of the RMAT stream of (seed, scale, n). */
void tcgen_rmat(uint64_t seed, int scale, int64_t n, int64_t e0, int64_t count,
                uint32_t t1, uint32_t t2, uint32_t t3,
                int32_t* src, int32_t* dst)
{
    uint64_t key = tcgen_key(seed, TAG_RMAT_PAIRS);
    uint64_t sp[3];
    tcgen_rmat_scramble_params(seed, scale, sp);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i)
        rmat_one(key, (uint64_t)(e0 + i), scale, (uint64_t)n, t1, t2, t3, sp,
                 &src[i], &dst[i]);
}

static inline int64_t upper_bound_u64(const uint64_t* cum, int64_t n, uint64_t x)
{
    /* smallest i in [0,n) with cum[i] > x; cum is inclusive and cum[n-1] > x */
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (cum[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static inline uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* Pairs [e0, e0+count) of the Chung-Lu stream: endpoint 2e and 2e+1 draws. */
void tcgen_chung_lu(uint64_t seed, const uint64_t* cum, int64_t n,
                    int64_t e0, int64_t count, int32_t* src, int32_t* dst)
{
    uint64_t key = tcgen_key(seed, TAG_CL_PAIRS);
    uint64_t total = cum[n - 1];
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        uint64_t e = (uint64_t)(e0 + i);
        uint64_t xu = mulhi64(tcgen_draw(key, 2 * e), total);
        uint64_t xv = mulhi64(tcgen_draw(key, 2 * e + 1), total);
        src[i] = (int32_t)upper_bound_u64(cum, n, xu);
        dst[i] = (int32_t)upper_bound_u64(cum, n, xv);
    }
}

/* G(n,p) by geometric skipping.  Writes at most cap pairs and returns the
 * number the model produced (which may exceed cap: call again with a larger
 * buffer).  Uniforms are (53-bit draw + 1) * 2^-53, in (0, 1]. */
int64_t tcgen_gnp(uint64_t seed, int64_t n, double p, int32_t* src, int32_t* dst,
                  int64_t cap)
{
    if (n < 2 || p <= 0.0) return 0;
    uint64_t key = tcgen_key(seed, TAG_GNP);
    int64_t cnt = 0;
    if (p >= 1.0) {
        for (int64_t v = 1; v < n; ++v)
            for (int64_t w = 0; w < v; ++w) {
                if (cnt < cap) { src[cnt] = (int32_t)v; dst[cnt] = (int32_t)w; }
                ++cnt;
            }
        return cnt;
    }
    double lq = log(1.0 - p);
    int64_t v = 1, w = -1;
    uint64_t ctr = 0;
    while (v < n) {
        double r = (double)((tcgen_draw(key, ctr++) >> 11) + 1ULL) * 0x1.0p-53;
        w = w + 1 + (int64_t)floor(log(r) / lq);
        while (w >= v && v < n) { w -= v; ++v; }
        if (v < n) {
            if (cnt < cap) { src[cnt] = (int32_t)v; dst[cnt] = (int32_t)w; }
            ++cnt;
        }
    }
    return cnt;
}
