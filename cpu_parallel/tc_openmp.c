/*
 * Shared-memory parallel triangle counter (OpenMP) -- a CPU speed baseline
 * and a second CPU count, independent of both the oracle and the CUDA
 * library (it shares no code with either).
 *
 * It is the paper's shared-memory formulation (Section 3.1, Eq. 6 and
 * Eq. 7: the triangles are the sum of (U L) masked by U, with L = U^T),
 * enumerated in the <j,i,k> order the paper prefers: for every vertex j the
 * row U_j is put into a map once, and every i of column j of U (row j of L)
 * probes it with the part of U_i after j.  The map follows Section 5.2: a
 * direct-indexed table when the labels of U_j span fewer slots than the
 * table has (no collisions), otherwise an open-addressing table indexed by
 * the label AND (size - 1).  Probes outside [min U_j, max U_j] cannot hit
 * and are skipped (the early exit of Section 5.2).
 *
 * Preprocessing follows Section 5.3 with parallel LSD radix sorts: pairs ->
 * canonical keys (self-loops dropped) -> sorted, unique edges -> degrees ->
 * ranks in (degree, id) order -> oriented keys sorted into the CSR of U ->
 * L by a counting scatter.  All counts are uint64.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t m;          /* simple undirected edges */
    int64_t max_outdeg; /* max |U_v| */
    int64_t max_deg;
    int32_t threads;    /* OpenMP threads used */
    int32_t pad;
} tcp_stats;

static int ceil_log2(uint64_t x)
{
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

/* Stable LSD radix sort of keys on bits [lo, hi), 8 bits per pass; the
 * result ends in *a (buffers may be swapped).  Each thread takes a fixed
 * contiguous block of the input, so a pass is stable. */
static void radix_sort(uint64_t** a, uint64_t** b, int64_t count, int lo, int hi)
{
    if (count <= 1 || hi <= lo) return;
    const int T = omp_get_max_threads();
    int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * 256 * (size_t)T);
    for (int shift = lo; shift < hi; shift += 8) {
        const int bits = (hi - shift) < 8 ? (hi - shift) : 8;
        const uint64_t mask = (1ull << bits) - 1ull;
        const uint64_t* in = *a;
        uint64_t* out = *b;
        memset(hist, 0, sizeof(int64_t) * 256 * (size_t)T);
#pragma omp parallel num_threads(T)
        {
            const int t = omp_get_thread_num();
            const int64_t e0 = count * t / T, e1 = count * (t + 1) / T;
            int64_t* h = hist + 256 * (size_t)t;
            for (int64_t e = e0; e < e1; ++e) h[(in[e] >> shift) & mask]++;
#pragma omp barrier
#pragma omp single
            {
                int64_t run = 0;
                for (int d = 0; d < 256; ++d)
                    for (int u = 0; u < T; ++u) {
                        const int64_t c = hist[256 * (size_t)u + d];
                        hist[256 * (size_t)u + d] = run;
                        run += c;
                    }
            }
            for (int64_t e = e0; e < e1; ++e) out[h[(in[e] >> shift) & mask]++] = in[e];
        }
        uint64_t* t = *a;
        *a = *b;
        *b = t;
    }
    free(hist);
}

/* exclusive prefix sum of c[0..n) into off[0..n], in parallel blocks */
static void prefix_sum(const int64_t* c, int64_t* off, int64_t n)
{
    const int T = omp_get_max_threads();
    int64_t* part = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int64_t v0 = n * t / T, v1 = n * (t + 1) / T;
        int64_t s = 0;
        for (int64_t v = v0; v < v1; ++v) s += c[v];
        part[t + 1] = s;
#pragma omp barrier
#pragma omp single
        for (int u = 0; u < T; ++u) part[u + 1] += part[u];
        s = part[t];
        for (int64_t v = v0; v < v1; ++v) {
            off[v] = s;
            s += c[v];
        }
    }
    off[n] = part[T];
    free(part);
}

/*
 * tcp_count: the exact triangle count of the simple undirected graph whose
 * edges are the pairs (src[e], dst[e]) with self-loops and duplicates
 * dropped.  t (NULL or n entries) receives the triangles through each
 * original vertex.  threads <= 0 uses every OpenMP thread.  Returns 0, or
 * -1 for an id outside [0, n) or a negative size.
 */
int tcp_count(const int32_t* src, const int32_t* dst, int64_t num_pairs, int64_t n,
              int threads, uint64_t* total_out, uint64_t* t, tcp_stats* st)
{
    if (num_pairs < 0 || n < 0) return -1;
    if (threads > 0) omp_set_num_threads(threads);
    const int T = omp_get_max_threads();
    const int bits = ceil_log2((uint64_t)(n > 1 ? n : 2));
    int bad = 0;

    /* canonical keys, self-loops dropped: per-thread counts, then places */
    int64_t* cnt = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
    uint64_t* k1 = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(num_pairs > 0 ? num_pairs : 1));
    uint64_t* k2 = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(num_pairs > 0 ? num_pairs : 1));
#pragma omp parallel num_threads(T) reduction(| : bad)
    {
        const int tt = omp_get_thread_num();
        const int64_t e0 = num_pairs * tt / T, e1 = num_pairs * (tt + 1) / T;
        int64_t c = 0;
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t a = src[e], b = dst[e];
            if (a < 0 || a >= n || b < 0 || b >= n) bad = 1;
            else if (a != b) ++c;
        }
        cnt[tt + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int u = 0; u < T; ++u) cnt[u + 1] += cnt[u];
        int64_t p = cnt[tt];
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t a = src[e], b = dst[e];
            if (a < 0 || a >= n || b < 0 || b >= n || a == b) continue;
            const uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
            k1[p++] = (lo << bits) | hi;
        }
    }
    if (bad) {
        free(cnt); free(k1); free(k2);
        return -1;
    }
    const int64_t P = cnt[T];
    free(cnt);
    radix_sort(&k1, &k2, P, 0, 2 * bits);

    /* unique: keep the first of each run (compacted into k2) */
    int64_t* part = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
#pragma omp parallel num_threads(T)
    {
        const int tt = omp_get_thread_num();
        const int64_t e0 = P * tt / T, e1 = P * (tt + 1) / T;
        int64_t c = 0;
        for (int64_t e = e0; e < e1; ++e) c += (e == 0 || k1[e] != k1[e - 1]);
        part[tt + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int u = 0; u < T; ++u) part[u + 1] += part[u];
        int64_t p = part[tt];
        for (int64_t e = e0; e < e1; ++e)
            if (e == 0 || k1[e] != k1[e - 1]) k2[p++] = k1[e];
    }
    const int64_t m = part[T];
    free(part);
    uint64_t* E = k2;   /* m unique edges, sorted */
    const uint64_t mask = (1ull << bits) - 1ull;

    /* degrees, then ranks in (degree, id) order */
    int64_t* deg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        __atomic_fetch_add(&deg[E[e] >> bits], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&deg[E[e] & mask], 1, __ATOMIC_RELAXED);
    }
    int64_t maxdeg = 0;
#pragma omp parallel for reduction(max : maxdeg)
    for (int64_t v = 0; v < n; ++v) maxdeg = deg[v] > maxdeg ? deg[v] : maxdeg;
    const int dbits = ceil_log2((uint64_t)maxdeg + 1);
    uint64_t* dk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint64_t* da = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) dk[v] = ((uint64_t)deg[v] << bits) | (uint64_t)v;
    radix_sort(&dk, &da, n, bits, bits + dbits);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) rank[dk[r] & mask] = (int32_t)r;
    free(dk);
    free(da);
    free(deg);

    /* U: each edge from its lower to its higher rank, sorted by (row, col) */
    uint64_t* U = k1;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        const uint64_t a = (uint64_t)rank[E[e] >> bits], b = (uint64_t)rank[E[e] & mask];
        U[e] = ((a < b ? a : b) << bits) | (a < b ? b : a);
    }
    radix_sort(&U, &E, m, 0, 2 * bits);
    int64_t* rowc = (int64_t*)calloc((size_t)(n > 0 ? n : 1) + 1, sizeof(int64_t));
    int64_t* colc = (int64_t*)calloc((size_t)(n > 0 ? n : 1) + 1, sizeof(int64_t));
    int32_t* adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        adj[e] = (int32_t)(U[e] & mask);
        __atomic_fetch_add(&rowc[U[e] >> bits], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&colc[U[e] & mask], 1, __ATOMIC_RELAXED);
    }
    free(k1 == U ? k2 : k1);   /* the buffer not holding U */
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* loff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    prefix_sum(rowc, off, n);
    prefix_sum(colc, loff, n);
    free(U);

    /* L = U^T: for pivot j, the rows i with j in U_i and where U_i goes on */
    int64_t* fill = rowc;   /* reused as per-column cursors */
    memcpy(fill, loff, sizeof(int64_t) * (size_t)n);
    int32_t* li = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t* lp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t maxout = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(max : maxout)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t d = off[i + 1] - off[i];
        if (d > maxout) maxout = d;
        for (int64_t p = off[i]; p < off[i + 1]; ++p) {
            const int32_t j = adj[p];
            const int64_t s = __atomic_fetch_add(&fill[j], 1, __ATOMIC_RELAXED);
            li[s] = (int32_t)i;
            lp[s] = p + 1;   /* the part of U_i after j starts here */
        }
    }
    free(colc);

    /* count: <j,i,k> with a map of U_j per pivot */
    uint64_t* tnew = t ? (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t)) : NULL;
    int tbits = 1;
    while ((1ll << tbits) < 2 * (maxout > 1 ? maxout : 1)) ++tbits;
    const int64_t tsize = 1ll << tbits;
    uint64_t total = 0;
#pragma omp parallel num_threads(T) reduction(+ : total)
    {
        int32_t* key = (int32_t*)malloc(sizeof(int32_t) * (size_t)tsize);
        int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)tsize);
        for (int64_t s = 0; s < tsize; ++s) stamp[s] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = 0; j < n; ++j) {
            const int64_t rb = off[j], re = off[j + 1];
            if (rb == re || loff[j] == loff[j + 1]) continue;
            const int32_t lo = adj[rb], hi = adj[re - 1];
            const int direct = (int64_t)hi - lo < tsize;
            const uint64_t hmask = (uint64_t)tsize - 1;
            for (int64_t p = rb; p < re; ++p) {
                const int32_t k = adj[p];
                uint64_t s = direct ? (uint64_t)(k - lo) : ((uint64_t)k & hmask);
                if (!direct)
                    while (stamp[s] == j) s = (s + 1) & hmask;
                stamp[s] = j;
                key[s] = k;
            }
            uint64_t hj = 0;
            for (int64_t q = loff[j]; q < loff[j + 1]; ++q) {
                const int64_t i = li[q];
                const int64_t p1 = off[i + 1];
                uint64_t c = 0;
                for (int64_t p = lp[q]; p < p1; ++p) {
                    const int32_t k = adj[p];
                    if (k < lo || k > hi) continue;
                    uint64_t s = direct ? (uint64_t)(k - lo) : ((uint64_t)k & hmask);
                    int hit = 0;
                    if (direct) {
                        hit = stamp[s] == j;
                    } else {
                        while (stamp[s] == j) {
                            if (key[s] == k) { hit = 1; break; }
                            s = (s + 1) & hmask;
                        }
                    }
                    if (hit) {
                        ++c;
                        if (tnew) __atomic_fetch_add(&tnew[k], 1, __ATOMIC_RELAXED);
                    }
                }
                if (c) {
                    hj += c;
                    if (tnew) __atomic_fetch_add(&tnew[i], c, __ATOMIC_RELAXED);
                }
            }
            total += hj;
            if (tnew && hj) __atomic_fetch_add(&tnew[j], hj, __ATOMIC_RELAXED);
        }
        free(key);
        free(stamp);
    }
    if (t) {
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < n; ++v) t[v] = tnew[rank[v]];
        free(tnew);
    }
    *total_out = total;
    if (st) {
        st->m = m;
        st->max_outdeg = maxout;
        st->max_deg = maxdeg;
        st->threads = T;
    }
    free(li); free(lp); free(off); free(loff); free(adj); free(rowc); free(rank);
    return 0;
}
