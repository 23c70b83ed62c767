/*
 * CPU oracle for exact triangle counting -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline leg may load this library.  The product path never calls it and
 * shares no code with it.
 *
 * It is deliberately plain and single threaded: qsort, arrays, two-pointer
 * merges, uint64 counters.  It follows the paper step by step:
 *
 *   1. Simple undirected graph (Section 2; Section 6.1 converts every input
 *      to an undirected simple graph): drop self-loops, store each edge once
 *      as (min, max), sort, remove duplicates.
 *   2. Degrees d(v) = |Adj(v)| over that edge set (Section 2).
 *   3. Non-decreasing degree order (Section 3.1, Section 5.3 "Reorder
 *      vertices"): new label = rank under (degree, original id) ascending;
 *      the tie-break by id is our reading, the paper leaves it open.
 *   4. Upper triangular part U (Section 5.3 "Create the upper and the lower
 *      triangular portion"): edge {a,b} goes into the row of the endpoint
 *      with the smaller new label, so each edge appears once in U; rows are
 *      sorted ascending (Section 5.2, early-exit paragraph, requires sorted
 *      adjacency).
 *   5. Eq. 1 and Eq. 2: for every edge (i,j) of U, c_ij = sum_{k>j} u_ik u_jk,
 *      which is the size of the intersection of rows i and j of U (row j only
 *      holds labels > j); the total is the sum of c_ij.  The intersection is
 *      the list-based joint traversal of Section 3.1.  Each common k is one
 *      triangle {i,j,k}; it is also credited to t[i], t[j] and t[k].
 *   6. Per-vertex counts are mapped back to original labels.
 *
 * A second routine counts, for a few sampled vertices, the triangles through
 * each of them straight from the definition of a triangle (Section 2): the
 * number of edges among the vertex's neighbours.  It needs no relabelling and
 * is cheap for low-degree samples, so it can check full-size graphs.
 *
 * Planted mistakes for the mutation tests are compiled in only when
 * TC_ORACLE_MUTANT is defined (never in the oracle the tests trust).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef TC_ORACLE_MUTANT
#define TC_ORACLE_MUTANT 0
#endif

typedef struct {
    int64_t  m;            /* undirected simple edges = nnz(U) */
    int64_t  max_outdeg;   /* max |Adj>(v)| */
    int64_t  max_deg;      /* max d(v) */
    uint64_t wedges_ijk;   /* sum over (i,j) in U of |Adj>(j)| */
    uint64_t wedges_jik;   /* sum over i of C(|Adj>(i)|, 2) */
} tc_oracle_stats;

static int cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Step 1: canonical, sorted, duplicate-free edge keys (min << 32 | max).
 * Returns the number of edges, or -1 on an id outside [0, n). */
static int64_t simple_edges(const int32_t* src, const int32_t* dst, int64_t num_pairs,
                            int64_t n, uint64_t** out)
{
    uint64_t* key = (uint64_t*)malloc((size_t)(num_pairs > 0 ? num_pairs : 1) * sizeof(uint64_t));
    int64_t cnt = 0;
    for (int64_t e = 0; e < num_pairs; ++e) {
        int64_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n) { free(key); return -1; }
#if TC_ORACLE_MUTANT == 1
        /* planted: self-loops kept */
#else
        if (a == b) continue;
#endif
        int64_t lo = a < b ? a : b, hi = a < b ? b : a;
        key[cnt++] = ((uint64_t)lo << 32) | (uint64_t)hi;
    }
    qsort(key, (size_t)cnt, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (int64_t e = 0; e < cnt; ++e) {
#if TC_ORACLE_MUTANT == 2
        key[m++] = key[e];   /* planted: duplicates kept */
#else
        if (m == 0 || key[e] != key[m - 1]) key[m++] = key[e];
#endif
    }
    *out = key;
    return m;
}

/* Steps 1-6.  total receives the triangle count; per_vertex (n entries,
 * original labels) may be NULL.  Returns 0, or -1 on invalid input. */
int tc_oracle_count(const int32_t* src, const int32_t* dst, int64_t num_pairs, int64_t n,
                    uint64_t* total, uint64_t* per_vertex, tc_oracle_stats* stats)
{
    if (n < 0 || num_pairs < 0 || !total) return -1;
    uint64_t* E = NULL;
    int64_t m = simple_edges(src, dst, num_pairs, n, &E);
    if (m < 0) return -1;

    /* Step 2: degrees. */
    int64_t* deg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        deg[E[e] >> 32]++;
        deg[E[e] & 0xffffffffu]++;
    }

    /* Step 3: rank under (degree, id) ascending. */
    uint64_t* order = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
    for (int64_t v = 0; v < n; ++v) order[v] = ((uint64_t)deg[v] << 32) | (uint64_t)v;
    qsort(order, (size_t)n, sizeof(uint64_t), cmp_u64);
    int64_t* perm = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* inv = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t r = 0; r < n; ++r) {
        int64_t v = (int64_t)(order[r] & 0xffffffffu);
        perm[v] = r;
        inv[r] = v;
    }

    /* Step 4: U in CSR, rows sorted. */
    int64_t* off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = perm[E[e] >> 32], b = perm[E[e] & 0xffffffffu];
#if TC_ORACLE_MUTANT == 3
        /* planted: the literal degree comparison, which sends an edge between
         * equal-degree vertices to L from both sides, so it never reaches U */
        if (deg[E[e] >> 32] == deg[E[e] & 0xffffffffu]) continue;
#endif
        off[(a < b ? a : b) + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    int32_t* adj = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int64_t* fill = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) fill[v] = off[v];
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = perm[E[e] >> 32], b = perm[E[e] & 0xffffffffu];
#if TC_ORACLE_MUTANT == 3
        if (deg[E[e] >> 32] == deg[E[e] & 0xffffffffu]) continue;
#endif
        int64_t lo = a < b ? a : b, hi = a < b ? b : a;
        adj[fill[lo]++] = (int32_t)hi;
    }
    for (int64_t v = 0; v < n; ++v)
        qsort(adj + off[v], (size_t)(off[v + 1] - off[v]), sizeof(int32_t), cmp_i32);

    /* Step 5: Eq. 1 per edge of U by a joint traversal; Eq. 2 sums them. */
    uint64_t* t = (uint64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    uint64_t sum = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t q = off[i]; q < off[i + 1]; ++q) {
            int64_t j = adj[q];
            int64_t x = off[i], xe = off[i + 1];
#if TC_ORACLE_MUTANT == 5
            int64_t y = off[j] + 1, ye = off[j + 1];   /* planted: off by one */
#else
            int64_t y = off[j], ye = off[j + 1];
#endif
            uint64_t cij = 0;
            while (x < xe && y < ye) {
                if (adj[x] < adj[y]) ++x;
                else if (adj[x] > adj[y]) ++y;
                else {
                    int64_t k = adj[x];
                    ++cij;
#if TC_ORACLE_MUTANT == 4
                    /* planted: t[k] credit dropped */
                    (void)k;
#else
                    t[k]++;
#endif
                    ++x; ++y;
                }
            }
            sum += cij;
            t[i] += cij;
#if TC_ORACLE_MUTANT == 6
            (void)j;                                   /* planted: t[j] dropped */
#else
            t[j] += cij;
#endif
        }
    }
    *total = sum;

    /* Step 6: back to original labels. */
    if (per_vertex)
        for (int64_t v = 0; v < n; ++v) per_vertex[v] = t[perm[v]];

    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->m = m;
        for (int64_t v = 0; v < n; ++v) {
            int64_t dp = off[v + 1] - off[v];
            if (dp > stats->max_outdeg) stats->max_outdeg = dp;
            if (deg[v] > stats->max_deg) stats->max_deg = deg[v];
            stats->wedges_jik += (uint64_t)(dp * (dp - 1) / 2);
            for (int64_t q = off[v]; q < off[v + 1]; ++q)
                stats->wedges_ijk += (uint64_t)(off[adj[q] + 1] - off[adj[q]]);
        }
    }
    (void)inv;
    free(E); free(deg); free(order); free(perm); free(inv);
    free(off); free(adj); free(fill); free(t);
    return 0;
}

/* Triangles through each sampled vertex s, from the definition: the number of
 * distinct edges {a,b} of the simple graph with both a and b adjacent to s.
 * At most 64 samples.  Two scans of the raw pairs; memory grows with the
 * samples' neighbourhoods, so pick low-degree samples on huge graphs.
 * Returns 0, or -1 on invalid input. */

typedef struct { int64_t key; uint64_t mask; } slot_t;

static int64_t hash_find(const slot_t* tab, int64_t cap, int64_t k)
{
    uint64_t h = ((uint64_t)k * 0x9E3779B97F4A7C15ULL) >> 20;
    for (int64_t s = (int64_t)(h & (uint64_t)(cap - 1));; s = (s + 1) & (cap - 1))
        if (tab[s].key == k || tab[s].key == -1) return s;
}

int tc_oracle_vertex_triangles(const int32_t* src, const int32_t* dst, int64_t num_pairs,
                               int64_t n, const int32_t* samples, int64_t ns, uint64_t* out)
{
    if (ns < 0 || ns > 64 || n < 0 || num_pairs < 0) return -1;
    for (int64_t s = 0; s < ns; ++s)
        if (samples[s] < 0 || samples[s] >= n) return -1;
    /* which sampled vertices each vertex is: vertex -> bitmask of samples */
    slot_t who[256];
    for (int64_t q = 0; q < 256; ++q) who[q].key = -1;
    for (int64_t s = 0; s < ns; ++s) {
        int64_t p = hash_find(who, 256, samples[s]);
        if (who[p].key == -1) { who[p].key = samples[s]; who[p].mask = 0; }
        who[p].mask |= 1ULL << s;
    }
    /* scan 1: neighbour sets, kept as vertex -> bitmask of samples adjacent to it */
    int64_t cap = 1024, used = 0;
    slot_t* tab = (slot_t*)malloc((size_t)cap * sizeof(slot_t));
    for (int64_t s = 0; s < cap; ++s) tab[s].key = -1;
    for (int64_t e = 0; e < num_pairs; ++e) {
        int64_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n) { free(tab); return -1; }
        if (a == b) continue;
        int64_t pa = hash_find(who, 256, a), pb = hash_find(who, 256, b);
        uint64_t sa = who[pa].key == a ? who[pa].mask : 0;   /* samples equal to a */
        uint64_t sb = who[pb].key == b ? who[pb].mask : 0;
        if (!(sa | sb)) continue;
        for (int64_t s = 0; s < ns; ++s) {
            int64_t x = -1;
            if ((sa >> s) & 1ULL) x = b; else if ((sb >> s) & 1ULL) x = a;
            if (x < 0) continue;
            if (2 * (used + 1) > cap) {
                int64_t ncap = cap * 2;
                slot_t* nt = (slot_t*)malloc((size_t)ncap * sizeof(slot_t));
                for (int64_t q = 0; q < ncap; ++q) nt[q].key = -1;
                for (int64_t q = 0; q < cap; ++q)
                    if (tab[q].key != -1) {
                        int64_t p = hash_find(nt, ncap, tab[q].key);
                        nt[p] = tab[q];
                    }
                free(tab); tab = nt; cap = ncap;
            }
            int64_t p = hash_find(tab, cap, x);
            if (tab[p].key == -1) { tab[p].key = x; tab[p].mask = 0; ++used; }
            tab[p].mask |= 1ULL << s;
        }
    }
    /* scan 2: edges with both ends in a sample's neighbourhood */
    int64_t hcap = 1024, hcnt = 0;
    uint64_t* hits = (uint64_t*)malloc((size_t)hcap * sizeof(uint64_t));
    int32_t* hs = (int32_t*)malloc((size_t)hcap * sizeof(int32_t));
    for (int64_t e = 0; e < num_pairs; ++e) {
        int64_t a = src[e], b = dst[e];
        if (a == b) continue;
        int64_t pa = hash_find(tab, cap, a), pb = hash_find(tab, cap, b);
        if (tab[pa].key == -1 || tab[pb].key == -1) continue;
        uint64_t both = tab[pa].mask & tab[pb].mask;
        int64_t lo = a < b ? a : b, hi = a < b ? b : a;
        for (int64_t s = 0; s < ns; ++s) {
            if (!((both >> s) & 1ULL)) continue;
            if (hcnt == hcap) {
                hcap *= 2;
                hits = (uint64_t*)realloc(hits, (size_t)hcap * sizeof(uint64_t));
                hs = (int32_t*)realloc(hs, (size_t)hcap * sizeof(int32_t));
            }
            hits[hcnt] = ((uint64_t)lo << 32) | (uint64_t)hi;
            hs[hcnt] = (int32_t)s;
            ++hcnt;
        }
    }
    /* distinct edges per sample: sort (sample, edge) pairs */
    uint64_t* comb = (uint64_t*)malloc((size_t)(hcnt > 0 ? hcnt : 1) * 2 * sizeof(uint64_t));
    for (int64_t q = 0; q < hcnt; ++q) { comb[2 * q] = (uint64_t)hs[q]; comb[2 * q + 1] = hits[q]; }
    /* sort by sample, then edge: pack into an index order */
    int64_t* idx = (int64_t*)malloc((size_t)(hcnt > 0 ? hcnt : 1) * sizeof(int64_t));
    for (int64_t s = 0; s < ns; ++s) out[s] = 0;
    for (int64_t s = 0; s < ns; ++s) {
        int64_t c = 0;
        for (int64_t q = 0; q < hcnt; ++q)
            if ((int64_t)comb[2 * q] == s) idx[c++] = q;
        uint64_t* ks = (uint64_t*)malloc((size_t)(c > 0 ? c : 1) * sizeof(uint64_t));
        for (int64_t q = 0; q < c; ++q) ks[q] = comb[2 * idx[q] + 1];
        qsort(ks, (size_t)c, sizeof(uint64_t), cmp_u64);
        uint64_t d = 0;
        for (int64_t q = 0; q < c; ++q)
            if (q == 0 || ks[q] != ks[q - 1]) ++d;
        out[s] = d;
        free(ks);
    }
    free(idx); free(comb); free(hits); free(hs); free(tab);
    return 0;
}
