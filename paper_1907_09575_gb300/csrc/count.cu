// tc_count: Eq. 1 / Eq. 2 by the paper's <j,i,k> map-based enumeration.
//
// For a pivot j the row U_j (the labels k > j adjacent to j) is put in a
// shared-memory table once; every task (i,j) of j -- an edge of U whose row
// U_i continues after j -- then probes the table with each entry of U_i
// after j.  Each hit k is one triangle {i, j, k} counted at edge (i, j)
// (Eq. 1 sums exactly the k > j with u_ik = u_jk = 1).
//
// Tables (Section 5.2, "Modifying the hashing routine for sparser vertices"):
// a bitmap over [min U_j, max U_j] when that label span fits (collision
// free); else, for slices of at most kTagMaxEntries entries, a tag table
// (one slot per label hash holding the rest of the hashed label and the
// entry's rank: one load decides a probe exactly); else buckets of 4 slots
// with bucket = k AND (buckets - 1) (tc_tuning.table_mode = 1 forces
// buckets everywhere).  A probe outside [min U_j, max U_j] cannot hit --
// the per-probe form of the early exit of Section 5.2: a bitmap lookup
// clamps it onto a guard bit that is always clear, a bucket lookup rejects
// it before reading the table, a tag lookup finds no equal tag.
//
// Work: units (graph, pivot, slice of U_j, range of tasks).  Pivots with
// |U_j| <= 64 become warp units (a private table per warp); larger ones CTA
// units (a shared table, slices of <= 4096 entries).  One persistent kernel
// pops CTA units first, heaviest pivots first, then warp units; units may
// come from many graphs at once (the batched form), each graph reached
// through a view table.
//
// Per-vertex counts (t[v] = triangles through v): a task's hits credit i once,
// per-entry hit counters credit k once per unit, j is credited once per unit.
#include <algorithm>

#include "common.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

#ifndef TC_TLOW32
#define TC_TLOW32 1            // per-task credit into 32-bit counters when they cannot overflow
#endif
#ifndef TC_LARGE_MINB
#define TC_LARGE_MINB 4        // CTAs per SM the CTA kernel's registers must allow
#endif

constexpr int kGrab = 4;          // warp units popped per queue access
constexpr int kEmpty = -1;
#ifndef TC_UNROLL
#define TC_UNROLL 4
#endif
constexpr int kUnroll = TC_UNROLL;   // independent loads in flight per lane
#ifndef TC_PV_BRANCHLESS
#define TC_PV_BRANCHLESS 1     // per-vertex bitmap probe: 1 computes the rank on every lane
#endif

// warp unit table region: 128 hash slots, or a 128-word bitmap (4095 labels
// and the guard bit)
// plus its 128 16-bit rank prefixes
constexpr int kSmallBitWords = 128;
constexpr int kSmallRegionWords = kSmallBitWords + kSmallBitWords / 2;
// CTA unit table region (32-bit words): hash slots <= 2 * slice <= 8192, or a
// bitmap of kBitWords words (kBitWords * 32 labels) plus 16-bit prefixes
#ifndef TC_REGION_WORDS
#define TC_REGION_WORDS 8192
#endif
constexpr int kRegionWords = TC_REGION_WORDS;
constexpr int kBitWords = (kRegionWords * 2 / 3) & ~31;
static_assert(kBitWords + kBitWords / 2 <= kRegionWords, "bitmap + prefix fit the region");

__device__ __forceinline__ int64_t shfl64(int64_t v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
}

__device__ __forceinline__ int warp_incl_scan_i32(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The rows a launch counts and where their tails sit: all rows at their
// place for a device-resident graph; for one tile of a host-resident graph
// the rows [i0, i1) of its row block, whose entries start `shift` entries
// into the tile's row buffer.
struct TaskWindow {
    int i0, i1;
    int64_t shift;
};

// *p += 1 in shared memory when h is set: one predicated reduction, no
// branch around it.  p must point into shared memory; when h is 0 the
// address is formed but never accessed, so it may lie outside the array.
__device__ __forceinline__ void add_if(unsigned* p, unsigned h) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t@q red.shared.add.u32 [%0], 1;\n\t}"
                 ::"r"(a), "r"(h) : "memory");
}

// bits [lo, hi) of a 32-bit mask, 0 <= lo <= hi <= 32
__device__ __forceinline__ unsigned bit_range(int lo, int hi) {
    const unsigned up = (hi >= 32) ? 0xffffffffu : ((1u << hi) - 1u);
    const unsigned dn = (lo >= 32) ? 0xffffffffu : ((1u << lo) - 1u);
    return up & ~dn;
}

// ---------------------------------------------------------------------------
// Tables for one pivot slice S = U_j[rb, re) (sorted labels lo..hi).
//
// Bitmap (the direct, collision-free case of Section 5.2): bit k - lo is set
// for k in S.  Membership is one shared load and a shift.  The rank of a hit
// among S -- its position in the slice, used to credit per-vertex counts --
// is the 16-bit prefix popcount of the words before it plus a popcount.
//
// Hash (labels too spread for a bitmap): 4-slot buckets, bucket = k AND
// (buckets - 1) (the paper's AND hash), overflow to the next bucket; the
// occupied slots of a bucket are a prefix, so an empty last slot ends a miss.
// Both return a counter index for per-vertex credit (rank or slot), or -1.
// A probe of -1 (a lane past the end of a tail) is a miss in every table:
// the bitmap clamps it onto the guard bit, the others fail the window test.
// ---------------------------------------------------------------------------
struct BitTab {
    const unsigned* bm;
    const unsigned short* pre;
    int lo, hi;
    // labels outside [lo, hi] are clamped onto bit hi - lo + 1, which the
    // table keeps clear: no range test, no branch
    __device__ __forceinline__ unsigned offset(int k) const {
        return min((unsigned)(k - lo), (unsigned)(hi - lo + 1));
    }
    template <bool PV>
    __device__ __forceinline__ int find(int k) const {
        const unsigned d = offset(k);
        const unsigned w = bm[d >> 5];
        if (!((w >> (d & 31)) & 1u)) return -1;
        if (!PV) return 0;
        return (int)pre[d >> 5] + __popc(w & ((1u << (d & 31)) - 1u));
    }
    __device__ __forceinline__ unsigned bit(int k) const {
        const unsigned d = offset(k);
        return (bm[d >> 5] >> (d & 31)) & 1u;
    }
    // membership and rank without a branch on the membership: the rank is
    // read for every probe (the guard bit's word has a prefix too), and only
    // the credit is predicated on the hit
    __device__ __forceinline__ void probe_credit(int k, unsigned* cnt, unsigned& mine) const {
        const unsigned d = offset(k);
        const unsigned w = bm[d >> 5];
        // bit d & 31 moved to the top: the sign is the hit, and the popc
        // counts the bits up to and including it
        const unsigned x = w << (~d & 31u);
        mine += x >> 31;
        const int r1 = (int)pre[d >> 5] + __popc(x);
        add_if(&cnt[r1 - 1], x >> 31);
    }
    // hit counters by rank (rank < slice <= 4096): one word each, so hits on
    // neighbouring entries never share an atomic's word
    __device__ __forceinline__ void credit(unsigned* cnt, int r) const { atomicAdd(&cnt[r], 1u); }
    __device__ __forceinline__ unsigned credited(const unsigned* cnt, int r) const { return cnt[r]; }
};

struct HashTab {
    const int* tab;
    unsigned bmask;
    int lo, hi;
    template <bool PV>
    __device__ __forceinline__ int find(int k) const {
        if ((unsigned)(k - lo) > (unsigned)(hi - lo)) return -1;
        unsigned b = (unsigned)k & bmask;
        while (true) {
            const int4 v = reinterpret_cast<const int4*>(tab)[b];
            if (v.x == k) return (int)(4 * b);
            if (v.y == k) return (int)(4 * b + 1);
            if (v.z == k) return (int)(4 * b + 2);
            if (v.w == k) return (int)(4 * b + 3);
            if (v.w == kEmpty) return -1;
            b = (b + 1) & bmask;
        }
    }
    __device__ __forceinline__ unsigned bit(int k) const { return find<false>(k) >= 0; }
    // hit counters by slot (up to twice the slice): 16 bits each, two a
    // word (a counter never exceeds the tasks of a unit, below 2^16 by the
    // unit size cap)
    __device__ __forceinline__ void credit(unsigned* cnt, int r) const {
        atomicAdd(&cnt[r >> 1], 1u << ((r & 1) << 4));
    }
    __device__ __forceinline__ unsigned credited(const unsigned* cnt, int r) const {
        return (cnt[r >> 1] >> ((r & 1) << 4)) & 0xffffu;
    }
};

// Tag table, for slices of at most kTagMaxEntries entries whose labels are
// too spread for the bitmap: p = k * kTagMul (mod 2^32) is a bijection of
// the label; its top b bits pick one of 2^b slots (per-vertex: about 8 an
// entry, 1024 to 8192; totals only: 8192, the whole table region) and the
// slot keeps the low 32 - b bits of p (the tag) with the entry's rank in
// the bits above, below bit 31, so one 32-bit load decides membership
// exactly and gives the rank.  A slot two entries map to holds kTagMulti;
// those entries go to a second table of 2048 slots (another multiplier,
// 21-bit tags) beside the hit counters, and an entry that collides there
// too is found by a binary search of the sorted slice.
constexpr int kTagMaxEntries = 1024;                 // ranks below 2^10 in the second table
constexpr int kTagSlots = 8192;                      // first table: at most 13 index bits
constexpr int kTagSlots2 = 2048, kTag2Shift = 21;    // second table: 11 index bits, 21 tag bits
constexpr unsigned kTag2Mask = (1u << kTag2Shift) - 1u;
static_assert(kTagMaxEntries <= (1 << (31 - kTag2Shift)), "ranks fit both tables below bit 31");
static_assert(kTagSlots <= kRegionWords, "the first table fills at most the region");
static_assert(kTagMaxEntries + kTagSlots2 <= kRegionWords / 2, "counters and second table share the counters' space");
#ifndef TC_TAG_SUB
#define TC_TAG_SUB 1024        // entries of a tag table; a longer slice is probed in sub-slices
#endif
constexpr int kTagSub = TC_TAG_SUB;
static_assert(kTagSub >= 1 && kTagSub <= kTagMaxEntries, "a sub-slice fits the tables");
constexpr unsigned kTagMul = 0x9E3779B1u, kTagMul2 = 0x85EBCA77u;
constexpr unsigned kTagEmpty = 0xffffffffu, kTagMulti = 0xfffffffeu;

struct TagTab {
    const unsigned* t1;        // 2^(32 - s1) words
    const unsigned* t2;        // kTagSlots2 words
    const int32_t* row;        // the sorted slice in device memory
    int dp;
    int s1;                    // tag bits of the first table
    unsigned m1;               // (1 << s1) - 1
    __device__ int slow(int k) const {
        const unsigned p = (unsigned)k * kTagMul2;
        const unsigned w = t2[p >> kTag2Shift];
        if (w != kTagMulti) return ((w & (0x80000000u | kTag2Mask)) == (p & kTag2Mask)) ? (int)(w >> kTag2Shift) : -1;
        int a = 0, b = dp;
        while (a < b) {
            const int c = (a + b) >> 1;
            if (__ldg(row + c) < k) a = c + 1; else b = c;
        }
        return (a < dp && __ldg(row + a) == k) ? a : -1;
    }
    template <bool PV>
    __device__ __forceinline__ int find(int k) const {
        const unsigned p = (unsigned)k * kTagMul;
        const unsigned w = t1[p >> s1];
        if (w == kTagMulti) return slow(k);
        return ((w & (0x80000000u | m1)) == (p & m1)) ? (int)(w >> s1) : -1;
    }
    __device__ __forceinline__ unsigned bit(int k) const { return find<false>(k) >= 0; }
    __device__ __forceinline__ void probe_credit(int k, unsigned* cnt, unsigned& mine) const {
        const unsigned p = (unsigned)k * kTagMul;
        const unsigned w = t1[p >> s1];
        unsigned h = (w & (0x80000000u | m1)) == (p & m1);
        int r = (int)(w >> s1);
        if (w == kTagMulti) {
            r = slow(k);
            h = r >= 0;
        }
        mine += h;
        add_if(&cnt[r], h);
    }
    __device__ __forceinline__ void credit(unsigned* cnt, int r) const { atomicAdd(&cnt[r], 1u); }
    __device__ __forceinline__ unsigned credited(const unsigned* cnt, int r) const { return cnt[r]; }
};

__device__ __forceinline__ void tag_insert2(unsigned* t2, int k, int q) {
    const unsigned p = (unsigned)k * kTagMul2;
    unsigned* s = t2 + (p >> kTag2Shift);
    if (atomicCAS(s, kTagEmpty, ((unsigned)q << kTag2Shift) | (p & kTag2Mask)) != kTagEmpty) atomicExch(s, kTagMulti);
}

// Search (the list-based joint traversal of Section 3.1, lane-parallel): the
// sorted pivot row U_j (at most 64 entries) sits in shared memory and each
// lane places its probe in it by a branchless binary search.  No table is
// built; the position found is the entry's index, so per-vertex credit
// needs no rank.
struct SearchTab {
    const int* piv;
    int dp, lo, hi;
    template <bool PV>
    __device__ __forceinline__ int find(int k) const {
        if ((unsigned)(k - lo) > (unsigned)(hi - lo)) return -1;
        int pos = 0;
#pragma unroll
        for (int step = 32; step > 0; step >>= 1)
            if (pos + step < dp && piv[pos + step] <= k) pos += step;
        return piv[pos] == k ? pos : -1;
    }
    __device__ __forceinline__ unsigned bit(int k) const { return find<false>(k) >= 0; }
    __device__ __forceinline__ void credit(unsigned* cnt, int r) const { atomicAdd(&cnt[r], 1u); }
    __device__ __forceinline__ unsigned credited(const unsigned* cnt, int r) const { return cnt[r]; }
};

__device__ __forceinline__ void hash_insert(int* tab, unsigned bmask, int k) {
    unsigned b = (unsigned)k & bmask;
    while (true) {
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (atomicCAS(&tab[4 * b + w], kEmpty, k) == kEmpty) return;
        b = (b + 1) & bmask;
    }
}

__device__ __forceinline__ unsigned hash_buckets(int dp) {
    unsigned b = 1;
    while (4 * b < 2u * (unsigned)dp) b <<= 1;   // load factor <= 1/2
    return b;
}


template <class Tab>
struct has_probe_credit {
    template <class U>
    static constexpr bool check(decltype(&U::probe_credit)) { return true; }
    template <class U>
    static constexpr bool check(...) { return false; }
    static constexpr bool value = check<Tab>(nullptr);
};

template <bool PV, class Tab>
__device__ __forceinline__ void probe_one(const Tab& T, int k, unsigned* cnt, unsigned& mine) {
    if constexpr (!PV) {
        mine += T.bit(k);
    } else if constexpr (TC_PV_BRANCHLESS && has_probe_credit<Tab>::value) {
        T.probe_credit(k, cnt, mine);
    } else {
        const int r = T.template find<PV>(k);
        if (r >= 0) {
            ++mine;
            T.credit(cnt, r);
        }
    }
}

// ---------------------------------------------------------------------------
// One warp walks one long tail (>= 32 entries with per-vertex counts, >= 64
// for totals only) adj[st, st+L): lane q of a
// step reads entry q, kUnroll steps a round.  Returns the task's hits (the
// same in all lanes) with per-vertex counts, else 0.
//
// Per-vertex: the next round's entries are loaded before this round is
// probed, so a tail of up to 2 * 32 * kUnroll entries waits on memory about
// once.  Totals only: unchecked full rounds, then a checked last one -- the
// lighter probe leaves no latency worth the extra registers to hide.
// ---------------------------------------------------------------------------
template <bool PV, class Tab>
__device__ __forceinline__ unsigned warp_walk_tail(int64_t st, int L, const int32_t* __restrict__ adj,
                                                   const Tab& T, unsigned* cnt, uint64_t& hits) {
    const int lane = threadIdx.x & 31;
    const int32_t* __restrict__ p = adj + st + lane;
    unsigned mine = 0;
    if constexpr (PV) {
        int k[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) k[u] = (32 * u + lane < L) ? __ldg(p + 32 * u) : -1;
        for (int q0 = 0; q0 < L; q0 += 32 * kUnroll) {
            const int q1 = q0 + 32 * kUnroll;
            int kn[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) kn[u] = (q1 + 32 * u + lane < L) ? __ldg(p + q1 + 32 * u) : -1;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) probe_one<PV>(T, k[u], cnt, mine);   // -1: a miss
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) k[u] = kn[u];
        }
        hits += mine;
        return __reduce_add_sync(0xffffffffu, mine);
    } else {
        int q0 = 0;
        for (; q0 + 32 * kUnroll <= L; q0 += 32 * kUnroll) {
            int k[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) k[u] = __ldg(p + q0 + 32 * u);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) probe_one<PV>(T, k[u], cnt, mine);
        }
        if (q0 < L) {
            int k[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int q = q0 + 32 * u + lane;
                k[u] = (q < L) ? __ldg(p + q0 + 32 * u) : -1;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) probe_one<PV>(T, k[u], cnt, mine);   // -1: a miss
        }
        hits += mine;
        return 0;
    }
}

// A task's hits (i's share of its triangles, at most C(|U_i|, 2)): into the
// 32-bit counters tlow when the caller provides them (the largest row keeps
// that share below 2^32; half the bytes of the 64-bit accumulator, so more
// of the scattered atomics stay in L2), else into tnew.
__device__ __forceinline__ void credit_task(unsigned long long* tnew, unsigned* tlow, int i, unsigned c) {
    if (tlow)
        atomicAdd(&tlow[i], c);
    else
        atomicAdd(&tnew[i], (unsigned long long)c);
}

// ---------------------------------------------------------------------------
// One warp takes up to 32 tasks [tb, min(tb+32, t1)).
//
// Long tails (>= kShort entries) are either walked right away (defer == null) or
// appended to the CTA's queue of long tasks (their index relative to t0), to
// be shared out one task per warp later.  Short tails are concatenated: lane
// q of a step reads entry q of the concatenation; its owner is the number of
// short tasks starting at or before the step's first position, plus those
// starting inside the step before q (a ballot and a warp OR-reduce), minus
// one; the short tasks' start - prefix are compacted into s_base by rank, so
// the address is s_base[owner] + q.
// PV: lane s keeps the hit ballot of step s (a group's short tails total at
// most 31 * 32 entries, so 31 steps); a short task, which spans at most two
// steps, takes its hits from their popcounts over its positions at the end.
// Each task's hits go once to tnew[i]; per-entry hits to the counters cnt.
// ---------------------------------------------------------------------------
template <bool PV, bool WIN, class Tab>
__device__ __forceinline__ void warp_probe_group(const Task* __restrict__ tasks, int64_t tb, int64_t t1,
                                                 const int32_t* __restrict__ adj, const Tab& T,
                                                 unsigned* cnt, unsigned long long* tnew, unsigned* tlow,
                                                 int64_t* s_base, int64_t t0, unsigned short* defer,
                                                 int* ndefer, uint64_t& hits, uint64_t& probes,
                                                 const TaskWindow& win) {
    const int lane = threadIdx.x & 31;
    const int64_t t = tb + lane;
    const bool valid = t < t1;
    int64_t start = 0;
    int len = 0, i = 0;
    if (valid) {
        const Task tk = tasks[t];
        start = tk.start;
        len = tk.len;
        i = tk.i;
        if (WIN) {
            // a tile of a host-resident graph: rows outside its block wait
            // for another tile; tails are read from the tile's row buffer
            if (i < win.i0 || i >= win.i1) len = 0;
            start -= win.shift;
        }
    }
    unsigned c = 0;
    const unsigned le = (2u << lane) - 1u;   // bits 0..lane

    // long tails
    // tails shorter than kShort are concatenated across the lanes: 32 with
    // per-vertex counts (a short task then spans at most two steps), 64
    // for totals only (measured: the per-vertex short path costs more per
    // step than the longer walk of tails of 32-63 entries)
    constexpr int kShort = PV ? 32 : 64;
    const bool lg = valid && len >= kShort;
    unsigned longm = __ballot_sync(0xffffffffu, lg);
    if (defer) {
        if (longm) {
            int slot = 0;
            if (lane == 0) slot = atomicAdd(ndefer, __popc(longm));
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (lg) defer[slot + __popc(longm & (le >> 1))] = (unsigned short)(t - t0);
        }
    } else {
        while (longm) {
            const int o = __ffs(longm) - 1;
            longm &= longm - 1;
            const int64_t st = shfl64(start, o);
            const int L = __shfl_sync(0xffffffffu, len, o);
            probes += (uint64_t)L;
            const unsigned ch = warp_walk_tail<PV>(st, L, adj, T, cnt, hits);
            if (PV && lane == o) c += ch;
        }
    }

    // short tails, concatenated
    const int slen = (valid && len < kShort) ? len : 0;
    const int incl = warp_incl_scan_i32(slen);
    const int excl = incl - slen;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const bool sv = slen > 0;
    const unsigned shortm = __ballot_sync(0xffffffffu, sv);
    if (sv) s_base[__popc(shortm & (le >> 1))] = start - excl;
    __syncwarp();
    probes += (uint64_t)total;
    unsigned step_hits = 0;   // PV: the hit ballot of step `lane`
    for (int q0 = 0; q0 < total; q0 += 32 * kUnroll) {
        int k[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int qb = q0 + 32 * u;
            const unsigned before = __ballot_sync(0xffffffffu, sv && excl <= qb);
            const int d = excl - qb;
            const unsigned head = (sv && d > 0 && d < 32) ? (1u << d) : 0u;
            const unsigned M = __reduce_or_sync(0xffffffffu, head);
            const int o = __popc(before) - 1 + __popc(M & le);
            const int q = qb + lane;
            k[u] = (q < total) ? __ldg(&adj[s_base[o] + q]) : -1;
        }
        int r[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) r[u] = T.template find<PV>(k[u]);   // -1 (past the end): a miss
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const bool hit = r[u] >= 0;
            hits += hit ? 1 : 0;
            if (PV) {
                const unsigned hm = __ballot_sync(0xffffffffu, hit);
                if (lane == (q0 >> 5) + u) step_hits = hm;
                if (hit) T.credit(cnt, r[u]);
            }
        }
    }
    if (PV && total > 0) {
        const int s0 = excl >> 5, b0 = excl & 31;
        const unsigned h0 = __shfl_sync(0xffffffffu, step_hits, s0);
        const unsigned h1 = __shfl_sync(0xffffffffu, step_hits, (s0 + 1) & 31);
        if (sv) {
            c += __popc(h0 & bit_range(b0, min(b0 + slen, 32)));
            if (b0 + slen > 32) c += __popc(h1 & bit_range(0, b0 + slen - 32));
        }
    }
    __syncwarp();   // s_base is rewritten by the warp's next group
    if (PV && valid && c) credit_task(tnew, tlow, i, c);
}

__device__ __forceinline__ int64_t off_at(const GraphView& G, int64_t v) {
    return G.off64 ? static_cast<const int64_t*>(G.off)[v]
                   : (int64_t) static_cast<const int32_t*>(G.off)[v];
}

// Per-warp running total of hits bound for one counter (a graph's total, or
// a component's total), flushed when the warp moves to a unit whose hits go
// elsewhere (and at the end).  Every triangle found at pivot j lies in j's
// component, so the pivot decides the counter.
__device__ __forceinline__ unsigned long long* unit_target(const GraphView& G, const Unit& U) {
    return G.comp ? G.comp_totals + G.comp[U.j] : G.total;
}

struct GraphAcc {
    unsigned long long* target = nullptr;
    uint64_t hits = 0;
    __device__ __forceinline__ void to(unsigned long long* t) {
        if (t == target) return;
        flush();
        target = t;
    }
    __device__ __forceinline__ void flush() {
        const uint64_t s = warp_sum_u64(hits);
        if ((threadIdx.x & 31) == 0 && target && s) atomicAdd(target, (unsigned long long)s);
        hits = 0;
    }
};

// ---------------------------------------------------------------------------
// Warp unit: a pivot with |U_j| <= 64 processed by one warp with a private
// table (a bitmap of <= 4095 labels, or 128 hash slots).
// ---------------------------------------------------------------------------
template <bool PV, bool MERGE, bool WIN>
__device__ __forceinline__ void warp_unit(const GraphView& G, const Unit& U, unsigned* region,
                                          unsigned* cnt, int64_t* s_base, bool hash_only, int merge_max,
                                          unsigned* tlow, uint64_t& hits, uint64_t& probes, uint64_t& staged) {
    const int lane = threadIdx.x & 31;
    const int64_t rb = off_at(G, U.j), re = off_at(G, U.j + 1);
    const int dp = (int)(re - rb);
    const int lo = G.adj[rb], hi = G.adj[re - 1];
    const int mine = (lane < dp) ? G.adj[rb + lane] : 0;
    const int mine2 = (lane + 32 < dp) ? G.adj[rb + 32 + lane] : 0;
    const bool bitmap = !hash_only && (int64_t)hi - lo + 1 < 32 * kSmallBitWords;   // labels + guard bit
    uint64_t uh = 0;
    if (PV)
        for (int s = lane; s < kSmallTable / 2; s += 32) cnt[s] = 0;
    if (MERGE && dp <= merge_max) {
        int* piv = reinterpret_cast<int*>(region);
        if (lane < dp) piv[lane] = mine;
        if (lane + 32 < dp) piv[lane + 32] = mine2;
        __syncwarp();
        const SearchTab T{piv, dp, lo, hi};
        for (int64_t tb = U.t0; tb < U.t1; tb += 32)
            warp_probe_group<PV, WIN>(G.tasks, tb, U.t1, G.adj, T, cnt, G.tnew, tlow, s_base, U.t0, nullptr,
                                      nullptr, uh, probes, TaskWindow{G.i0, G.i1, G.tail_shift});
        __syncwarp();
        if (PV) {
            if (lane < dp) {
                const unsigned h = T.credited(cnt, lane);
                if (h) atomicAdd(&G.tnew[mine], (unsigned long long)h);
            }
            if (lane + 32 < dp) {
                const unsigned h = T.credited(cnt, lane + 32);
                if (h) atomicAdd(&G.tnew[mine2], (unsigned long long)h);
            }
        }
    } else if (bitmap) {
        const int words = ((hi - lo + 1) >> 5) + 1;
        for (int s = lane; s < words; s += 32) region[s] = 0;
        __syncwarp();
        if (lane < dp) atomicOr(&region[(mine - lo) >> 5], 1u << ((mine - lo) & 31));
        if (lane + 32 < dp) atomicOr(&region[(mine2 - lo) >> 5], 1u << ((mine2 - lo) & 31));
        __syncwarp();
        unsigned short* pre = reinterpret_cast<unsigned short*>(region + kSmallBitWords);
        if (PV) {
            // prefix popcounts of the (at most 128) words, 4 per lane
            int a[4], sum = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int wi = lane * 4 + q;
                a[q] = (wi < words) ? __popc(region[wi]) : 0;
                sum += a[q];
            }
            int run = warp_incl_scan_i32(sum) - sum;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int wi = lane * 4 + q;
                if (wi < words) pre[wi] = (unsigned short)run;
                run += a[q];
            }
        }
        __syncwarp();
        const BitTab T{region, pre, lo, hi};
        for (int64_t tb = U.t0; tb < U.t1; tb += 32)
            warp_probe_group<PV, WIN>(G.tasks, tb, U.t1, G.adj, T, cnt, G.tnew, tlow, s_base, U.t0, nullptr,
                                      nullptr, uh, probes, TaskWindow{G.i0, G.i1, G.tail_shift});
        __syncwarp();
        if (PV) {
            if (lane < dp) {
                const unsigned h = T.credited(cnt, lane);
                if (h) atomicAdd(&G.tnew[mine], (unsigned long long)h);
            }
            if (lane + 32 < dp) {
                const unsigned h = T.credited(cnt, lane + 32);
                if (h) atomicAdd(&G.tnew[mine2], (unsigned long long)h);
            }
        }
    } else {
        int* tab = reinterpret_cast<int*>(region);
        const unsigned bmask = hash_buckets(dp) - 1u;
        for (int s = lane; s < kSmallTable; s += 32) tab[s] = kEmpty;
        __syncwarp();
        if (lane < dp) hash_insert(tab, bmask, mine);
        if (lane + 32 < dp) hash_insert(tab, bmask, mine2);
        __syncwarp();
        const HashTab T{tab, bmask, lo, hi};
        for (int64_t tb = U.t0; tb < U.t1; tb += 32)
            warp_probe_group<PV, WIN>(G.tasks, tb, U.t1, G.adj, T, cnt, G.tnew, tlow, s_base, U.t0, nullptr,
                                      nullptr, uh, probes, TaskWindow{G.i0, G.i1, G.tail_shift});
        __syncwarp();
        if (PV)
            for (int s = lane; s < kSmallTable; s += 32) {
                const unsigned h = T.credited(cnt, s);
                if (h) atomicAdd(&G.tnew[tab[s]], (unsigned long long)h);
            }
    }
    staged += (uint64_t)dp;
    hits += uh;
    if (PV) {
        uh = warp_sum_u64(uh);
        if (lane == 0 && uh) atomicAdd(&G.tnew[G.jbase + U.j], (unsigned long long)uh);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// CTA unit: a slice of a larger pivot with its table shared by the CTA.
// Phase A: warps take groups of 32 tasks from a shared counter, probe the
// short tails and queue the long ones; phase B: warps pop one long task at a
// time, with later tasks' records already loading and the next tail
// prefetched into L2 while the current tail is walked.
// ---------------------------------------------------------------------------
template <bool PV, bool WIN, class Tab>
__device__ __forceinline__ void cta_probe_unit(const GraphView& G, const Unit& U, const Tab& T,
                                               unsigned* cnt, int* s_ctl, int64_t* s_base,
                                               unsigned short* s_long, unsigned* tlow, uint64_t& uh,
                                               uint64_t& probes) {
    // s_ctl: [0] next group, [1] deferred long tasks, [2] next long task
    const int lane = threadIdx.x & 31;
    const Task* __restrict__ tasks = G.tasks;
    const int32_t* __restrict__ adj = G.adj;
    while (true) {
        int g = 0;
        if (lane == 0) g = atomicAdd(&s_ctl[0], 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        const int64_t tb = U.t0 + (int64_t)g * 32;
        if (tb >= U.t1) break;
        warp_probe_group<PV, WIN>(tasks, tb, U.t1, adj, T, cnt, G.tnew, tlow, s_base, U.t0, s_long,
                                  &s_ctl[1], uh, probes, TaskWindow{G.i0, G.i1, G.tail_shift});
    }
    __syncthreads();
    const int nlong = s_ctl[1];
    auto pop = [&]() {
        int v = 0;
        if (lane == 0) v = atomicAdd(&s_ctl[2], 1);
        return __shfl_sync(0xffffffffu, v, 0);
    };
    // deferred tasks passed the window in phase A; only their tails move
    const int64_t shift = WIN ? G.tail_shift : 0;
    auto record = [&](int x) {
        Task t;
        t.len = 0;
        if (x < nlong) {
            t = tasks[U.t0 + s_long[x]];
            t.start -= shift;
        }
        return t;
    };
    // the next task's tail is prefetched into L2 while this one is walked
    auto prefetch_tail = [&](const Task& t) {
        if (32 * lane < t.len) asm volatile("prefetch.global.L2 [%0];" ::"l"(adj + t.start + 32 * lane));
    };
    if constexpr (!PV) {
        // records two tasks ahead: the record load of task x+2 overlaps the
        // walk of task x, and the prefetch of x+1's tail waits on nothing
        int x = pop(), x1 = pop();
        Task cur = record(x), nxt = record(x1);
        while (x < nlong) {
            const int x2 = pop();
            const Task nn = record(x2);
            prefetch_tail(nxt);
            probes += (uint64_t)cur.len;
            warp_walk_tail<PV>(cur.start, cur.len, adj, T, cnt, uh);
            x = x1;
            x1 = x2;
            cur = nxt;
            nxt = nn;
        }
    } else {
        // one task ahead (a third record would spill the per-vertex kernel;
        // written out, as the helpers above cost it registers too)
        int x = pop();
        Task cur;
        cur.len = 0;
        if (x < nlong) {
            cur = tasks[U.t0 + s_long[x]];
            cur.start -= shift;
        }
        while (x < nlong) {
            const int xn = pop();
            Task nxt;
            nxt.len = 0;
            if (xn < nlong) {
                nxt = tasks[U.t0 + s_long[xn]];
                nxt.start -= shift;
                if (32 * lane < nxt.len)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(adj + nxt.start + 32 * lane));
            }
            probes += (uint64_t)cur.len;
            const unsigned ch = warp_walk_tail<PV>(cur.start, cur.len, adj, T, cnt, uh);
            if (lane == 0 && ch) credit_task(G.tnew, tlow, cur.i, ch);
            x = xn;
            cur = nxt;
        }
    }
}

// BUCKETS: the instance for tc_tuning.table_mode = 1, every slice in
// 4-slot buckets; otherwise a bitmap when the slice's label span fits, else
// tag tables.  The two are separate instances because the bucket code,
// compiled into the default kernel, slowed its bitmap walk (2 %).
template <bool PV, bool WIN, bool BUCKETS>
__device__ __forceinline__ void cta_unit(const GraphView& G, const Unit& U, int slice_max,
                                         unsigned* region, unsigned* cnt, int* s_ctl,
                                         int64_t* s_base, unsigned short* s_long,
                                         unsigned* s_wsum, unsigned* tlow, uint64_t& hits, uint64_t& probes) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t rb = off_at(G, U.j) + (int64_t)U.slice * slice_max;
    const int64_t re = min64(off_at(G, U.j + 1), rb + slice_max);
    const int dp = (int)(re - rb);
    const int lo = G.adj[rb], hi = G.adj[re - 1];
    const bool bitmap = !BUCKETS && (int64_t)hi - lo + 1 < 32ll * kBitWords;   // labels + guard bit
    uint64_t uh = 0;
    // counters: by rank (< dp) for bitmaps and tag tables, by 16-bit slot
    // for buckets
    if (PV)
        for (int s = threadIdx.x; s < (BUCKETS ? kRegionWords / 2 : dp); s += blockDim.x) cnt[s] = 0;
    if (bitmap) {
        const int words = ((hi - lo + 1) >> 5) + 1;
        for (int s = threadIdx.x; s < words; s += blockDim.x) region[s] = 0;
        __syncthreads();
        for (int q = threadIdx.x; q < dp; q += blockDim.x) {
            const int k = G.adj[rb + q] - lo;
            atomicOr(&region[k >> 5], 1u << (k & 31));
        }
        __syncthreads();
        unsigned short* pre = reinterpret_cast<unsigned short*>(region + kBitWords);
        if (PV) {
            // prefix popcounts over the words: each thread a contiguous run
            const int per = (words + blockDim.x - 1) / blockDim.x;
            const int w0 = threadIdx.x * per;
            int sum = 0;
            for (int q = 0; q < per; ++q)
                if (w0 + q < words) sum += __popc(region[w0 + q]);
            const int inc = warp_incl_scan_i32(sum);
            if (lane == 31) s_wsum[w] = (unsigned)inc;
            __syncthreads();
            int before = 0;
            for (int q = 0; q < w; ++q) before += (int)s_wsum[q];
            int run = before + inc - sum;
            for (int q = 0; q < per; ++q)
                if (w0 + q < words) {
                    pre[w0 + q] = (unsigned short)run;
                    run += __popc(region[w0 + q]);
                }
            __syncthreads();
        }
        const BitTab T{region, pre, lo, hi};
        cta_probe_unit<PV, WIN>(G, U, T, cnt, s_ctl, s_base, s_long, tlow, uh, probes);
        __syncthreads();
        if (PV)
            for (int r = threadIdx.x; r < dp; r += blockDim.x) {
                const unsigned h = T.credited(cnt, r);
                if (h) atomicAdd(&G.tnew[G.adj[rb + r]], (unsigned long long)h);
            }
    } else if (!BUCKETS) {
        // tag tables over sub-slices of at most kTagMaxEntries entries, the
        // unit's tasks probing each in turn (a slice that long and that
        // spread is rare: none in RMAT scale 26)
        for (int sb = 0; sb < dp; sb += kTagSub) {
            const int sd = min(dp - sb, kTagSub);
            const int64_t sr = rb + sb;
            // the second table sits past the counters the slice can use (for
            // totals only, where the counters are); a barrier first, as the
            // counters were just cleared (or the last pass just read them)
            unsigned* t2 = cnt + (PV ? kTagMaxEntries : 0);
            __syncthreads();
            if (sb > 0) {
                if (threadIdx.x == 0) {
                    s_ctl[0] = 0;
                    s_ctl[1] = 0;
                    s_ctl[2] = 0;
                }
                if (PV)
                    for (int s = threadIdx.x; s < kTagMaxEntries; s += blockDim.x) cnt[s] = 0;
            }
            // index bits: with per-vertex counts 2^b1 >= 8 * sd, 10..13 (the
            // rank then fits below bit 31; less to clear a unit), for totals
            // only 13 (fewer shared slots: measured faster each way)
            int b1 = PV ? 10 : 13;
            while (b1 < 13 && (1 << b1) < 8 * sd) ++b1;
            const int s1 = 32 - b1;
            const unsigned m1 = (1u << s1) - 1u;
            for (int s = threadIdx.x; s < (1 << b1); s += blockDim.x) region[s] = kTagEmpty;
            for (int s = threadIdx.x; s < kTagSlots2; s += blockDim.x) t2[s] = kTagEmpty;
            __syncthreads();
            for (int q = threadIdx.x; q < sd; q += blockDim.x) {
                const int k = G.adj[sr + q];
                const unsigned p = (unsigned)k * kTagMul;
                unsigned* slot = region + (p >> s1);
                if (atomicCAS(slot, kTagEmpty, ((unsigned)q << s1) | (p & m1)) != kTagEmpty) {
                    // a shared slot: this entry and the one displaced (if still
                    // there) move to the second table
                    const unsigned old = atomicExch(slot, kTagMulti);
                    tag_insert2(t2, k, q);
                    if (old != kTagMulti) {
                        const int q2 = (int)(old >> s1);
                        tag_insert2(t2, G.adj[sr + q2], q2);
                    }
                }
            }
            __syncthreads();
            const TagTab T{region, t2, G.adj + sr, sd, s1, m1};
            cta_probe_unit<PV, WIN>(G, U, T, cnt, s_ctl, s_base, s_long, tlow, uh, probes);
            __syncthreads();
            if (PV)
                for (int r = threadIdx.x; r < sd; r += blockDim.x) {
                    const unsigned h = T.credited(cnt, r);
                    if (h) atomicAdd(&G.tnew[G.adj[sr + r]], (unsigned long long)h);
                }
        }
    } else {
        int* tab = reinterpret_cast<int*>(region);
        const unsigned buckets = hash_buckets(dp);
        const unsigned bmask = buckets - 1u;
        for (int s = threadIdx.x; s < 4 * (int)buckets; s += blockDim.x) tab[s] = kEmpty;
        __syncthreads();
        for (int q = threadIdx.x; q < dp; q += blockDim.x) hash_insert(tab, bmask, G.adj[rb + q]);
        __syncthreads();
        const HashTab T{tab, bmask, lo, hi};
        cta_probe_unit<PV, WIN>(G, U, T, cnt, s_ctl, s_base, s_long, tlow, uh, probes);
        __syncthreads();
        if (PV)
            for (int s = threadIdx.x; s < 4 * (int)buckets; s += blockDim.x) {
                const unsigned h = T.credited(cnt, s);
                if (h) atomicAdd(&G.tnew[tab[s]], (unsigned long long)h);
            }
    }
    hits += uh;
    if (PV) {
        // j's credit: each warp adds its share (no barrier at the unit's end)
        uh = warp_sum_u64(uh);
        if (lane == 0 && uh) atomicAdd(&G.tnew[G.jbase + U.j], (unsigned long long)uh);
    }
}

// ---------------------------------------------------------------------------
// The count kernel: persistent CTAs first pop CTA units (heaviest first),
// then each warp pops warp units until both queues are empty.  Units may
// belong to different graphs (the batched form): each carries its graph's
// index into the view table, and hits are added to that graph's total.
//
// Dynamic shared memory: per-warp bases (nw x 32 int64) | table region
// (kRegionWords words; warp units use 192-word slices of it) | hit counters
// (PV: kRegionWords/2 words, a tag table's second table past the first
// kTagMaxEntries of them; totals only: the second table alone) | long-task
// queue (unit_tasks x 16 bit).
// ---------------------------------------------------------------------------
template <bool PV, bool MERGE, bool WIN, bool BUCKETS>
__global__ void __launch_bounds__(256, TC_LARGE_MINB)
    k_count(const GraphView* __restrict__ views, const Unit* __restrict__ large, int64_t nlarge,
            const Unit* __restrict__ small, int64_t nsmall, int slice_max, int table_mode,
            int merge_max, unsigned* tlow, unsigned long long* __restrict__ ctr) {
    extern __shared__ __align__(16) unsigned smem[];
    __shared__ long long s_unit;
    __shared__ int s_ctl[4];
    __shared__ unsigned s_wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t* s_base = reinterpret_cast<int64_t*>(smem) + 32 * w;
    unsigned* region = smem + 64 * nw;
    unsigned* cnt = region + kRegionWords;
    unsigned short* s_long =
        reinterpret_cast<unsigned short*>(cnt + (PV ? kRegionWords / 2 : kTagSlots2));
    __shared__ unsigned long long s_work[6];   // units, tasks, staged for [warp, CTA] units
    if (threadIdx.x < 6) s_work[threadIdx.x] = 0;
    GraphAcc acc;
    uint64_t probes = 0;

    // CTA units
    while (true) {
        if (threadIdx.x == 0) {
            s_unit = (long long)atomicAdd(&ctr[CTR_LARGE_HEAD], 1ull);
            s_ctl[0] = 0;
            s_ctl[1] = 0;
            s_ctl[2] = 0;
        }
        __syncthreads();
        const long long u = s_unit;
        if (u >= nlarge) break;
        const Unit U = large[u];
        const GraphView G = views[U.g];
        acc.to(unit_target(G, U));
        cta_unit<PV, WIN, BUCKETS>(G, U, slice_max, region, cnt, s_ctl, s_base, s_long, s_wsum,
                                   tlow, acc.hits, probes);
        if (threadIdx.x == 0) {
            s_work[1] += 1;
            s_work[3] += (unsigned long long)(U.t1 - U.t0);
            s_work[5] += (unsigned long long)min64(
                off_at(G, U.j + 1) - off_at(G, U.j) - (int64_t)U.slice * slice_max, slice_max);
        }
        __syncthreads();
    }
    if (lane == 0 && probes) atomicAdd(&ctr[CTR_PROBES + 1], (unsigned long long)probes);
    probes = 0;

    // warp units, each warp on its own slice of the region
    unsigned* wregion = region + w * kSmallRegionWords;
    unsigned* wcnt = cnt + w * (kSmallTable / 2);
    uint64_t staged = 0;
    while (true) {
        long long u0 = 0;
        if (lane == 0) u0 = (long long)atomicAdd(&ctr[CTR_SMALL_HEAD], (unsigned long long)kGrab);
        u0 = __shfl_sync(0xffffffffu, u0, 0);
        if (u0 >= nsmall) break;
        const int64_t u1 = min64(u0 + kGrab, nsmall);
        for (int64_t u = u0; u < u1; ++u) {
            const Unit U = small[u];
            const GraphView G = views[U.g];
            acc.to(unit_target(G, U));
            warp_unit<PV, MERGE, WIN>(G, U, wregion, wcnt, s_base, BUCKETS, merge_max, tlow, acc.hits,
                                 probes, staged);
            if (lane == 0) {
                atomicAdd(&s_work[0], 1ull);
                atomicAdd(&s_work[2], (unsigned long long)(U.t1 - U.t0));
            }
        }
    }
    acc.flush();
    if (lane == 0) {
        if (probes) atomicAdd(&ctr[CTR_PROBES + 0], (unsigned long long)probes);
        if (staged) atomicAdd(&s_work[4], (unsigned long long)staged);
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int k = threadIdx.x;
        atomicAdd(&ctr[CTR_UNITS + k], s_work[k]);
        atomicAdd(&ctr[CTR_TASKS + k], s_work[2 + k]);
        atomicAdd(&ctr[CTR_STAGED + k], s_work[4 + k]);
    }
}

// per-vertex counts in original ids: the 64-bit accumulator plus, when used,
// the 32-bit per-task shares
__global__ void k_gather_pv(const unsigned long long* __restrict__ tnew, const unsigned* __restrict__ tlow,
                            const int32_t* __restrict__ perm, int64_t n,
                            uint64_t* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = perm[v];
        out[v] = tnew[x] + (tlow ? (uint64_t)tlow[x] : 0ull);
    }
}

__global__ void k_copy_total(const unsigned long long* __restrict__ ctr, uint64_t* __restrict__ out) {
    *out = ctr[CTR_TOTAL];
}

// ---------------------------------------------------------------------------
// Work units over one or many graphs.  Vertex v of the concatenation of the
// graphs (vpre = prefix of vertex counts) is visited in reverse order, so
// the last graph's heaviest pivots come first (batches list their graphs by
// ascending size, so the largest graph leads).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_graph(const int64_t* __restrict__ vpre, int num, int64_t v) {
    int lo = 0, hi = num - 1;   // largest g with vpre[g] <= v
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vpre[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_unit_counts(const GraphView* __restrict__ views, const int64_t* __restrict__ vpre,
                              int num, int64_t V, int small_max, int tw, int tcta, int slice,
                              int32_t* __restrict__ cs, int32_t* __restrict__ cl) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < V;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = V - 1 - x;
        const int g = find_graph(vpre, num, v);
        const GraphView& G = views[g];
        const int64_t j = v - vpre[g];
        const int64_t dp = off_at(G, j + 1) - off_at(G, j);
        const int64_t nt = G.loff[j + 1] - G.loff[j];
        int32_t a = 0, b = 0;
        if (dp > 0 && nt > 0) {
            if (dp <= small_max) {
                a = (int32_t)((nt + tw - 1) / tw);
            } else {
                const int64_t slices = (dp + slice - 1) / slice;
                b = (int32_t)(slices * ((nt + tcta - 1) / tcta));
            }
        }
        cs[x] = a;
        cl[x] = b;
    }
}

__global__ void k_unit_fill(const GraphView* __restrict__ views, const int64_t* __restrict__ vpre,
                            int num, int64_t V, int small_max, int tw, int tcta, int slice,
                            const int64_t* __restrict__ ps, const int64_t* __restrict__ pl,
                            Unit* __restrict__ us, Unit* __restrict__ ul) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < V;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = V - 1 - x;
        const int g = find_graph(vpre, num, v);
        const GraphView& G = views[g];
        const int64_t j = v - vpre[g];
        const int64_t dp = off_at(G, j + 1) - off_at(G, j);
        const int64_t a = G.loff[j], b = G.loff[j + 1];
        if (dp <= 0 || b <= a) continue;
        if (dp <= small_max) {
            int64_t p = ps[x];
            for (int64_t t = a; t < b; t += tw)
                us[p++] = Unit{(int32_t)j, 0, g, 0, t, min64(t + tw, b)};
        } else {
            const int64_t slices = (dp + slice - 1) / slice;
            int64_t p = pl[x];
            for (int64_t t = a; t < b; t += tcta)
                for (int64_t s = 0; s < slices; ++s)
                    ul[p++] = Unit{(int32_t)j, (int32_t)s, g, 0, t, min64(t + tcta, b)};
        }
    }
}

}  // namespace

tc_tuning clamp_tuning(const tc_tuning& t) {
    tc_tuning tt = t;
    tt.slice_max = std::min(tt.slice_max, kRegionWords / 2);   // a hashed slice needs 2 slots per entry
    return tt;
}

void plan_units(UnitPlan& P, const GraphView* views_dev, const int64_t* vpre_dev, int num, int64_t V,
                const tc_tuning& t, Alloc& al, cudaStream_t st) {
    const unsigned G = (unsigned)(num_sms() * 8);
    P.V = V;
    P.num = num;
    P.views = views_dev;
    P.vpre = vpre_dev;
    P.t = t;
    P.cs = Buf<int32_t>(al, (size_t)std::max<int64_t>(V, 1));
    P.cl = Buf<int32_t>(al, (size_t)std::max<int64_t>(V, 1));
    P.ps = Buf<int64_t>(al, (size_t)(V + 1));
    P.pl = Buf<int64_t>(al, (size_t)(V + 1));
    if (V > 0) {
        Prof prof_("k_unit_counts", st);
        k_unit_counts<<<grid_for(V, 256, G), 256, 0, st>>>(views_dev, vpre_dev, num, V,
                                                           t.small_max_outdeg, t.warp_unit_tasks,
                                                           t.cta_unit_tasks, t.slice_max, P.cs.get(),
                                                           P.cl.get());
    }
    TC_LAUNCH_CHECK();
    exclusive_scan2_i32_to_i64(P.cs.get(), P.ps.get(), P.ps.get() + V, P.cl.get(), P.pl.get(), P.pl.get() + V, V,
                               al, st);
}

UnitLists fill_units(UnitPlan& P, int64_t ns, int64_t nl, Alloc& al, cudaStream_t st) {
    const unsigned G = (unsigned)(num_sms() * 8);
    UnitLists L;
    L.bytes = sizeof(Unit) * (size_t)std::max<int64_t>(ns + nl, 1);
    L.mem = al.get(L.bytes);
    L.large = static_cast<Unit*>(L.mem);
    L.small = L.large + nl;
    L.nlarge = nl;
    L.nsmall = ns;
    if (P.V > 0) {
        {
            Prof prof_("k_unit_fill", st);
            k_unit_fill<<<grid_for(P.V, 256, G), 256, 0, st>>>(
                P.views, P.vpre, P.num, P.V, P.t.small_max_outdeg, P.t.warp_unit_tasks,
                P.t.cta_unit_tasks, P.t.slice_max, P.ps.get(), P.pl.get(), L.small, L.large);
        }
        TC_LAUNCH_CHECK();
    }
    P.cs.release();
    P.cl.release();
    P.ps.release();
    P.pl.release();
    return L;
}

UnitLists build_unit_lists(const GraphView* views_dev, const int64_t* vpre_dev, int num, int64_t V,
                           const tc_tuning& t, Alloc& al, cudaStream_t st) {
    UnitPlan P;
    plan_units(P, views_dev, vpre_dev, num, V, t, al, st);
    int64_t ns = 0, nl = 0;
    TC_CUDA(cudaMemcpyAsync(&ns, P.ps.get() + V, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&nl, P.pl.get() + V, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    return fill_units(P, ns, nl, al, st);
}

void adopt_units(tc_graph* g, const UnitLists& L, const tc_tuning& tt) {
    if (g->units_mem) g->alloc.put(g->units_mem, g->units_bytes);
    g->units_mem = L.mem;
    g->units_bytes = L.bytes;
    g->small_units = L.small;
    g->large_units = L.large;
    g->n_small = L.nsmall;
    g->n_large = L.nlarge;
    g->units_tuning = tt;
    g->stats.small_units = L.nsmall;
    g->stats.large_units = L.nlarge;
}

size_t count_smem_bytes(bool pv, int threads, int unit_tasks) {
    return sizeof(int64_t) * 32 * (size_t)(threads / 32) +
           sizeof(unsigned) * (size_t)(kRegionWords + (pv ? kRegionWords / 2 : kTagSlots2)) +
           sizeof(unsigned short) * (size_t)unit_tasks;
}

using CountKernel = void (*)(const GraphView*, const Unit*, int64_t, const Unit*, int64_t, int, int, int,
                            unsigned*, unsigned long long*);

// the count kernel instance for a launch: per-vertex or totals, with or
// without the search path for short pivot rows, or the instance that counts
// one tile of a host-resident graph (a window of rows); each in its bucket
// form for table_mode 1 (the search path is not used there)
CountKernel count_kernel(bool pv, bool merge, bool win, bool buckets) {
    if (buckets)
        return win ? (pv ? k_count<true, false, true, true> : k_count<false, false, true, true>)
                   : (pv ? k_count<true, false, false, true> : k_count<false, false, false, true>);
    if (win) return pv ? k_count<true, false, true, false> : k_count<false, false, true, false>;
    return pv ? (merge ? k_count<true, true, false, false> : k_count<true, false, false, false>)
              : (merge ? k_count<false, true, false, false> : k_count<false, false, false, false>);
}

CountLaunch prepare_count(const UnitLists& L, const tc_tuning& t, bool pv, bool win) {
    CountLaunch c;
    c.threads = t.cta_threads;
    c.smem = count_smem_bytes(pv, c.threads, t.cta_unit_tasks);
    c.pv = pv;
    c.buckets = t.table_mode == 1;
    c.merge = t.merge_max_outdeg > 0 && !win && !c.buckets;
    c.win = win;
    auto kern = count_kernel(pv, c.merge, c.win, c.buckets);
    TC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem));
    int per_sm = 0;
    TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, c.threads, c.smem));
    per_sm = std::max(per_sm, 1);
    const int64_t want =
        L.nlarge + (L.nsmall + kGrab * (c.threads / 32) - 1) / (kGrab * (c.threads / 32));
    c.grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, want));
    return c;
}

void launch_count_raw(const CountLaunch& c, const GraphView* views_dev, const UnitLists& L,
                      const tc_tuning& t, unsigned long long* ctr, cudaStream_t st, unsigned* tlow) {
    if (L.nlarge + L.nsmall == 0) return;
    auto kern = count_kernel(c.pv, c.merge, c.win, c.buckets);
    kern<<<c.grid, c.threads, c.smem, st>>>(views_dev, L.large, L.nlarge, L.small, L.nsmall,
                                            t.slice_max, t.table_mode, t.merge_max_outdeg, tlow, ctr);
    TC_LAUNCH_CHECK();
}

void launch_count(const GraphView* views_dev, const UnitLists& L, const tc_tuning& t, bool pv,
                  unsigned long long* ctr, cudaStream_t st, bool profile, unsigned* tlow, bool win) {
    if (L.nlarge + L.nsmall == 0) return;
    const CountLaunch c = prepare_count(L, t, pv, win);
    if (profile) {
        Prof prof_("k_count", st);
        launch_count_raw(c, views_dev, L, t, ctr, st, tlow);
    } else {
        launch_count_raw(c, views_dev, L, t, ctr, st, tlow);
    }
}

void build_units(tc_graph* g, const tc_tuning& t, cudaStream_t st) {
    const tc_tuning tt = clamp_tuning(t);
    Alloc& al = g->alloc;
    Buf<int64_t> vpre(al, 2);
    const int64_t hv[2] = {0, g->n};
    TC_CUDA(cudaMemcpyAsync(vpre.get(), hv, sizeof(hv), cudaMemcpyHostToDevice, st));
    UnitLists L = build_unit_lists(g->view, vpre.get(), 1, g->n, tt, al, st);
    adopt_units(g, L, tt);
}

void count_components(tc_graph* g, const tc_tuning& t, uint64_t* comp_totals_dev,
                      cudaStream_t st) {
    const tc_tuning tt = clamp_tuning(size_tuning(t, g->m));
    if (!tuning_equal(tt, g->units_tuning)) build_units(g, tt, st);
    TC_CUDA(cudaMemsetAsync(g->counters, 0, sizeof(unsigned long long) * CTR_COUNT, st));
    TC_CUDA(cudaMemsetAsync(g->comp_totals, 0, sizeof(unsigned long long) * (size_t)g->num_comps, st));
    UnitLists L;
    L.large = g->large_units;
    L.small = g->small_units;
    L.nlarge = g->n_large;
    L.nsmall = g->n_small;
    launch_count(g->view_comp, L, tt, false, g->counters, st, true, nullptr);
    TC_CUDA(cudaMemcpyAsync(comp_totals_dev, g->comp_totals, sizeof(uint64_t) * (size_t)g->num_comps,
                            cudaMemcpyDeviceToDevice, st));
}

void count(tc_graph* g, const tc_tuning& t, uint64_t* total_dev, uint64_t* per_vertex_dev,
           cudaStream_t st) {
    // the unit lists are a cache of the tuning they were built for
    const tc_tuning tt = clamp_tuning(size_tuning(t, g->m));
    if (!tuning_equal(tt, g->units_tuning)) build_units(g, tt, st);
    const bool pv = per_vertex_dev != nullptr;
    TC_CUDA(cudaMemsetAsync(g->counters, 0, sizeof(unsigned long long) * CTR_COUNT, st));
    if (pv && g->n > 0) TC_CUDA(cudaMemsetAsync(g->tnew, 0, sizeof(uint64_t) * (size_t)g->n, st));
    // a task's share is at most C(max |U_i|, 2): 32-bit counters when that fits
    const uint64_t dmax = (uint64_t)g->stats.max_outdeg;
    const bool tlow32 = TC_TLOW32 && pv && g->n > 0 && dmax * (dmax - (dmax > 0)) / 2 < (1ull << 32);
    if (tlow32) {
        if (!g->tlow) {
            g->tlow_bytes = sizeof(unsigned) * (size_t)g->n;
            g->tlow = static_cast<unsigned*>(g->alloc.get(g->tlow_bytes));
        }
        TC_CUDA(cudaMemsetAsync(g->tlow, 0, g->tlow_bytes, st));
    }
    UnitLists L;
    L.large = g->large_units;
    L.small = g->small_units;
    L.nlarge = g->n_large;
    L.nsmall = g->n_small;
    launch_count(g->view, L, tt, pv, g->counters, st, true, tlow32 ? g->tlow : nullptr);
    if (pv && g->n > 0) {
        {
            Prof prof_("k_gather_pv", st);
            k_gather_pv<<<grid_for(g->n, 256, num_sms() * 8), 256, 0, st>>>(
                reinterpret_cast<const unsigned long long*>(g->tnew), tlow32 ? g->tlow : nullptr, g->perm, g->n, per_vertex_dev);
        }
        TC_LAUNCH_CHECK();
    }
    if (total_dev) {
        {
            Prof prof_("k_copy_total", st);
            k_copy_total<<<1, 1, 0, st>>>(g->counters, total_dev);
        }
        TC_LAUNCH_CHECK();
    }
}

}  // namespace tc
