// Counting a graph whose arrays do not fit the device budget: tiles of U
// streamed through device memory.
//
// The paper bounds each rank's memory by distributing U and L over a
// sqrt(p) x sqrt(p) grid of blocks and shifting blocks between ranks
// (Section 5.1, Eq. 4 and Eq. 5).  On one device the same decomposition
// bounds device memory instead: the <j,i,k> tasks are split by pivot block
// J (a range of pivots j: their rows U_j and their tasks) and, within it, by
// row block I (a range of rows i whose tails the tasks probe).  A tile
// (I, J) needs only the rows of I, the rows of J and the tasks of J with i
// in I, so the count holds one pivot block and two row blocks at a time:
// while the count kernel works on tile (I_a, J), the rows of I_{a+1} are
// uploaded into the other buffer on a copy stream -- the shift step of
// Eq. 5 as a double-buffered transfer.
//
// The graph's arrays live in page-locked host memory (tc_graph_offload).
// A pivot block's tasks, pivot rows and work units are built once; each
// tile then runs the count kernel's tile instance over them with a window
// of rows [i0, i1): tasks of other rows are skipped, tails are read from the
// row buffer, pivot labels start at the block's first pivot.  Totals and
// per-vertex counts accumulate over the tiles.  Row traffic is about the
// number of pivot blocks times the rows, so tasks get the largest share of
// the budget; row blocks are visited in alternating order so the one loaded
// last is reused first.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {




struct JBlock {
    int64_t j0, j1;   // pivots [j0, j1)
    int64_t t0, t1;   // their tasks [t0, t1) (a sub-range when one pivot is split)
};
struct IBlock {
    int64_t i0, i1;   // rows [i0, i1)
};

int64_t off_h(const tc_graph* g, int64_t v) {
    return g->off64 ? static_cast<const int64_t*>(g->host->off)[v]
                    : (int64_t) static_cast<const int32_t*>(g->host->off)[v];
}

// RAII: a non-blocking stream and events, released on every path
struct Streams {
    cudaStream_t copy = nullptr;
    cudaEvent_t ready[2] = {}, freed[2] = {};
    Streams() {
        TC_CUDA(cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            TC_CUDA(cudaEventCreateWithFlags(&ready[b], cudaEventDisableTiming));
            TC_CUDA(cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming));
        }
    }
    ~Streams() {
        if (copy) {
            cudaStreamSynchronize(copy);
            cudaStreamDestroy(copy);
        }
        for (int b = 0; b < 2; ++b) {
            if (ready[b]) cudaEventDestroy(ready[b]);
            if (freed[b]) cudaEventDestroy(freed[b]);
        }
    }
};

}  // namespace

void graph_offload(tc_graph* g, cudaStream_t st) {
    if (g->host) return;
    if (g->num_comps > 0) TC_FAIL(TC_EINVAL, "tc_graph_offload: graphs with components stay on the device");
    HostCopy* h = new HostCopy();
    auto take = [&](void** p, size_t bytes) {
        if (cudaHostAlloc(p, bytes ? bytes : 1, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            TC_FAIL(TC_ENOMEM, "tc_graph_offload: page-locked host allocation of %zu bytes failed", bytes);
        }
    };
    const int64_t n = g->n, m = g->m, T = g->n_tasks;
    const size_t ob = g->off64 ? 8 : 4;
    try {
        take(&h->off, ob * (size_t)(n + 1));
        take(reinterpret_cast<void**>(&h->adj), 4 * (size_t)m);
        take(reinterpret_cast<void**>(&h->loff), 8 * (size_t)(n + 1));
        take(reinterpret_cast<void**>(&h->tasks), sizeof(Task) * (size_t)T);
        take(reinterpret_cast<void**>(&h->perm), 4 * (size_t)n);
        TC_CUDA(cudaMemcpyAsync(h->off, g->off, ob * (size_t)(n + 1), cudaMemcpyDeviceToHost, st));
        if (m) TC_CUDA(cudaMemcpyAsync(h->adj, g->adj, 4 * (size_t)m, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaMemcpyAsync(h->loff, g->loff, 8 * (size_t)(n + 1), cudaMemcpyDeviceToHost, st));
        if (T) TC_CUDA(cudaMemcpyAsync(h->tasks, g->tasks, sizeof(Task) * (size_t)T, cudaMemcpyDeviceToHost, st));
        if (n) TC_CUDA(cudaMemcpyAsync(h->perm, g->perm, 4 * (size_t)n, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        host_copy_free(h);
        throw;
    }
    g->alloc.stream = st;
    if (g->units_mem) g->alloc.put(g->units_mem, g->units_bytes);
    if (g->tlow) g->alloc.put(g->tlow, g->tlow_bytes);
    if (g->arena) g->alloc.put(g->arena, g->arena_bytes);
    g->units_mem = nullptr;
    g->tlow = nullptr;
    g->arena = nullptr;
    g->off = nullptr;
    g->adj = nullptr;
    g->perm = nullptr;
    g->loff = nullptr;
    g->tasks = nullptr;
    g->counters = nullptr;
    g->view = g->view_comp = nullptr;
    g->tnew = nullptr;
    g->small_units = g->large_units = nullptr;
    g->n_small = g->n_large = 0;
    g->units_bytes = g->arena_bytes = g->tlow_bytes = 0;
    g->units_tuning = tc_tuning{};
    g->host = h;
}

void host_copy_free(HostCopy* h) {
    if (!h) return;
    if (h->off) cudaFreeHost(h->off);
    if (h->adj) cudaFreeHost(h->adj);
    if (h->loff) cudaFreeHost(h->loff);
    if (h->tasks) cudaFreeHost(h->tasks);
    if (h->perm) cudaFreeHost(h->perm);
    delete h;
}

void count_tiled(const tc_graph* g, int64_t budget, Alloc& al, const tc_tuning& t0, uint64_t* total_host,
                 uint64_t* per_vertex_host, TiledStats* ts, cudaStream_t st) {
    tc_tuning tt = clamp_tuning(size_tuning(t0, g->m));
    tt.merge_max_outdeg = 0;   // tiles use the table instance only
    const HostCopy* h = g->host;
    const int64_t n = g->n;
    const bool pv = per_vertex_host != nullptr && n > 0;

    // --- sizes within the budget --------------------------------------------
    // Row traffic is about (pivot blocks) x (rows), so tasks get the largest
    // share: every pivot block re-reads the rows below its last pivot.
    const int64_t fixed = (pv ? 8 * n : 0) + 64 * 1024;
    if (budget <= fixed) TC_FAIL(TC_ENOMEM, "tc_count_tiled: a budget of %lld bytes leaves nothing for tiles "
                                            "(%lld needed before any tile)", (long long)budget, (long long)fixed);
    const int64_t avail = (budget - fixed) * 4 / 5;    // the rest: units, scan scratch, alignment
    const int64_t capI = std::max<int64_t>(avail / 4 / 8, 1);       // row entries per row block (2 buffers)
    const int64_t capJ = std::max<int64_t>(avail * 3 / 20 / 8, 1);  // row entries of a pivot block (2 copies)
    const int64_t capT = std::max<int64_t>(avail * 2 / 5 / 16, 1);  // tasks of a pivot block
    const int64_t capP = std::max<int64_t>(avail / 20 / 40, 1);     // pivots of a pivot block
    const int64_t maxrow = g->stats.max_outdeg;
    if (maxrow > capI || maxrow > capJ)
        TC_FAIL(TC_ENOMEM, "tc_count_tiled: a row of %lld entries does not fit a budget of %lld bytes",
                (long long)maxrow, (long long)budget);

    // --- blocks (host, from the host-resident offsets) ----------------------
    std::vector<JBlock> jb;
    int64_t split_pivots = 0;
    for (int64_t j = 0; j < n;) {
        const int64_t j0 = j;
        int64_t rows = 0, tasks = 0;
        bool split = false;
        while (j < n) {
            const int64_t dj = off_h(g, j + 1) - off_h(g, j);
            const int64_t nt = h->loff[j + 1] - h->loff[j];
            if (j == j0 && nt > capT) {          // one pivot's tasks over several blocks
                for (int64_t t = h->loff[j]; t < h->loff[j + 1]; t += capT)
                    jb.push_back(JBlock{j, j + 1, t, std::min(t + capT, h->loff[j + 1])});
                ++j;
                ++split_pivots;
                split = true;
                break;
            }
            if (j > j0 && (rows + dj > capJ || tasks + nt > capT || j - j0 + 1 > capP)) break;
            rows += dj;
            tasks += nt;
            ++j;
        }
        if (!split && h->loff[j] > h->loff[j0]) jb.push_back(JBlock{j0, j, h->loff[j0], h->loff[j]});
    }
    std::vector<IBlock> ib;
    for (int64_t i = 0; i < n;) {
        const int64_t i0 = i;
        int64_t rows = 0;
        while (i < n) {
            const int64_t di = off_h(g, i + 1) - off_h(g, i);
            if (i > i0 && rows + di > capI) break;
            rows += di;
            ++i;
        }
        ib.push_back(IBlock{i0, i});
    }
    int64_t maxP = 1, maxT = 1;
    for (const JBlock& b : jb) {
        maxP = std::max(maxP, b.j1 - b.j0);
        maxT = std::max(maxT, b.t1 - b.t0);
    }

    // --- device buffers ---------------------------------------------------------
    Buf<unsigned long long> ctr(al, CTR_COUNT);
    Buf<uint64_t> tnew(al, pv ? (size_t)n : 1);
    Buf<GraphView> view(al, 1);
    Buf<int64_t> vpre(al, 2);
    Buf<int32_t> rows[2] = {Buf<int32_t>(al, (size_t)(capI + capJ)), Buf<int32_t>(al, (size_t)(capI + capJ))};
    Buf<Task> jtasks(al, (size_t)maxT);
    Buf<int64_t> joff(al, (size_t)maxP + 1), jloff(al, (size_t)maxP + 1);
    TC_CUDA(cudaMemsetAsync(ctr.get(), 0, sizeof(unsigned long long) * CTR_COUNT, st));
    if (pv) TC_CUDA(cudaMemsetAsync(tnew.get(), 0, sizeof(uint64_t) * (size_t)n, st));
    Streams S;
    std::vector<int64_t> hj(maxP + 1), hl(maxP + 1);
    int64_t holds[2] = {-1, -1};   // the row block each buffer holds
    if (ts) {
        *ts = TiledStats{};
        ts->pivot_blocks = (int64_t)jb.size();
        ts->row_blocks = (int64_t)ib.size();
        ts->split_pivots = split_pivots;
    }
    // row block a into buffer slot, on the copy stream, once the count that
    // last read that buffer is done
    auto upload_rows = [&](int64_t a, int slot) {
        const int64_t r0 = off_h(g, ib[a].i0), r1 = off_h(g, ib[a].i1);
        TC_CUDA(cudaStreamWaitEvent(S.copy, S.freed[slot], 0));
        if (r1 > r0)
            TC_CUDA(cudaMemcpyAsync(rows[slot].get(), h->adj + r0, 4 * (size_t)(r1 - r0),
                                    cudaMemcpyHostToDevice, S.copy));
        TC_CUDA(cudaEventRecord(S.ready[slot], S.copy));
        holds[slot] = a;
        if (ts) ts->h2d_bytes += 4 * (r1 - r0);
    };
    for (int b = 0; b < 2; ++b) {
        TC_CUDA(cudaEventRecord(S.freed[b], st));
        TC_CUDA(cudaEventRecord(S.ready[b], S.copy));
    }

    for (size_t bi = 0; bi < jb.size(); ++bi) {
        const JBlock& b = jb[bi];
        const int64_t nJ = b.j1 - b.j0, Tb = b.t1 - b.t0;
        const int64_t c0 = off_h(g, b.j0), c1 = off_h(g, b.j1);
        // the row blocks this pivot block needs (tasks have i < j), in
        // alternating order so the block loaded last is needed first next
        std::vector<int64_t> need;
        for (int64_t a = 0; a < (int64_t)ib.size(); ++a)
            if (ib[a].i0 < b.j1) need.push_back(a);
        if (bi % 2) std::reverse(need.begin(), need.end());
        // pivot rows into the top of both buffers, tasks and local offsets
        for (int s = 0; s < 2; ++s) {
            TC_CUDA(cudaStreamWaitEvent(st, S.freed[s], 0));
            if (c1 > c0)
                TC_CUDA(cudaMemcpyAsync(rows[s].get() + capI, h->adj + c0, 4 * (size_t)(c1 - c0),
                                        cudaMemcpyHostToDevice, st));
        }
        TC_CUDA(cudaMemcpyAsync(jtasks.get(), h->tasks + b.t0, sizeof(Task) * (size_t)Tb,
                                cudaMemcpyHostToDevice, st));
        for (int64_t q = 0; q <= nJ; ++q) {
            hj[q] = off_h(g, b.j0 + q) - c0 + capI;
            hl[q] = std::min(std::max(h->loff[b.j0 + q], b.t0), b.t1) - b.t0;
        }
        // pageable sources: staged before the calls return
        TC_CUDA(cudaMemcpyAsync(joff.get(), hj.data(), 8 * (size_t)(nJ + 1), cudaMemcpyHostToDevice, st));
        TC_CUDA(cudaMemcpyAsync(jloff.get(), hl.data(), 8 * (size_t)(nJ + 1), cudaMemcpyHostToDevice, st));
        if (ts) ts->h2d_bytes += 4 * (c1 - c0) * 2 + (int64_t)sizeof(Task) * Tb + 16 * (nJ + 1);
        // work units of the whole pivot block, built once; each tile runs
        // them with its row window and skips tasks of other rows
        GraphView v{};
        v.off = joff.get();
        v.off64 = 1;
        v.adj = rows[0].get();
        v.loff = jloff.get();
        v.tasks = jtasks.get();
        v.tnew = pv ? reinterpret_cast<unsigned long long*>(tnew.get()) : nullptr;
        v.total = ctr.get() + CTR_TOTAL;
        v.n = nJ;
        v.jbase = (int32_t)b.j0;
        v.i0 = 0;
        v.i1 = 0;
        const int64_t hv[2] = {0, nJ};
        TC_CUDA(cudaMemcpyAsync(view.get(), &v, sizeof(v), cudaMemcpyHostToDevice, st));
        TC_CUDA(cudaMemcpyAsync(vpre.get(), hv, sizeof(hv), cudaMemcpyHostToDevice, st));
        UnitPlan P;
        plan_units(P, view.get(), vpre.get(), 1, nJ, tt, al, st);
        int64_t cnt[2] = {0, 0};
        TC_CUDA(cudaMemcpyAsync(&cnt[0], P.ps.get() + nJ, 8, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaMemcpyAsync(&cnt[1], P.pl.get() + nJ, 8, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        UnitLists L = fill_units(P, cnt[0], cnt[1], al, st);
        const CountLaunch launch = prepare_count(L, tt, pv, true);
        try {
            for (size_t a = 0; a < need.size(); ++a) {
                const int64_t blk = need[a];
                int slot = holds[0] == blk ? 0 : holds[1] == blk ? 1 : -1;
                if (slot < 0) {
                    // the buffer not holding the row block counted just before
                    slot = (a > 0 && holds[0] == need[a - 1]) ? 1 : 0;
                    upload_rows(blk, slot);
                }
                // the next row block goes out while this tile counts
                if (a + 1 < need.size()) {
                    const int64_t nb = need[a + 1];
                    if (holds[0] != nb && holds[1] != nb) upload_rows(nb, 1 - slot);
                }
                v.adj = rows[slot].get();
                v.i0 = (int32_t)ib[blk].i0;
                v.i1 = (int32_t)ib[blk].i1;
                v.tail_shift = off_h(g, ib[blk].i0);
                TC_CUDA(cudaMemcpyAsync(view.get(), &v, sizeof(v), cudaMemcpyHostToDevice, st));
                TC_CUDA(cudaStreamWaitEvent(st, S.ready[slot], 0));
                TC_CUDA(cudaMemsetAsync(ctr.get() + CTR_SMALL_HEAD, 0, 2 * sizeof(unsigned long long), st));
                if (L.nlarge + L.nsmall > 0) {
                    Prof prof_("k_count", st);
                    launch_count_raw(launch, view.get(), L, tt, ctr.get(), st, nullptr);
                }
                TC_CUDA(cudaEventRecord(S.freed[slot], st));
                if (ts) ts->tiles += 1;
            }
        } catch (...) {
            al.put(L.mem, L.bytes);
            throw;
        }
        al.put(L.mem, L.bytes);
        if (ts) ts->tile_tasks += Tb;
    }

    // totals and per-vertex counts back to the host
    unsigned long long tot = 0;
    TC_CUDA(cudaMemcpyAsync(&tot, ctr.get() + CTR_TOTAL, sizeof(tot), cudaMemcpyDeviceToHost, st));
    std::vector<uint64_t> tn;
    if (pv) {
        tn.resize((size_t)n);
        TC_CUDA(cudaMemcpyAsync(tn.data(), tnew.get(), 8 * (size_t)n, cudaMemcpyDeviceToHost, st));
    }
    TC_CUDA(cudaStreamSynchronize(st));
    if (pv)
        for (int64_t v = 0; v < n; ++v) per_vertex_host[v] = tn[(size_t)h->perm[v]];
    *total_host = tot;
    if (ts) {
        unsigned long long c[CTR_COUNT];
        TC_CUDA(cudaMemcpyAsync(c, ctr.get(), sizeof(c), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        ts->probes = c[CTR_PROBES] + c[CTR_PROBES + 1];
    }
}

}  // namespace tc
