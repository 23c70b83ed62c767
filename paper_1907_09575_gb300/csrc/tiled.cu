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
// Per tile, the tasks of J with i in I are compacted (order kept, so they
// stay grouped by pivot) with their tails rebased onto the row buffer,
// work units are built for the tile and the ordinary count kernel runs on
// a view whose pivot labels start at J's first pivot.  Totals and
// per-vertex counts accumulate over the tiles.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int kT = 256;

__global__ void k_tile_flags(const Task* __restrict__ tasks, int64_t count, int32_t i0, int32_t i1,
                             int32_t* __restrict__ flags) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = tasks[t].i;
        flags[t] = (i >= i0 && i < i1) ? 1 : 0;
    }
}

// the selected tasks, in order, with their tails rebased onto the row buffer
__global__ void k_tile_compact(const Task* __restrict__ tasks, const int32_t* __restrict__ flags,
                               const int64_t* __restrict__ pos, int64_t count, int64_t shift,
                               Task* __restrict__ out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        if (flags[t]) {
            Task x = tasks[t];
            x.start -= shift;
            out[pos[t]] = x;
        }
}

// tile task offsets per local pivot: the selected tasks before its first task
__global__ void k_tile_loff(const int64_t* __restrict__ jloff, const int64_t* __restrict__ pos,
                            int64_t npiv, int64_t* __restrict__ tloff) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= npiv;
         j += (int64_t)gridDim.x * blockDim.x)
        tloff[j] = pos[jloff[j]];
}

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
    const tc_tuning tt = clamp_tuning(t0);
    const HostCopy* h = g->host;
    const int64_t n = g->n;
    const bool pv = per_vertex_host != nullptr && n > 0;
    const unsigned G = (unsigned)(num_sms() * 8);

    // --- sizes within the budget --------------------------------------------
    const int64_t fixed = (pv ? 8 * n : 0) + 64 * 1024;
    if (budget <= fixed) TC_FAIL(TC_ENOMEM, "tc_count_tiled: a budget of %lld bytes leaves nothing for tiles "
                                            "(%lld needed before any tile)", (long long)budget, (long long)fixed);
    const int64_t avail = (budget - fixed) * 3 / 4;    // the rest: units, scan scratch, alignment
    const int64_t capI = std::max<int64_t>(avail * 4 / 10 / 8, 1);   // row entries per row block
    const int64_t capJ = std::max<int64_t>(avail / 10 / 8, 1);       // row entries of a pivot block
    const int64_t capT = std::max<int64_t>(avail * 35 / 100 / 44, 1);  // tasks of a pivot block
    const int64_t capP = std::max<int64_t>(avail * 5 / 100 / 48, 1);   // pivots of a pivot block
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
    Buf<Task> jtasks(al, (size_t)maxT), ttasks(al, (size_t)maxT);
    Buf<int32_t> flags(al, (size_t)maxT);
    Buf<int64_t> pos(al, (size_t)maxT + 1);
    Buf<int64_t> joff(al, (size_t)maxP + 1), jloff(al, (size_t)maxP + 1), tloff(al, (size_t)maxP + 1);
    TC_CUDA(cudaMemsetAsync(ctr.get(), 0, sizeof(unsigned long long) * CTR_COUNT, st));
    if (pv) TC_CUDA(cudaMemsetAsync(tnew.get(), 0, sizeof(uint64_t) * (size_t)n, st));
    Streams S;
    std::vector<int64_t> hj(maxP + 1), hl(maxP + 1);
    int64_t ntile = 0;   // tiles issued (double-buffer slot = ntile % 2)
    if (ts) *ts = TiledStats{};
    if (ts) {
        ts->pivot_blocks = (int64_t)jb.size();
        ts->row_blocks = (int64_t)ib.size();
        ts->split_pivots = split_pivots;
    }

    // the row blocks a pivot block needs: every I with i0 < j1 (tasks have i < j)
    auto upload_rows = [&](const IBlock& b, int slot) {
        const int64_t r0 = off_h(g, b.i0), r1 = off_h(g, b.i1);
        TC_CUDA(cudaStreamWaitEvent(S.copy, S.freed[slot], 0));
        if (r1 > r0)
            TC_CUDA(cudaMemcpyAsync(rows[slot].get(), h->adj + r0, 4 * (size_t)(r1 - r0),
                                    cudaMemcpyHostToDevice, S.copy));
        TC_CUDA(cudaEventRecord(S.ready[slot], S.copy));
        if (ts) ts->h2d_bytes += 4 * (r1 - r0);
    };
    // both buffers start free
    for (int b = 0; b < 2; ++b) TC_CUDA(cudaEventRecord(S.freed[b], st));

    for (const JBlock& b : jb) {
        const int64_t nJ = b.j1 - b.j0, Tb = b.t1 - b.t0;
        const int64_t c0 = off_h(g, b.j0), c1 = off_h(g, b.j1);
        // pivot rows into the top of both buffers, tasks, local offsets
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
        std::vector<const IBlock*> need;
        for (const IBlock& r : ib)
            if (r.i0 < b.j1) need.push_back(&r);
        // the first row block of this pivot block goes out now; each tile
        // then sends the next one before it counts
        if (!need.empty()) upload_rows(*need[0], (int)(ntile % 2));
        for (size_t a = 0; a < need.size(); ++a) {
            const int slot = (int)((ntile + a) % 2);
            if (a + 1 < need.size()) upload_rows(*need[a + 1], (int)((ntile + a + 1) % 2));
            const IBlock& r = *need[a];
            {
                Prof prof_("k_tile_flags", st);
                k_tile_flags<<<grid_for(Tb, kT, G), kT, 0, st>>>(jtasks.get(), Tb, (int32_t)r.i0,
                                                                   (int32_t)r.i1, flags.get());
            }
            TC_LAUNCH_CHECK();
            exclusive_scan_i32_to_i64(flags.get(), pos.get(), Tb, pos.get() + Tb, al, st);
            {
                Prof prof_("k_tile_compact", st);
                k_tile_compact<<<grid_for(Tb, kT, G), kT, 0, st>>>(jtasks.get(), flags.get(), pos.get(), Tb,
                                                                     off_h(g, r.i0), ttasks.get());
            }
            TC_LAUNCH_CHECK();
            {
                Prof prof_("k_tile_loff", st);
                k_tile_loff<<<grid_for(nJ + 1, kT, G), kT, 0, st>>>(jloff.get(), pos.get(), nJ, tloff.get());
            }
            TC_LAUNCH_CHECK();
            GraphView v{};
            v.off = joff.get();
            v.off64 = 1;
            v.adj = rows[slot].get();
            v.loff = tloff.get();
            v.tasks = ttasks.get();
            v.tnew = pv ? reinterpret_cast<unsigned long long*>(tnew.get()) : nullptr;
            v.total = ctr.get() + CTR_TOTAL;
            v.n = nJ;
            v.jbase = (int32_t)b.j0;
            const int64_t hv[2] = {0, nJ};
            TC_CUDA(cudaMemcpyAsync(view.get(), &v, sizeof(v), cudaMemcpyHostToDevice, st));
            TC_CUDA(cudaMemcpyAsync(vpre.get(), hv, sizeof(hv), cudaMemcpyHostToDevice, st));
            UnitPlan P;
            plan_units(P, view.get(), vpre.get(), 1, nJ, tt, al, st);
            int64_t cnt[3] = {0, 0, 0};
            TC_CUDA(cudaMemcpyAsync(&cnt[0], P.ps.get() + nJ, 8, cudaMemcpyDeviceToHost, st));
            TC_CUDA(cudaMemcpyAsync(&cnt[1], P.pl.get() + nJ, 8, cudaMemcpyDeviceToHost, st));
            TC_CUDA(cudaMemcpyAsync(&cnt[2], pos.get() + Tb, 8, cudaMemcpyDeviceToHost, st));
            TC_CUDA(cudaStreamSynchronize(st));
            UnitLists L = fill_units(P, cnt[0], cnt[1], al, st);
            TC_CUDA(cudaStreamWaitEvent(st, S.ready[slot], 0));
            TC_CUDA(cudaMemsetAsync(ctr.get() + CTR_SMALL_HEAD, 0, 2 * sizeof(unsigned long long), st));
            try {
                launch_count(view.get(), L, tt, pv, ctr.get(), st, true, nullptr);
            } catch (...) {
                al.put(L.mem, L.bytes);
                throw;
            }
            al.put(L.mem, L.bytes);
            TC_CUDA(cudaEventRecord(S.freed[slot], st));
            if (ts) {
                ts->tiles += 1;
                ts->tile_tasks += cnt[2];
            }
        }
        ntile += (int64_t)need.size();
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
