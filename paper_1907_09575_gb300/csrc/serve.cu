// Serving: a continuously batched request loop for exact triangle counts.
//
// Requests (seeded RMAT graph specs) queue in arrival order.  Worker
// threads, each with its own CUDA stream, repeatedly form a tick: they take
// requests from the head of the queue while the tick stays under its size
// caps and the device bytes of all ticks in flight stay under the HBM
// budget (admission by footprint), expand the requests on the device in one
// launch, preprocess their disjoint union as one graph, count it with
// per-component totals and post one result per request.  With several
// workers, the ticks of requests that arrive while others are on the GPU
// overlap on the device; a tick is admitted as soon as a worker and memory
// free up.  Every result is an exact count of its own graph, whatever it was
// batched with.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "tc_internal.cuh"

namespace {

struct Pending {
    int64_t ticket;
    tc_rmat_spec spec;
    double t_arrival;
    int64_t bytes;
};

int64_t footprint(const tc_rmat_spec& s) {
    // pairs on the device (8 B), preprocessing scratch (~28 B per pair),
    // graph arena (~24 B per edge, ~40 B per vertex), plus slack
    return 64 * s.num_pairs + 48 * s.n + 4096;
}

}  // namespace

struct tc_server {
    tc_server_config cfg{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    cudaEvent_t ev_ref = nullptr;        // device time origin of the tick spans
    std::vector<std::pair<double, double>> spans;   // per tick: device start, end (s)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> pending;
    std::vector<tc_server_result> done;
    std::vector<std::thread> workers;
    bool stop = false;
    int64_t next_ticket = 0;
    int64_t bytes_in_flight = 0;
    int64_t peak_bytes = 0;
    int64_t submitted = 0, completed = 0, ticks = 0, failed = 0;
    int64_t busy_workers = 0;
    tc_status first_error = TC_OK;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace tc {
namespace {

// Runs one tick on stream st; fills totals (one per request).  e0 and e1 are
// recorded on st before the tick's first device operation and after its last.
void run_tick(const std::vector<Pending>& reqs, std::vector<uint64_t>& totals, cudaStream_t st,
              cudaEvent_t e0, cudaEvent_t e1) {
    const int nreq = (int)reqs.size();
    std::vector<int64_t> ppre(nreq + 1, 0), vpre(nreq + 1, 0);
    std::vector<RmatJob> jobs(nreq);
    for (int r = 0; r < nreq; ++r) {
        const tc_rmat_spec& s = reqs[r].spec;
        jobs[r] = make_rmat_job(s.seed, s.scale, s.n, s.t1, s.t2, s.t3, vpre[r]);
        ppre[r + 1] = ppre[r] + s.num_pairs;
        vpre[r + 1] = vpre[r] + s.n;
    }
    const int64_t P = ppre[nreq];
    Alloc al;
    al.stream = st;
    Buf<RmatJob> djobs(al, (size_t)nreq);
    Buf<int64_t> dppre(al, (size_t)nreq + 1);
    Buf<int32_t> src(al, (size_t)std::max<int64_t>(P, 1)), dst(al, (size_t)std::max<int64_t>(P, 1));
    Buf<uint64_t> dtot(al, (size_t)nreq);
    TC_CUDA(cudaEventRecord(e0, st));
    TC_CUDA(cudaMemcpyAsync(djobs.get(), jobs.data(), sizeof(RmatJob) * nreq, cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaMemcpyAsync(dppre.get(), ppre.data(), sizeof(int64_t) * (nreq + 1), cudaMemcpyHostToDevice, st));
    generate_rmat_multi(djobs.get(), dppre.get(), nreq, P, src.get(), dst.get(), st);
    tc_graph* g = new tc_graph();
    try {
        g->n = vpre[nreq];
        g->num_pairs = P;
        g->bits = std::max(1, ceil_log2_u64((uint64_t)std::max<int64_t>(g->n, 1)));
        g->alloc.stream = st;
        g->stats.n = g->n;
        g->stats.num_pairs = P;
        preprocess_with_components(g, src.get(), dst.get(), P, TC_INPUT_ON_DEVICE, vpre.data(), nreq, st);
        tc_tuning t;
        tuning_resolve(nullptr, &t);
        count_components(g, t, dtot.get(), st);
        totals.assign(nreq, 0);
        TC_CUDA(cudaMemcpyAsync(totals.data(), dtot.get(), sizeof(uint64_t) * nreq, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaEventRecord(e1, st));
        TC_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        if (g->units_mem) g->alloc.put(g->units_mem, g->units_bytes);
        if (g->arena) g->alloc.put(g->arena, g->arena_bytes);
        delete g;
        throw;
    }
    if (g->units_mem) g->alloc.put(g->units_mem, g->units_bytes);
    if (g->arena) g->alloc.put(g->arena, g->arena_bytes);
    delete g;
}

void worker_loop(tc_server* S) {
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->first_error = TC_ECUDA;
        return;
    }
    while (true) {
        std::vector<Pending> tick;
        int64_t tick_bytes = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] {
                if (S->stop) return true;
                if (S->pending.empty()) return false;
                // the head request must fit next to what is already in flight
                return S->bytes_in_flight + S->pending.front().bytes <= S->cfg.hbm_budget_bytes;
            });
            if (S->stop && S->pending.empty()) break;
            if (S->stop && S->bytes_in_flight + S->pending.front().bytes > S->cfg.hbm_budget_bytes)
                break;
            int64_t pairs = 0;
            while (!S->pending.empty() && (int)tick.size() < S->cfg.max_batch) {
                const Pending& p = S->pending.front();
                if (!tick.empty() && pairs + p.spec.num_pairs > S->cfg.max_tick_pairs) break;
                if (S->bytes_in_flight + tick_bytes + p.bytes > S->cfg.hbm_budget_bytes) break;
                tick.push_back(p);
                tick_bytes += p.bytes;
                pairs += p.spec.num_pairs;
                S->pending.pop_front();
            }
            S->bytes_in_flight += tick_bytes;
            S->peak_bytes = std::max(S->peak_bytes, S->bytes_in_flight);
            S->busy_workers += 1;
        }
        const double t_admit = S->now();
        std::vector<uint64_t> totals;
        tc_status status = TC_OK;
        double d0 = -1.0, d1 = -1.0;
        try {
            run_tick(tick, totals, st, e0, e1);
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, S->ev_ref, e0) == cudaSuccess &&
                cudaEventElapsedTime(&b, S->ev_ref, e1) == cudaSuccess) {
                d0 = a * 1e-3;
                d1 = b * 1e-3;
            }
        } catch (const Error& e) {
            status = e.status;
        } catch (...) {
            status = TC_ECUDA;
        }
        const double t_done = S->now();
        int64_t tick_pairs = 0;
        for (const Pending& p : tick) tick_pairs += p.spec.num_pairs;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t r = 0; r < tick.size(); ++r) {
                tc_server_result res{};
                res.ticket = tick[r].ticket;
                res.triangles = status == TC_OK ? totals[r] : 0;
                res.t_arrival = tick[r].t_arrival;
                res.t_admit = t_admit;
                res.t_done = t_done;
                res.status = status;
                res.tick_requests = (int32_t)tick.size();
                res.tick_pairs = tick_pairs;
                res.t_dev_start = d0;
                res.t_dev_end = d1;
                S->done.push_back(res);
            }
            if (d0 >= 0.0) S->spans.emplace_back(d0, d1);
            S->completed += (int64_t)tick.size();
            if (status != TC_OK) {
                S->failed += (int64_t)tick.size();
                if (S->first_error == TC_OK) S->first_error = status;
            }
            S->ticks += 1;
            S->bytes_in_flight -= tick_bytes;
            S->busy_workers -= 1;
        }
        S->cv.notify_all();
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

// Device time covered by at least one tick and by at least two, from the
// ticks' [start, end] spans.
void span_cover(std::vector<std::pair<double, double>> v, double& busy, double& overlap) {
    busy = overlap = 0.0;
    std::vector<std::pair<double, int>> ev;
    ev.reserve(2 * v.size());
    for (auto& p : v) {
        ev.emplace_back(p.first, +1);
        ev.emplace_back(p.second, -1);
    }
    std::sort(ev.begin(), ev.end());
    int depth = 0;
    double last = 0.0;
    for (auto& e : ev) {
        if (depth >= 1) busy += e.first - last;
        if (depth >= 2) overlap += e.first - last;
        depth += e.second;
        last = e.first;
    }
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_server_create(const tc_server_config* cfg, tc_server** out) {
    clear_error();
    if (!out) {
        set_error("tc_server_create: out is NULL");
        return TC_EINVAL;
    }
    tc_server* S = new tc_server();
    S->cfg.device = -1;
    if (cfg) S->cfg = *cfg;
    if (S->cfg.hbm_budget_bytes <= 0) S->cfg.hbm_budget_bytes = 16ll << 30;
    if (S->cfg.workers <= 0) S->cfg.workers = 2;
    if (S->cfg.max_batch <= 0) S->cfg.max_batch = 512;
    if (S->cfg.max_tick_pairs <= 0) S->cfg.max_tick_pairs = 1ll << 27;
    if (S->cfg.device < 0) {
        if (cudaGetDevice(&S->device) != cudaSuccess) {
            delete S;
            set_error("tc_server_create: no current device");
            return TC_ECUDA;
        }
    } else {
        S->device = S->cfg.device;
    }
    {
        int prev = 0;
        cudaGetDevice(&prev);
        bool ok = cudaSetDevice(S->device) == cudaSuccess &&
                  cudaEventCreate(&S->ev_ref) == cudaSuccess &&
                  cudaEventRecord(S->ev_ref, nullptr) == cudaSuccess &&
                  cudaEventSynchronize(S->ev_ref) == cudaSuccess;
        cudaSetDevice(prev);
        if (!ok) {
            const int dev = S->device;
            if (S->ev_ref) cudaEventDestroy(S->ev_ref);
            delete S;
            set_error("tc_server_create: cannot set up device %d", dev);
            return TC_ECUDA;
        }
    }
    S->t0 = std::chrono::steady_clock::now();
    for (int w = 0; w < S->cfg.workers; ++w) S->workers.emplace_back(worker_loop, S);
    *out = S;
    return TC_OK;
}

double tc_server_now(const tc_server* s) { return s ? s->now() : 0.0; }

}  // extern "C"

namespace {

bool spec_ok(const tc_rmat_spec& s) {
    return s.scale >= 1 && s.scale <= 31 && s.n >= 1 && s.n <= (1ll << s.scale) &&
           s.num_pairs >= 0 && s.num_pairs <= (int64_t)0x7fffffff && s.t1 <= s.t2 && s.t2 <= s.t3;
}

}  // namespace

extern "C" {

tc_status tc_server_submit_rmat(tc_server* s, const tc_rmat_spec* spec, double t_arrival,
                                int64_t* ticket) {
    return tc_server_submit_rmat_many(s, spec, 1, &t_arrival, ticket);
}

tc_status tc_server_submit_rmat_many(tc_server* s, const tc_rmat_spec* specs, int32_t count,
                                     const double* t_arrival, int64_t* tickets) {
    clear_error();
    if (!s || count < 0 || (count > 0 && (!specs || !t_arrival))) {
        set_error("tc_server_submit_rmat: NULL argument or negative count");
        return TC_EINVAL;
    }
    for (int32_t k = 0; k < count; ++k)
        if (!spec_ok(specs[k])) {
            set_error("tc_server_submit_rmat: bad request spec (request %d)", k);
            return TC_EINVAL;
        }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int32_t k = 0; k < count; ++k) {
            const int64_t bytes = footprint(specs[k]);
            if (bytes > s->cfg.hbm_budget_bytes) {
                set_error("tc_server_submit_rmat: request %d needs %lld bytes, over the %lld-byte "
                          "budget", k, (long long)bytes, (long long)s->cfg.hbm_budget_bytes);
                return TC_EBUSY;
            }
        }
        for (int32_t k = 0; k < count; ++k) {
            Pending p;
            p.spec = specs[k];
            p.t_arrival = t_arrival[k];
            p.bytes = footprint(specs[k]);
            p.ticket = s->next_ticket++;
            s->pending.push_back(p);
            s->submitted += 1;
            if (tickets) tickets[k] = p.ticket;
        }
    }
    s->cv.notify_all();
    return TC_OK;
}

tc_status tc_server_poll(tc_server* s, tc_server_result* out, int32_t max, int32_t* count,
                         int32_t wait_ms) {
    clear_error();
    if (!s || !count || (max > 0 && !out)) {
        set_error("tc_server_poll: NULL argument");
        return TC_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    const int32_t k = (int32_t)std::min<size_t>((size_t)std::max(max, 0), s->done.size());
    for (int32_t i = 0; i < k; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + k);
    *count = k;
    return TC_OK;
}

tc_status tc_server_drain(tc_server* s, int32_t timeout_ms) {
    clear_error();
    if (!s) {
        set_error("tc_server_drain: NULL server");
        return TC_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                                   [&] { return s->completed == s->submitted; });
    if (!ok) {
        set_error("tc_server_drain: %lld of %lld requests still open after %d ms",
                  (long long)(s->submitted - s->completed), (long long)s->submitted, timeout_ms);
        return TC_ETIMEOUT;
    }
    return s->first_error;
}

tc_status tc_server_get_stats(tc_server* s, tc_server_stats* out) {
    clear_error();
    if (!s || !out) {
        set_error("tc_server_get_stats: NULL argument");
        return TC_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->pending = (int64_t)s->pending.size();
    out->ticks = s->ticks;
    out->bytes_in_flight = s->bytes_in_flight;
    out->peak_bytes_in_flight = s->peak_bytes;
    out->busy_workers = s->busy_workers;
    span_cover(s->spans, out->device_busy_s, out->device_overlap_s);
    return TC_OK;
}

void tc_server_free(tc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto& t : s->workers) t.join();
    if (s->ev_ref) cudaEventDestroy(s->ev_ref);
    delete s;
}

}  // extern "C"
