// Serving loop over a resident index (declarations and contract in include/fmocc.h).
//
// Continuous batching with several batches in flight.  Requests are copied at submission into
// a FIFO.  The server runs `inflight` worker threads (3 by default).  Each owns a search
// context (a second handle onto the same resident index, with scratch, error words and
// graph state of its own), a stream, and pinned and device batch buffers.  A worker that is
// free takes the pending requests in arrival order, of any search mode, while their reads fit
// the batch's read slots and its share of the device-memory budget for search scratch.  It
// packs their reads with one search-mode byte per read, copies them to the device and runs
// the search (the same call as fm_inexact, with z and max_gaps taken read by read) on its own
// stream, then copies the interval sets back and hands each request its slice.  A request
// that arrives while a batch is on the GPU therefore starts as soon as a worker is free, while
// that batch still runs: the two batches overlap on the device (the second batch's CTAs take
// SMs as the first one's warps finish, and one batch's copies, D pass and grouping run beside
// the other's search).
//
// Admission by memory: a context's scratch may not grow past its share of the budget (the
// growth fails with FM_ENOMEM instead of allocating).  Each worker sizes its next batch by a
// model of the scratch the search allocates (staging records, raw intervals, grouping buffers,
// the spill region), with the raw intervals per query learned from its own batches; a batch
// whose search still runs out of budget is split in two and each half searched on its own.
// Waits are host-side and bounded (fm_server_poll's wait_ms); no kernel waits for work that
// the host appends.
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fm_internal.cuh"

namespace fm {
namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket = 0;
    uint32_t n_reads = 0, z = 0, gaps = 0;
    std::vector<uint8_t> codes;
    std::vector<uint32_t> offs;   // rebased to 0
    std::vector<uint32_t> counts;
    std::vector<uint64_t> offsets;
    std::vector<uint32_t> pairs;
    int status = FM_OK;
    bool done = false;
    uint64_t t_submit = 0, t_start = 0, t_done = 0;
    uint32_t batch_reads = 0;
    uint32_t batch_id = 0;
};

using Batch = std::vector<std::shared_ptr<Request>>;

// One batch in flight: a search context, its stream and its batch buffers.
struct Worker {
    fm_index *ctx = nullptr;
    cudaStream_t stream = nullptr;
    uint8_t *d_codes = nullptr, *h_codes = nullptr, *d_modes = nullptr, *h_modes = nullptr;
    uint32_t *d_offs = nullptr, *h_offs = nullptr;
    uint32_t *d_counts = nullptr, *h_counts = nullptr;
    uint64_t *d_offsets = nullptr, *h_offsets = nullptr;
    uint32_t *d_pairs = nullptr, *h_pairs = nullptr;
    size_t cap_codes = 0, cap_reads = 0, cap_pairs = 0;
    // scratch model: the spill region's bytes once known, raw intervals per query (the
    // largest ratio seen, at least 4)
    uint64_t spill_bytes = 0;
    double raw_per_query = 4.0;
    std::thread thr;
};

// Device bytes the search of nq queries allocates (run_inexact's sizing: staging records,
// raw intervals at 16 B, grouping buffers with 8-byte grouped and temporary keys per raw
// interval, per-query counters and offsets, and the spill region).
uint64_t scratch_model(const Worker &w, uint64_t nq) {
    const double raw = w.raw_per_query * (double)nq;
    const double raw_cap = raw * 1.25 + 1024.0 > (double)nq * 4 + (1 << 20) ? raw * 1.25 + 1024.0
                                                                           : (double)nq * 4 + (1 << 20);
    const uint64_t spill = w.spill_bytes ? w.spill_bytes : (uint64_t)152 * 32 * 4096 * 16;
    return (uint64_t)((double)nq * (kStageU4 * 16 + 64) + raw_cap * 16 + raw * 16) + spill + 4096;
}

}  // namespace
}  // namespace fm

struct fm_server {
    fm_index *h = nullptr;
    fm_server_params p{};
    uint32_t inflight = 3;
    uint64_t budget_per_worker = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<fm::Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<fm::Request>> all;
    bool stopping = false;
    uint64_t next_ticket = 1;
    uint32_t next_batch = 1;
    std::vector<std::unique_ptr<fm::Worker>> workers;
    // counters
    std::atomic<uint64_t> n_batches{0}, n_reads{0}, n_done{0}, busy_ns{0};
};

using namespace fm;

namespace {

void free_buffers(Worker *w) {
    cudaFree(w->d_codes);
    cudaFree(w->d_modes);
    cudaFree(w->d_offs);
    cudaFree(w->d_counts);
    cudaFree(w->d_offsets);
    cudaFree(w->d_pairs);
    cudaFreeHost(w->h_codes);
    cudaFreeHost(w->h_modes);
    cudaFreeHost(w->h_offs);
    cudaFreeHost(w->h_counts);
    cudaFreeHost(w->h_offsets);
    cudaFreeHost(w->h_pairs);
    w->d_codes = w->h_codes = w->d_modes = w->h_modes = nullptr;
    w->d_offs = w->h_offs = w->d_counts = w->h_counts = w->d_pairs = w->h_pairs = nullptr;
    w->d_offsets = w->h_offsets = nullptr;
    w->cap_codes = w->cap_reads = w->cap_pairs = 0;
}

// grow a worker's batch buffers (device and pinned host) to hold the given sizes
int reserve(Worker *w, uint32_t strands, size_t codes, size_t reads, size_t pairs) {
    if (codes > w->cap_codes) {
        cudaFree(w->d_codes);
        cudaFreeHost(w->h_codes);
        w->d_codes = w->h_codes = nullptr;
        w->cap_codes = 0;
        size_t c = codes + codes / 2 + 4096;
        if (cudaMalloc((void **)&w->d_codes, c) || cudaMallocHost((void **)&w->h_codes, c)) {
            cudaGetLastError();
            return FM_ENOMEM;
        }
        w->cap_codes = c;
    }
    if (reads > w->cap_reads) {
        cudaFree(w->d_offs);
        cudaFree(w->d_modes);
        cudaFree(w->d_counts);
        cudaFree(w->d_offsets);
        cudaFreeHost(w->h_offs);
        cudaFreeHost(w->h_modes);
        cudaFreeHost(w->h_counts);
        cudaFreeHost(w->h_offsets);
        w->d_offs = w->h_offs = w->d_counts = w->h_counts = nullptr;
        w->d_modes = w->h_modes = nullptr;
        w->d_offsets = w->h_offsets = nullptr;
        w->cap_reads = 0;
        size_t r = reads + reads / 2 + 64;
        size_t q = r * strands;
        if (cudaMalloc((void **)&w->d_offs, (r + 1) * 4) || cudaMalloc((void **)&w->d_modes, r) ||
            cudaMalloc((void **)&w->d_counts, q * 4) || cudaMalloc((void **)&w->d_offsets, (q + 1) * 8) ||
            cudaMallocHost((void **)&w->h_offs, (r + 1) * 4) || cudaMallocHost((void **)&w->h_modes, r) ||
            cudaMallocHost((void **)&w->h_counts, q * 4) ||
            cudaMallocHost((void **)&w->h_offsets, (q + 1) * 8)) {
            cudaGetLastError();
            return FM_ENOMEM;
        }
        w->cap_reads = r;
    }
    if (pairs > w->cap_pairs) {
        cudaFree(w->d_pairs);
        cudaFreeHost(w->h_pairs);
        w->d_pairs = w->h_pairs = nullptr;
        w->cap_pairs = 0;
        size_t c = pairs + pairs / 2 + 4096;
        if (cudaMalloc((void **)&w->d_pairs, c * 8) || cudaMallocHost((void **)&w->h_pairs, c * 8)) {
            cudaGetLastError();
            return FM_ENOMEM;
        }
        w->cap_pairs = c;
    }
    return FM_OK;
}

void worker_loop(fm_server *s, Worker *w);

void stop_workers(fm_server *s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto &w : s->workers)
        if (w->thr.joinable()) w->thr.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->h->device);
    for (auto &w : s->workers) {
        free_buffers(w.get());
        if (w->stream) cudaStreamDestroy(w->stream);
        free_search_context(w->ctx);
    }
    s->workers.clear();
    if (prev >= 0) cudaSetDevice(prev);
}

}  // namespace

extern "C" {

int fm_server_start(fm_index *h, const fm_server_params *p, fm_server **out) {
    if (!h || !out) return set_global_error(FM_EINVAL, "null argument");
    *out = nullptr;
    if (!h->has_rev) return set_error(h, FM_EINVAL, "index built without reverse(R)");
    fm_server_params q = p ? *p : fm_server_params{};
    if (q.strands == 0) q.strands = 2;
    if (q.strands > 2) return set_error(h, FM_EINVAL, "strands must be 1 or 2");
    if (q.max_batch_reads == 0) q.max_batch_reads = 262144;
    if (q.frontier_budget == 0) q.frontier_budget = (uint64_t)64 << 30;
    if (q.kernel > FM_KERNEL_PERSISTENT) return set_error(h, FM_EINVAL, "unknown kernel");
    if (q.inflight > 4) return set_error(h, FM_EINVAL, "inflight must be 0..4");
    if (q.inflight == 0) q.inflight = 3;
    std::unique_ptr<fm_server> s(new fm_server());
    s->h = h;
    s->p = q;
    s->inflight = q.inflight;
    s->budget_per_worker = q.frontier_budget / q.inflight;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    int rc = FM_OK;
    // the interval and pair tables are built here, on the owner handle, before any context
    // borrows them and not inside the first batch's latency
    cudaStream_t st0 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st0, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_status(h, e, "cudaStreamCreate(server)");
    if (!rc) rc = ensure_kmer(h, st0);
    if (!rc) rc = ensure_pairs(h, st0);
    if (st0) {
        cudaStreamSynchronize(st0);
        cudaStreamDestroy(st0);
    }
    for (uint32_t i = 0; !rc && i < q.inflight; ++i) {
        std::unique_ptr<Worker> w(new Worker());
        w->ctx = new_search_context(h);
        if (!w->ctx) {
            rc = set_error(h, FM_ENOMEM, "search context of the server");
            break;
        }
        w->ctx->scratch_budget = s->budget_per_worker;
        w->ctx->use_graphs = false;   // batch sizes change from one batch to the next
        // scratch for a full batch now: a regrowth during serving would free the old buffer,
        // and cudaFree waits for the whole device, the other workers' batches included (best
        // effort: a budget too small for it leaves the growth to the batches)
        {
            uint64_t nq = (uint64_t)q.max_batch_reads * q.strands;
            while (nq > 1024 && scratch_model(*w, nq) > s->budget_per_worker) nq /= 2;
            if (reserve_search_scratch(w->ctx, nq) != FM_OK) w->ctx->err.clear();
        }
        e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            free_search_context(w->ctx);
            rc = cuda_status(h, e, "cudaStreamCreate(server worker)");
            break;
        }
        s->workers.push_back(std::move(w));
    }
    if (rc) {
        for (auto &w : s->workers) {
            if (w->stream) cudaStreamDestroy(w->stream);
            free_search_context(w->ctx);
        }
        if (prev >= 0) cudaSetDevice(prev);
        return rc;
    }
    if (prev >= 0) cudaSetDevice(prev);
    fm_server *sp = s.release();
    for (auto &w : sp->workers) w->thr = std::thread(worker_loop, sp, w.get());
    *out = sp;
    return FM_OK;
}

int fm_server_submit(fm_server *s, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                     uint32_t z, uint32_t max_gaps, uint64_t *ticket) {
    if (!s || !ticket || (n_reads && (!reads || !offs))) return set_global_error(FM_EINVAL, "null argument");
    if (z > (uint32_t)kMaxZ || max_gaps > (uint32_t)kMaxGaps)
        return set_global_error(FM_EINVAL, "z and max_gaps must be at most 7");
    auto r = std::make_shared<Request>();
    r->n_reads = n_reads;
    r->z = z;
    r->gaps = max_gaps;
    const uint32_t base = n_reads ? offs[0] : 0;
    r->offs.assign(n_reads + 1, 0);
    for (uint32_t i = 1; i <= n_reads; ++i) {
        r->offs[i] = offs[i] - base;
        if (i && (r->offs[i] <= r->offs[i - 1] || r->offs[i] - r->offs[i - 1] > (uint32_t)kMaxReadLen))
            return set_global_error(FM_EINVAL, "read lengths must be 1..255");
    }
    r->codes.assign(reads + base, reads + base + r->offs[n_reads]);
    // one OR over all codes (a loop without an early exit, which the compiler vectorizes)
    uint8_t any = 0;
    for (uint8_t c : r->codes) any |= c;
    if (any > 3) return set_global_error(FM_EINVAL, "a read holds a code above 3");
    if (n_reads > s->p.max_batch_reads)
        return set_global_error(FM_EINVAL, "request larger than one batch");
    r->t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return set_global_error(FM_EINVAL, "server is stopping");
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->pending.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return FM_OK;
}

int fm_server_poll(fm_server *s, uint64_t ticket, uint32_t wait_ms, fm_server_result *res) {
    if (!s || !res) return set_global_error(FM_EINVAL, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_global_error(FM_EINVAL, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    if (!r->done && wait_ms)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return r->done; });
    if (!r->done) return FM_ETIMEOUT;
    res->status = r->status;
    res->n_queries = r->n_reads * s->p.strands;
    res->counts = r->counts.data();
    res->offsets = r->offsets.data();
    res->pairs = r->pairs.data();
    res->t_submit_ns = r->t_submit;
    res->t_start_ns = r->t_start;
    res->t_done_ns = r->t_done;
    res->batch_reads = r->batch_reads;
    res->batch_id = r->batch_id;
    return FM_OK;
}

int fm_server_release(fm_server *s, uint64_t ticket) {
    if (!s) return set_global_error(FM_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end() || !it->second->done) return set_global_error(FM_EINVAL, "unknown or unfinished ticket");
    s->all.erase(it);
    return FM_OK;
}

int fm_server_stats(fm_server *s, uint64_t out[4]) {
    if (!s || !out) return set_global_error(FM_EINVAL, "null argument");
    out[0] = s->n_batches.load();
    out[1] = s->n_reads.load();
    out[2] = s->n_done.load();
    out[3] = s->busy_ns.load() / 1000000;
    return FM_OK;
}

int fm_server_stop(fm_server *s) {
    if (!s) return FM_OK;
    stop_workers(s);
    delete s;
    return FM_OK;
}

}  // extern "C"

namespace {

// Search one batch on a worker and hand every request its slice of the interval sets.  When
// the search runs out of the worker's scratch budget, the batch is split in two halves, each
// searched on its own (a single request that does not fit reports FM_ENOMEM).
void run_batch(fm_server *s, Worker *w, Batch &batch) {
    const uint64_t t0 = now_ns();
    const uint32_t st = s->p.strands;
    uint64_t n = 0, codes = 0;
    for (auto &r : batch) {
        n += r->n_reads;
        codes += r->codes.size();
    }
    int rc = reserve(w, st, codes + 1, n + 1, 4 * n * st + 1024);
    uint64_t need = 0;
    if (!rc) {
        uint64_t pos = 0, rd = 0;
        w->h_offs[0] = 0;
        for (auto &r : batch) {
            memcpy(w->h_codes + pos, r->codes.data(), r->codes.size());
            for (uint32_t i = 1; i <= r->n_reads; ++i) w->h_offs[rd + i] = (uint32_t)(pos + r->offs[i]);
            memset(w->h_modes + rd, (int)(r->z | (r->gaps << 4)), r->n_reads);
            pos += r->codes.size();
            rd += r->n_reads;
        }
        if (cudaMemcpyAsync(w->d_codes, w->h_codes, codes + 1, cudaMemcpyHostToDevice, w->stream) ||
            cudaMemcpyAsync(w->d_offs, w->h_offs, (n + 1) * 4, cudaMemcpyHostToDevice, w->stream) ||
            (n && cudaMemcpyAsync(w->d_modes, w->h_modes, n, cudaMemcpyHostToDevice, w->stream)))
            rc = cuda_status(w->ctx, cudaGetLastError(), "cudaMemcpyAsync(batch)");
    }
    if (!rc) {
        fm_search_params sp{};
        sp.strands = st;
        sp.kernel = s->p.kernel;   // z and max_gaps come read by read from d_modes
        rc = run_inexact(w->ctx, w->d_codes, w->d_offs, (uint32_t)n, &sp, w->d_counts, w->d_offsets,
                         w->d_pairs, w->cap_pairs, &need, w->stream, w->d_modes);
        if (rc == FM_ETRUNC) {
            rc = reserve(w, st, 0, 0, need);
            if (!rc) rc = fetch_inexact(w->ctx, w->d_pairs, w->cap_pairs, w->stream);
        }
    }
    if (rc == FM_ENOMEM && batch.size() > 1) {
        // out of this worker's share of the budget: search the halves one after the other
        Batch a(batch.begin(), batch.begin() + batch.size() / 2), b(batch.begin() + batch.size() / 2, batch.end());
        run_batch(s, w, a);
        run_batch(s, w, b);
        return;
    }
    const uint64_t nq = n * st;
    if (!rc && nq) {
        // learn the raw intervals per query and the spill region's size for the next batches
        unsigned long long rawn = 0;
        if (cudaMemcpyAsync(&rawn, w->ctx->s_misc.ptr, 8, cudaMemcpyDeviceToHost, w->stream) == cudaSuccess &&
            cudaStreamSynchronize(w->stream) == cudaSuccess) {
            const double ratio = (double)rawn / (double)nq;
            if (ratio > w->raw_per_query) w->raw_per_query = ratio;
        }
        w->spill_bytes = w->ctx->s_spill.bytes;
    }
    if (!rc) {
        if (cudaMemcpyAsync(w->h_counts, w->d_counts, nq * 4, cudaMemcpyDeviceToHost, w->stream) ||
            cudaMemcpyAsync(w->h_offsets, w->d_offsets, (nq + 1) * 8, cudaMemcpyDeviceToHost, w->stream) ||
            (need && cudaMemcpyAsync(w->h_pairs, w->d_pairs, need * 8, cudaMemcpyDeviceToHost, w->stream)) ||
            cudaStreamSynchronize(w->stream))
            rc = cuda_status(w->ctx, cudaGetLastError(), "cudaMemcpyAsync(results)");
    }
    const uint64_t t1 = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const uint32_t bid = s->next_batch++;
        uint64_t q0 = 0;
        for (auto &r : batch) {
            const uint64_t rq = (uint64_t)r->n_reads * st;
            r->status = rc;
            if (!rc) {
                const uint64_t p0 = w->h_offsets[q0], p1 = w->h_offsets[q0 + rq];
                r->counts.assign(w->h_counts + q0, w->h_counts + q0 + rq);
                r->offsets.resize(rq + 1);
                for (uint64_t q = 0; q <= rq; ++q) r->offsets[q] = w->h_offsets[q0 + q] - p0;
                r->pairs.assign(w->h_pairs + 2 * p0, w->h_pairs + 2 * p1);
            } else {
                r->counts.assign(rq, 0);
                r->offsets.assign(rq + 1, 0);
            }
            r->t_start = t0;
            r->batch_reads = (uint32_t)n;
            r->batch_id = bid;
            r->t_done = t1;
            r->done = true;
            q0 += rq;
        }
    }
    s->cv_done.notify_all();
    s->n_batches += 1;
    s->n_reads += n;
    s->n_done += batch.size();
    s->busy_ns += t1 - t0;
}

void worker_loop(fm_server *s, Worker *w) {
    cudaSetDevice(s->h->device);
    for (;;) {
        Batch batch;
        bool more = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stopping || !s->pending.empty(); });
            if (s->pending.empty()) {
                if (s->stopping) break;
                continue;
            }
            // requests of any mode join in arrival order while the batch's read slots and
            // the worker's share of the scratch budget (by the scratch model) last; the first
            // request always joins
            uint64_t reads = 0;
            while (!s->pending.empty()) {
                auto &r = s->pending.front();
                const uint64_t nr = reads + r->n_reads;
                if (!batch.empty() && (nr > s->p.max_batch_reads ||
                                       scratch_model(*w, nr * s->p.strands) > s->budget_per_worker))
                    break;
                reads = nr;
                batch.push_back(r);
                s->pending.pop_front();
            }
            more = !s->pending.empty();
        }
        if (more) s->cv_work.notify_one();   // another worker can start on the rest
        run_batch(s, w, batch);
    }
}

}  // namespace
