// Serving loop over a resident index (declarations and contract in include/fmocc.h).
//
// One server thread per fm_server.  Requests are copied at submission into a FIFO.  The
// thread forms a batch from the oldest pending request's search mode (z, max_gaps): it takes
// the pending requests of that mode in arrival order while their reads fit the batch's read
// slots and the per-batch device-memory budget, packs their reads into pinned host memory,
// copies them to the device, runs the search (the same call as fm_inexact) on its own stream,
// copies the interval sets back and splits them per request.  Requests that arrive meanwhile
// wait for the next batch: batches are formed continuously, one after the other, as long as
// work is pending.  Waits for results are bounded (fm_server_poll's wait_ms).
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
};

// device-memory estimate of one query's search scratch (metadata, raw intervals, grouping)
constexpr uint64_t kScratchPerQuery = 16 + 4 * 16 + 4 * 4 + 16 + 2 * 4 * 8;

}  // namespace
}  // namespace fm

struct fm_server {
    fm_index *h = nullptr;
    fm_server_params p{};
    uint32_t batch_reads_cap = 0;
    std::thread thr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<fm::Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<fm::Request>> all;
    bool stopping = false;
    uint64_t next_ticket = 1;
    // batch buffers (grown on demand, owned by the server thread)
    cudaStream_t stream = nullptr;
    uint8_t *d_codes = nullptr, *h_codes = nullptr;
    uint32_t *d_offs = nullptr, *h_offs = nullptr;
    uint32_t *d_counts = nullptr, *h_counts = nullptr;
    uint64_t *d_offsets = nullptr, *h_offsets = nullptr;
    uint32_t *d_pairs = nullptr, *h_pairs = nullptr;
    size_t cap_codes = 0, cap_reads = 0, cap_pairs = 0;
    // counters
    std::atomic<uint64_t> n_batches{0}, n_reads{0}, n_done{0}, busy_ns{0};
};

using namespace fm;

namespace {

void free_buffers(fm_server *s) {
    cudaFree(s->d_codes);
    cudaFree(s->d_offs);
    cudaFree(s->d_counts);
    cudaFree(s->d_offsets);
    cudaFree(s->d_pairs);
    cudaFreeHost(s->h_codes);
    cudaFreeHost(s->h_offs);
    cudaFreeHost(s->h_counts);
    cudaFreeHost(s->h_offsets);
    cudaFreeHost(s->h_pairs);
    s->d_codes = s->h_codes = nullptr;
    s->d_offs = s->h_offs = s->d_counts = s->h_counts = s->d_pairs = s->h_pairs = nullptr;
    s->d_offsets = s->h_offsets = nullptr;
    s->cap_codes = s->cap_reads = s->cap_pairs = 0;
}

// grow the batch buffers (device and pinned host) to hold the given sizes
int reserve(fm_server *s, size_t codes, size_t reads, size_t pairs) {
    const uint32_t st = s->p.strands;
    if (codes > s->cap_codes) {
        cudaFree(s->d_codes);
        cudaFreeHost(s->h_codes);
        s->d_codes = s->h_codes = nullptr;
        size_t c = codes + codes / 2 + 4096;
        if (cudaMalloc((void **)&s->d_codes, c) || cudaMallocHost((void **)&s->h_codes, c)) {
            cudaGetLastError();
            return FM_ENOMEM;
        }
        s->cap_codes = c;
    }
    if (reads > s->cap_reads) {
        cudaFree(s->d_offs);
        cudaFree(s->d_counts);
        cudaFree(s->d_offsets);
        cudaFreeHost(s->h_offs);
        cudaFreeHost(s->h_counts);
        cudaFreeHost(s->h_offsets);
        size_t r = reads + reads / 2 + 64;
        size_t q = r * st;
        if (cudaMalloc((void **)&s->d_offs, (r + 1) * 4) || cudaMalloc((void **)&s->d_counts, q * 4) ||
            cudaMalloc((void **)&s->d_offsets, (q + 1) * 8) ||
            cudaMallocHost((void **)&s->h_offs, (r + 1) * 4) ||
            cudaMallocHost((void **)&s->h_counts, q * 4) ||
            cudaMallocHost((void **)&s->h_offsets, (q + 1) * 8)) {
            cudaGetLastError();
            return FM_ENOMEM;
        }
        s->cap_reads = r;
    }
    if (pairs > s->cap_pairs) {
        cudaFree(s->d_pairs);
        cudaFreeHost(s->h_pairs);
        s->d_pairs = s->h_pairs = nullptr;
        size_t c = pairs + pairs / 2 + 4096;
        if (cudaMalloc((void **)&s->d_pairs, c * 8) || cudaMallocHost((void **)&s->h_pairs, c * 8)) {
            cudaGetLastError();
            return FM_ENOMEM;
        }
        s->cap_pairs = c;
    }
    return FM_OK;
}

void run_batch(fm_server *s, std::vector<std::shared_ptr<Request>> &batch);
void server_loop(fm_server *s);

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
    fm_server *s = new fm_server();
    s->h = h;
    s->p = q;
    // admission by device memory: reads per batch bounded by the frontier budget
    uint64_t by_mem = q.frontier_budget / (kScratchPerQuery * q.strands + 256);
    s->batch_reads_cap = (uint32_t)(by_mem < q.max_batch_reads ? by_mem : q.max_batch_reads);
    if (s->batch_reads_cap == 0) {
        delete s;
        return set_error(h, FM_EINVAL, "frontier budget below one read");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        delete s;
        return cuda_status(h, e, "cudaStreamCreate(server)");
    }
    // the interval and pair tables are built here, not inside the first batch's latency
    cudaSetDevice(h->device);
    int rc = ensure_kmer(h, s->stream);
    if (!rc) rc = ensure_pairs(h, s->stream);
    if (prev >= 0) cudaSetDevice(prev);
    if (rc) {
        cudaStreamDestroy(s->stream);
        delete s;
        return rc;
    }
    s->thr = std::thread(server_loop, s);
    *out = s;
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
    for (uint8_t c : r->codes)
        if (c > 3) return set_global_error(FM_EINVAL, "a read holds a code above 3");
    if (n_reads > s->batch_reads_cap)
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
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->thr.joinable()) s->thr.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->h->device);
    free_buffers(s);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
    return FM_OK;
}

}  // extern "C"

namespace {

// Search one batch and hand every request its own slice of the interval sets.
void run_batch(fm_server *s, std::vector<std::shared_ptr<Request>> &batch) {
    const uint64_t t0 = now_ns();
    const uint32_t st = s->p.strands;
    uint64_t n = 0, codes = 0;
    for (auto &r : batch) {
        r->t_start = t0;
        n += r->n_reads;
        codes += r->codes.size();
    }
    int rc = reserve(s, codes + 1, n + 1, 4 * n * st + 1024);
    uint64_t need = 0;
    if (!rc) {
        uint64_t pos = 0, rd = 0;
        s->h_offs[0] = 0;
        for (auto &r : batch) {
            memcpy(s->h_codes + pos, r->codes.data(), r->codes.size());
            for (uint32_t i = 1; i <= r->n_reads; ++i) s->h_offs[rd + i] = (uint32_t)(pos + r->offs[i]);
            pos += r->codes.size();
            rd += r->n_reads;
        }
        if (cudaMemcpyAsync(s->d_codes, s->h_codes, codes + 1, cudaMemcpyHostToDevice, s->stream) ||
            cudaMemcpyAsync(s->d_offs, s->h_offs, (n + 1) * 4, cudaMemcpyHostToDevice, s->stream))
            rc = cuda_status(s->h, cudaGetLastError(), "cudaMemcpyAsync(batch)");
    }
    if (!rc) {
        fm_search_params sp{};
        sp.z = batch[0]->z;
        sp.max_gaps = batch[0]->gaps;
        sp.strands = st;
        sp.kernel = s->p.kernel;
        // batch sizes change from one batch to the next: launch eagerly, no graph capture
        const bool graphs = s->h->use_graphs;
        s->h->use_graphs = false;
        rc = run_inexact(s->h, s->d_codes, s->d_offs, (uint32_t)n, &sp, s->d_counts, s->d_offsets,
                         s->d_pairs, s->cap_pairs, &need, s->stream);
        if (rc == FM_ETRUNC) {
            rc = reserve(s, 0, 0, need);
            if (!rc) rc = fetch_inexact(s->h, s->d_pairs, s->cap_pairs, s->stream);
        }
        s->h->use_graphs = graphs;
    }
    const uint64_t nq = n * st;
    if (!rc) {
        if (cudaMemcpyAsync(s->h_counts, s->d_counts, nq * 4, cudaMemcpyDeviceToHost, s->stream) ||
            cudaMemcpyAsync(s->h_offsets, s->d_offsets, (nq + 1) * 8, cudaMemcpyDeviceToHost, s->stream) ||
            (need && cudaMemcpyAsync(s->h_pairs, s->d_pairs, need * 8, cudaMemcpyDeviceToHost, s->stream)) ||
            cudaStreamSynchronize(s->stream))
            rc = cuda_status(s->h, cudaGetLastError(), "cudaMemcpyAsync(results)");
    }
    const uint64_t t1 = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    uint64_t q0 = 0;
    for (auto &r : batch) {
        const uint64_t rq = (uint64_t)r->n_reads * st;
        r->status = rc;
        if (!rc) {
            const uint64_t p0 = s->h_offsets[q0], p1 = s->h_offsets[q0 + rq];
            r->counts.assign(s->h_counts + q0, s->h_counts + q0 + rq);
            r->offsets.resize(rq + 1);
            for (uint64_t q = 0; q <= rq; ++q) r->offsets[q] = s->h_offsets[q0 + q] - p0;
            r->pairs.assign(s->h_pairs + 2 * p0, s->h_pairs + 2 * p1);
        } else {
            r->counts.assign(rq, 0);
            r->offsets.assign(rq + 1, 0);
        }
        r->batch_reads = (uint32_t)n;
        r->t_done = t1;
        r->done = true;
        q0 += rq;
    }
    s->n_batches += 1;
    s->n_reads += n;
    s->n_done += batch.size();
    s->busy_ns += t1 - t0;
}

void server_loop(fm_server *s) {
    cudaSetDevice(s->h->device);
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stopping || !s->pending.empty(); });
            if (s->pending.empty()) {
                if (s->stopping) break;
                continue;
            }
            // the oldest request fixes the mode; later requests of that mode join in arrival
            // order while the batch's read slots (bounded by the memory budget) last
            const uint32_t z = s->pending.front()->z, g = s->pending.front()->gaps;
            uint64_t reads = 0;
            for (auto it = s->pending.begin(); it != s->pending.end();) {
                auto &r = *it;
                if (r->z == z && r->gaps == g && reads + r->n_reads <= s->batch_reads_cap) {
                    reads += r->n_reads;
                    batch.push_back(r);
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        run_batch(s, batch);
        s->cv_done.notify_all();
    }
}

}  // namespace
