// Serving loop over a resident index (MICA, Section 2: the host keeps the
// accelerator busy with batches of reads while it handles the waiting and
// I/O; here requests of any size arrive while earlier ones are on the GPU).
//
// Continuous batching: a request is queued on submit.  Each worker thread
// (own CUDA stream and workspace) repeatedly admits queued requests in FIFO
// order while their reads fit the tick size and their device-memory estimate
// fits the server's budget, concatenates them into one batch (a "tick") and
// runs the whole search path on it: the tasks of all admitted requests share
// one persistent-kernel launch, so their work interleaves in the same warps.
// With two or more workers, one tick's search overlaps another's hit
// assembly and copies.  Results are split back per request.  Every wait has a
// bound; no device kernel waits on the host.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mica_internal.cuh"

namespace mica {
namespace {

using clock_t_ = std::chrono::steady_clock;

enum ReqState { PENDING = 0, RUNNING = 1, DONE = 2 };

struct Request {
    uint64_t id = 0;
    std::vector<uint32_t> words;
    std::vector<uint64_t> off;
    std::vector<uint16_t> len;
    std::vector<uint8_t> k;
    uint64_t n = 0;
    uint64_t est_bytes = 0;
    int state = PENDING;
    int rc = 0;
    mica_result *result = nullptr;
    clock_t_::time_point t_submit, t_done;
};

// device bytes one read may need in a tick: staged read + per-read outputs +
// intervals + hits at the usual density (the workspace grows on demand)
uint64_t estimate_bytes(uint64_t n, uint64_t words)
{
    return words * 4 + n * 160 + (1u << 20);
}

struct HostBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int reserve(size_t b)
    {
        if (b <= bytes && p) return 0;
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        if (cudaMallocHost(&p, std::max<size_t>(b, 4096)) != cudaSuccess) { cudaGetLastError(); return MICA_ENOMEM; }
        bytes = std::max<size_t>(b, 4096);
        return 0;
    }
    ~HostBuf() { if (p) cudaFreeHost(p); }
};

}  // namespace
}  // namespace mica

using namespace mica;

struct mica_server {
    mica_index *idx = nullptr;
    mica_server_params p{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_id = 1;
    uint64_t budget = 0, in_use = 0;
    bool stopping = false, paused = false;
    std::vector<std::thread> threads;
    mica_server_stats stats{};
};

namespace mica {
namespace {

int run_tick(mica_server *srv, std::vector<Request *> &tick, Workspace &ws, mica_stats &st, cudaStream_t s,
             HostBuf &stage)
{
    uint64_t n = 0, nw = 0;
    for (Request *r : tick) { n += r->n; nw += r->off[r->n]; }
    // stage the concatenated batch in pinned memory
    size_t in_bytes = nw * 4 + (n + 1) * 8 + n * 2 + n;
    if (int rc = stage.reserve(in_bytes + 64)) return rc;
    char *base = (char *)stage.p;
    uint32_t *hw = (uint32_t *)base;
    uint64_t *ho = (uint64_t *)(base + ((nw * 4 + 7) & ~7ull));
    uint16_t *hl = (uint16_t *)(ho + n + 1);
    uint8_t *hk = (uint8_t *)(hl + n);
    uint64_t wpos = 0, rpos = 0;
    for (Request *r : tick) {
        uint64_t rw = r->off[r->n];
        if (rw) memcpy(hw + wpos, r->words.data(), rw * 4);
        for (uint64_t i = 0; i < r->n; i++) ho[rpos + i] = r->off[i] + wpos;
        if (r->n) {
            memcpy(hl + rpos, r->len.data(), r->n * 2);
            memcpy(hk + rpos, r->k.data(), r->n);
        }
        wpos += rw;
        rpos += r->n;
    }
    ho[n] = wpos;
    int rc;
    if ((rc = dev_reserve(ws.reads_words, std::max<uint64_t>(nw, 1) * 4)) ||
        (rc = dev_reserve(ws.reads_off, (n + 1) * 8)) || (rc = dev_reserve(ws.reads_len, std::max<uint64_t>(n, 1) * 2)) ||
        (rc = dev_reserve(ws.reads_k, std::max<uint64_t>(n, 1))))
        return rc;
    if (nw) MICA_CUDA_TRY(cudaMemcpyAsync(ws.reads_words.p, hw, nw * 4, cudaMemcpyHostToDevice, s));
    MICA_CUDA_TRY(cudaMemcpyAsync(ws.reads_off.p, ho, (n + 1) * 8, cudaMemcpyHostToDevice, s));
    if (n) {
        MICA_CUDA_TRY(cudaMemcpyAsync(ws.reads_len.p, hl, n * 2, cudaMemcpyHostToDevice, s));
        MICA_CUDA_TRY(cudaMemcpyAsync(ws.reads_k.p, hk, n, cudaMemcpyHostToDevice, s));
    }
    ReadsView rd{(const uint32_t *)ws.reads_words.p, (const uint64_t *)ws.reads_off.p,
                 (const uint16_t *)ws.reads_len.p, (const uint8_t *)ws.reads_k.p, n};
    mica_align_params ap;
    ap.hit_cap = srv->p.hit_cap;
    ap.kernel = srv->p.kernel;
    ap.cuda_stream = s;
    uint64_t nh = 0;
    st.launches = 0;
    // ticks change shape every time: no graph capture
    if ((rc = align_on_device(srv->idx, ws, st, rd, ap, s, &nh, false))) return rc;
    // results back, split per request
    std::vector<uint64_t> total(std::max<uint64_t>(n, 1)), offs(n + 1);
    std::vector<mica_hit> hits(std::max<uint64_t>(nh, 1));
    if (n) MICA_CUDA_TRY(cudaMemcpyAsync(total.data(), ws.total.p, n * 8, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaMemcpyAsync(offs.data(), ws.hit_off.p, (n + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (nh) MICA_CUDA_TRY(cudaMemcpyAsync(hits.data(), ws.hits.p, nh * sizeof(mica_hit), cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    rpos = 0;
    for (Request *r : tick) {
        uint64_t h0 = offs[rpos], h1 = offs[rpos + r->n];
        mica_result *res = result_new(r->n, h1 - h0);
        if (!res) {
            r->rc = MICA_ENOMEM;
        } else {
            if (r->n) memcpy(res->total, total.data() + rpos, r->n * 8);
            for (uint64_t i = 0; i <= r->n; i++) res->offsets[i] = offs[rpos + i] - h0;
            if (h1 > h0) memcpy(res->hits, hits.data() + h0, (h1 - h0) * sizeof(mica_hit));
            r->result = res;
            r->rc = 0;
        }
        rpos += r->n;
    }
    return 0;
}

void worker_main(mica_server *srv)
{
    cudaSetDevice(srv->idx->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    Workspace ws;
    mica_stats st{};
    HostBuf stage;
    for (;;) {
        std::vector<Request *> tick;
        uint64_t charged = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                if (srv->stopping && srv->pending.empty()) break;
                if (!srv->paused && !srv->pending.empty()) {
                    uint64_t reads = 0;
                    while (!srv->pending.empty()) {
                        Request *r = srv->pending.front();
                        if (!tick.empty() && reads + r->n > srv->p.max_tick_reads) break;
                        if (srv->in_use + charged + r->est_bytes > srv->budget) break;   // wait for memory
                        srv->pending.pop_front();
                        r->state = RUNNING;
                        tick.push_back(r);
                        reads += r->n;
                        charged += r->est_bytes;
                    }
                    if (!tick.empty()) break;
                }
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
            if (tick.empty()) break;   // stopping and nothing queued
            srv->in_use += charged;
        }
        auto t0 = clock_t_::now();
        int rc = run_tick(srv, tick, ws, st, s, stage);
        auto t1 = clock_t_::now();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->in_use -= charged;
            srv->stats.ticks++;
            srv->stats.busy_s += std::chrono::duration<double>(t1 - t0).count();
            for (Request *r : tick) {
                if (rc) r->rc = rc;
                r->state = DONE;
                r->t_done = t1;
                if (r->rc) srv->stats.failed++;
                else { srv->stats.completed++; srv->stats.reads += r->n; }
            }
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
    free_workspace(ws);
    if (s) cudaStreamDestroy(s);
}

}  // namespace
}  // namespace mica

extern "C" {

void mica_server_params_default(mica_server_params *p)
{
    p->max_device_bytes = 0;
    p->max_tick_reads = 1u << 20;
    p->hit_cap = 1000;
    p->kernel = MICA_KERNEL_PERSISTENT;
    p->workers = 2;
    p->start_paused = 0;
}

int mica_server_start(mica_index *idx, const mica_server_params *params, mica_server **out)
{
    if (!idx || !out) return MICA_EINVAL;
    *out = nullptr;
    mica_server_params p;
    mica_server_params_default(&p);
    if (params) p = *params;
    if (p.kernel < MICA_KERNEL_PERSISTENT || p.kernel > MICA_KERNEL_PLAIN_BY_LENGTH) return MICA_EINVAL;
    if (p.workers <= 0) p.workers = 2;
    if (p.workers > 8) return MICA_EINVAL;
    if (p.max_tick_reads == 0) p.max_tick_reads = 1u << 20;
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    if (p.max_device_bytes == 0) {
        size_t fr = 0, tot = 0;
        MICA_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        p.max_device_bytes = fr / 2;
    }
    mica_server *srv = new mica_server();
    srv->idx = idx;
    srv->p = p;
    srv->budget = p.max_device_bytes;
    srv->paused = p.start_paused != 0;
    for (int i = 0; i < p.workers; i++) srv->threads.emplace_back(worker_main, srv);
    *out = srv;
    return 0;
}

int mica_server_submit(mica_server *srv, const uint32_t *packed_reads, const uint64_t *word_offsets,
                       const uint16_t *lengths, const uint8_t *k, uint64_t n_reads, uint64_t *req_id)
{
    if (!srv || !req_id || !word_offsets || (n_reads && (!packed_reads || !lengths || !k))) return MICA_EINVAL;
    if (n_reads >= (1ull << 31)) return MICA_EINVAL;
    if (int rc = validate_host_batch(srv->idx, word_offsets, lengths, k, n_reads)) return rc;
    Request *r = new Request();
    uint64_t nw = word_offsets[n_reads] - word_offsets[0];
    r->n = n_reads;
    r->words.assign(packed_reads + word_offsets[0], packed_reads + word_offsets[0] + nw);
    r->off.resize(n_reads + 1);
    for (uint64_t i = 0; i <= n_reads; i++) r->off[i] = word_offsets[i] - word_offsets[0];
    r->len.assign(lengths, lengths + n_reads);
    r->k.assign(k, k + n_reads);
    r->est_bytes = estimate_bytes(n_reads, nw);
    r->t_submit = clock_t_::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stopping) { delete r; return MICA_EBUSY; }
        if (r->est_bytes > srv->budget) { delete r; return MICA_ENOMEM; }   // can never be admitted
        r->id = srv->next_id++;
        srv->reqs[r->id] = r;
        srv->pending.push_back(r);
        srv->stats.submitted++;
        *req_id = r->id;
    }
    srv->cv_work.notify_one();
    return 0;
}

static int take_result(mica_server *srv, Request *r, mica_result **out, double *latency_ms)
{
    // caller holds srv->mu; r is DONE
    int rc = r->rc;
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (out) *out = r->result;
    else mica_result_free(r->result);
    srv->reqs.erase(r->id);
    delete r;
    return rc;
}

int mica_server_poll(mica_server *srv, uint64_t req_id, mica_result **out, double *latency_ms)
{
    if (!srv) return MICA_EINVAL;
    if (out) *out = nullptr;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return MICA_ENOTFOUND;
    if (it->second->state != DONE) return MICA_EBUSY;
    return take_result(srv, it->second, out, latency_ms);
}

int mica_server_wait(mica_server *srv, uint64_t req_id, uint32_t timeout_ms, mica_result **out,
                     double *latency_ms)
{
    if (!srv) return MICA_EINVAL;
    if (out) *out = nullptr;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto deadline = clock_t_::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = srv->reqs.find(req_id);
        if (it == srv->reqs.end()) return MICA_ENOTFOUND;
        if (it->second->state == DONE) return take_result(srv, it->second, out, latency_ms);
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = srv->reqs.find(req_id);
            if (it2 != srv->reqs.end() && it2->second->state == DONE)
                return take_result(srv, it2->second, out, latency_ms);
            return MICA_ETIMEOUT;
        }
    }
}

int mica_server_cancel(mica_server *srv, uint64_t req_id)
{
    if (!srv) return MICA_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return MICA_ENOTFOUND;
    Request *r = it->second;
    if (r->state != PENDING) return MICA_EBUSY;
    srv->pending.erase(std::find(srv->pending.begin(), srv->pending.end(), r));
    srv->reqs.erase(it);
    srv->stats.cancelled++;
    delete r;
    return 0;
}

void mica_server_resume(mica_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->paused = false;
    }
    srv->cv_work.notify_all();
}

int mica_server_get_stats(mica_server *srv, mica_server_stats *out)
{
    if (!srv || !out) return MICA_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    out->pending = srv->pending.size();
    out->device_bytes_in_use = srv->in_use;
    out->device_budget = srv->budget;
    return 0;
}

void mica_server_stop(mica_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        srv->paused = false;
        // queued requests that no tick has taken are dropped
        for (Request *r : srv->pending) {
            srv->reqs.erase(r->id);
            srv->stats.cancelled++;
            delete r;
        }
        srv->pending.clear();
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->threads) t.join();
    for (auto &kv : srv->reqs) {
        mica_result_free(kv.second->result);
        delete kv.second;
    }
    delete srv;
}

}  // extern "C"
