// Serving loop over a resident index (MICA, Section 2: the host keeps the
// accelerator busy with batches of reads while it handles the waiting and
// I/O; here requests of any size arrive while earlier ones are on the GPU).
//
// Continuous batching: a request is split on submit into chunks of at most
// chunk_reads reads and queued.  Each worker thread (own CUDA stream and
// workspace) repeatedly forms a "tick": it takes the next chunk of every
// queued request in arrival order, then their following chunks, round after
// round, while the tick's reads fit max_tick_reads and the device memory the
// search path needs for them fits the worker's share of the budget; the tick
// runs as one search launch, so the work of all its requests interleaves in
// the same warps.  A 1M-read request thus advances a chunk per tick beside
// the small requests that arrive meanwhile instead of holding a worker for
// its whole length, and with two or more workers one tick's search overlaps
// another's hit assembly and copies.  A request completes when its last chunk
// does; its result is its chunks' results in order, identical to aligning it
// alone.  Every wait has a bound; no device kernel waits on the host.
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

struct Request;

// Reads [r0, r0 + n) of a request, and their result once a tick ran them.
struct Chunk {
    Request *req = nullptr;
    uint64_t r0 = 0, n = 0, nw = 0;
    std::vector<uint64_t> total, off;   // off: n + 1 offsets from 0
    std::vector<mica_hit> hits;
};

struct Request {
    uint64_t id = 0;
    std::vector<uint32_t> words;
    std::vector<uint64_t> off;
    std::vector<uint16_t> len;
    std::vector<uint8_t> k;
    uint64_t n = 0;
    std::vector<Chunk> chunks;
    size_t next_chunk = 0;     // chunks handed to ticks
    size_t chunks_done = 0;
    int state = PENDING;
    int rc = 0;
    mica_result *result = nullptr;
    clock_t_::time_point t_submit, t_done;
};

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

// Device bytes a worker's workspace takes to run one tick of n reads held in
// nw packed words: the staged batch, the search's buffers and the post
// pipeline's at the sizes the first call reserves (hits at 4 per read +
// 65,536; a tick with more grows them).
int tick_workspace_bytes(const mica_index *idx, uint64_t n, uint64_t nw, uint64_t *bytes)
{
    uint64_t sb = 0;
    if (int rc = search_workspace_bytes(idx, n, &sb)) return rc;
    uint64_t iv_cap = std::min<uint64_t>(4 * n + 65536, 1ull << 30);
    *bytes = std::max<uint64_t>(nw, 1) * 4 + (n + 1) * 8 + 3 * std::max<uint64_t>(n, 1) + sb +
             post_workspace_bytes(n, iv_cap, 4 * n + 65536);
    return 0;
}

}  // namespace mica

using namespace mica;

struct mica_server {
    mica_index *idx = nullptr;
    mica_server_params p{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;            // requests with chunks not yet handed to a tick
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_id = 1;
    uint64_t budget = 0, share = 0;           // device bytes: all workers, one worker
    std::vector<uint64_t> ws_bytes;           // per worker: workspace its ticks have needed (grow-only)
    bool stopping = false, paused = false;
    std::vector<std::thread> threads;
    mica_server_stats stats{};
};

namespace mica {
namespace {

uint64_t in_use(const mica_server *srv)
{
    uint64_t t = 0;
    for (uint64_t b : srv->ws_bytes) t += b;
    return t;
}

// The request's result from its chunks, in order (caller holds no lock the
// workers need: called by the worker that finished the last chunk).
int assemble(Request *r)
{
    uint64_t nh = 0;
    for (const Chunk &c : r->chunks) nh += c.hits.size();
    mica_result *res = result_new(r->n, nh);
    if (!res) return MICA_ENOMEM;
    uint64_t h = 0;
    for (const Chunk &c : r->chunks) {
        if (c.n) memcpy(res->total + c.r0, c.total.data(), c.n * 8);
        for (uint64_t i = 0; i < c.n; i++) res->offsets[c.r0 + i] = h + c.off[i];
        if (!c.hits.empty()) memcpy(res->hits + h, c.hits.data(), c.hits.size() * sizeof(mica_hit));
        h += c.hits.size();
    }
    res->offsets[r->n] = h;
    r->result = res;
    for (Chunk &c : r->chunks) {
        std::vector<uint64_t>().swap(c.total);
        std::vector<uint64_t>().swap(c.off);
        std::vector<mica_hit>().swap(c.hits);
    }
    return 0;
}

int run_tick(mica_server *srv, std::vector<Chunk *> &tick, Workspace &ws, mica_stats &st, cudaStream_t s,
             HostBuf &stage, HostBuf &back)
{
    uint64_t n = 0, nw = 0;
    for (Chunk *c : tick) { n += c->n; nw += c->nw; }
    // stage the concatenated batch in pinned memory
    size_t in_bytes = nw * 4 + (n + 1) * 8 + n * 2 + n;
    if (int rc = stage.reserve(in_bytes + 64)) return rc;
    char *base = (char *)stage.p;
    uint32_t *hw = (uint32_t *)base;
    uint64_t *ho = (uint64_t *)(base + ((nw * 4 + 7) & ~7ull));
    uint16_t *hl = (uint16_t *)(ho + n + 1);
    uint8_t *hk = (uint8_t *)(hl + n);
    uint64_t wpos = 0, rpos = 0;
    for (Chunk *c : tick) {
        const Request *r = c->req;
        const uint64_t w0 = r->off[c->r0];
        if (c->nw) memcpy(hw + wpos, r->words.data() + w0, c->nw * 4);
        for (uint64_t i = 0; i < c->n; i++) ho[rpos + i] = r->off[c->r0 + i] - w0 + wpos;
        if (c->n) {
            memcpy(hl + rpos, r->len.data() + c->r0, c->n * 2);
            memcpy(hk + rpos, r->k.data() + c->r0, c->n);
        }
        wpos += c->nw;
        rpos += c->n;
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
    mica_align_params_default(&ap);
    ap.hit_cap = srv->p.hit_cap;
    ap.kernel = srv->p.kernel;
    ap.cuda_stream = s;
    uint64_t nh = 0;
    st.launches = 0;
    // ticks change shape every time: no graph capture
    if ((rc = align_on_device(srv->idx, ws, st, rd, ap, s, &nh, false))) return rc;
    // results back through pinned memory, split per chunk
    const size_t tb = (std::max<uint64_t>(n, 1) * 8 + 63) & ~63ull, ob = ((n + 1) * 8 + 63) & ~63ull;
    if ((rc = back.reserve(tb + ob + std::max<uint64_t>(nh, 1) * sizeof(mica_hit)))) return rc;
    uint64_t *total = (uint64_t *)back.p;
    uint64_t *offs = (uint64_t *)((char *)back.p + tb);
    mica_hit *hits = (mica_hit *)((char *)back.p + tb + ob);
    if (n) MICA_CUDA_TRY(cudaMemcpyAsync(total, ws.total.p, n * 8, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaMemcpyAsync(offs, ws.hit_off.p, (n + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (nh) MICA_CUDA_TRY(cudaMemcpyAsync(hits, ws.hits.p, nh * sizeof(mica_hit), cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    rpos = 0;
    for (Chunk *c : tick) {
        const uint64_t h0 = offs[rpos], h1 = offs[rpos + c->n];
        c->total.assign(total + rpos, total + rpos + c->n);
        c->off.resize(c->n + 1);
        for (uint64_t i = 0; i <= c->n; i++) c->off[i] = offs[rpos + i] - h0;
        c->hits.assign(hits + h0, hits + h1);
        rpos += c->n;
    }
    return 0;
}

// Under srv->mu: the next tick for a worker, taking chunks round-robin over
// the queued requests while reads and device memory fit.
void form_tick(mica_server *srv, std::vector<Chunk *> &tick, uint64_t &tick_bytes)
{
    uint64_t reads = 0, words = 0;
    tick_bytes = 0;
    for (bool progress = true; progress;) {
        progress = false;
        for (auto it = srv->pending.begin(); it != srv->pending.end();) {
            Request *r = *it;
            Chunk &c = r->chunks[r->next_chunk];
            uint64_t nb = 0;
            if (!tick.empty() && reads + c.n > srv->p.max_tick_reads) { ++it; continue; }
            if (tick_workspace_bytes(srv->idx, reads + c.n, words + c.nw, &nb) || nb > srv->share) {
                ++it;
                continue;
            }
            tick.push_back(&c);
            reads += c.n;
            words += c.nw;
            tick_bytes = nb;
            r->state = RUNNING;
            progress = true;
            if (++r->next_chunk == r->chunks.size()) it = srv->pending.erase(it);
            else ++it;
        }
    }
}

void worker_main(mica_server *srv, int wid)
{
    cudaSetDevice(srv->idx->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    Workspace ws;
    mica_stats st{};
    HostBuf stage, back;
    for (;;) {
        std::vector<Chunk *> tick;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                if (srv->stopping && srv->pending.empty()) break;
                if (!srv->paused && !srv->pending.empty()) {
                    uint64_t tb = 0;
                    form_tick(srv, tick, tb);
                    if (!tick.empty()) {
                        srv->ws_bytes[wid] = std::max(srv->ws_bytes[wid], tb);
                        break;
                    }
                }
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
            if (tick.empty()) break;   // stopping and nothing queued
        }
        srv->cv_work.notify_all();     // more chunks may be left for the other workers
        auto t0 = clock_t_::now();
        int rc = run_tick(srv, tick, ws, st, s, stage, back);
        // requests whose last chunk this was: assemble outside the lock
        std::vector<Request *> finished;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            for (Chunk *c : tick) {
                Request *r = c->req;
                if (rc) r->rc = rc;
                if (++r->chunks_done == r->chunks.size()) finished.push_back(r);
            }
        }
        for (Request *r : finished)
            if (!r->rc) r->rc = assemble(r);
        auto t1 = clock_t_::now();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->stats.ticks++;
            srv->stats.busy_s += std::chrono::duration<double>(t1 - t0).count();
            for (Request *r : finished) {
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
    p->kernel = MICA_KERNEL_BIDIRECTIONAL;
    p->workers = 2;
    p->start_paused = 0;
    p->chunk_reads = 1u << 18;
}

int mica_server_workspace_bytes(const mica_index *idx, uint64_t n_reads, uint64_t n_words, uint64_t *bytes)
{
    if (!idx || !bytes) return MICA_EINVAL;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    return tick_workspace_bytes(idx, n_reads, n_words, bytes);
}

int mica_server_start(mica_index *idx, const mica_server_params *params, mica_server **out)
{
    if (!idx || !out) return MICA_EINVAL;
    *out = nullptr;
    mica_server_params p;
    mica_server_params_default(&p);
    if (params) p = *params;
    if (p.kernel < MICA_KERNEL_PERSISTENT || p.kernel > MICA_KERNEL_BIDIRECTIONAL) return MICA_EINVAL;
    if (p.workers <= 0) p.workers = 2;
    if (p.workers > 8) return MICA_EINVAL;
    if (p.max_tick_reads == 0) p.max_tick_reads = 1u << 20;
    if (p.chunk_reads == 0) p.chunk_reads = 1u << 18;
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
    srv->share = p.max_device_bytes / (uint64_t)p.workers;
    srv->ws_bytes.assign(p.workers, 0);
    srv->paused = p.start_paused != 0;
    for (int i = 0; i < p.workers; i++) srv->threads.emplace_back(worker_main, srv, i);
    *out = srv;
    return 0;
}

int mica_server_submit(mica_server *srv, const uint32_t *packed_reads, const uint64_t *word_offsets,
                       const uint16_t *lengths, const uint8_t *k, uint64_t n_reads, uint64_t *req_id)
{
    if (!srv || !req_id || !word_offsets || (n_reads && (!packed_reads || !lengths || !k))) return MICA_EINVAL;
    if (n_reads >= (1ull << 31)) return MICA_EINVAL;
    if (int rc = validate_host_batch(srv->idx, word_offsets, lengths, k, n_reads)) return rc;
    DeviceGuard g(srv->idx->device);
    MICA_CUDA_TRY(cudaSetDevice(srv->idx->device));
    // a tick of one read must fit a worker's share, or the request could never run
    uint64_t one = 0;
    if (int rc = tick_workspace_bytes(srv->idx, 1, MICA_MAX_READ_LEN / 16, &one)) return rc;
    if (one > srv->share) return MICA_ENOMEM;
    Request *r = new Request();
    uint64_t nw = word_offsets[n_reads] - word_offsets[0];
    r->n = n_reads;
    r->words.assign(packed_reads + word_offsets[0], packed_reads + word_offsets[0] + nw);
    r->off.resize(n_reads + 1);
    for (uint64_t i = 0; i <= n_reads; i++) r->off[i] = word_offsets[i] - word_offsets[0];
    r->len.assign(lengths, lengths + n_reads);
    r->k.assign(k, k + n_reads);
    // chunks: at most chunk_reads reads, and no more than a worker's share holds
    uint64_t cmax = std::max<uint64_t>(1, std::min<uint64_t>(srv->p.chunk_reads, srv->p.max_tick_reads));
    for (uint64_t b = 0; b == 0 || cmax > 1;) {
        if (int rc = tick_workspace_bytes(srv->idx, cmax, cmax * (MICA_MAX_READ_LEN / 16), &b)) { delete r; return rc; }
        if (b <= srv->share) break;
        cmax /= 2;
    }
    for (uint64_t r0 = 0; r0 < n_reads || (n_reads == 0 && r->chunks.empty()); r0 += cmax) {
        Chunk c;
        c.req = r;
        c.r0 = r0;
        c.n = std::min<uint64_t>(cmax, n_reads - r0);
        c.nw = r->off[r0 + c.n] - r->off[r0];
        r->chunks.push_back(std::move(c));
        if (n_reads == 0) break;
    }
    r->t_submit = clock_t_::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stopping) { delete r; return MICA_EBUSY; }
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
    if (r->state != PENDING) return MICA_EBUSY;   // a chunk is on the GPU or done
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
    out->device_bytes_in_use = in_use(srv);
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
        // queued requests that no tick has taken are dropped; those with a
        // chunk on the GPU already are finished by the workers
        for (auto it = srv->pending.begin(); it != srv->pending.end();) {
            Request *r = *it;
            if (r->state != PENDING) { ++it; continue; }
            srv->reqs.erase(r->id);
            srv->stats.cancelled++;
            delete r;
            it = srv->pending.erase(it);
        }
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
