// The extern "C" boundary of libmica_gb300 (declared in include/mica.h).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "host_parallel.h"
#include "mica_internal.cuh"

namespace mica {

static thread_local char g_last_error[512];

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

static thread_local char g_last_internal[256];

void set_last_internal(const char *msg)
{
    snprintf(g_last_internal, sizeof(g_last_internal), "%s", msg);
}

int dev_reserve(DevBuf &b, size_t bytes)
{
    if (bytes <= b.bytes && b.p) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        b.p = nullptr;
        return MICA_ENOMEM;
    }
    b.bytes = want;
    return 0;
}

// ---- host results in pinned memory ----
//
// A host result's arrays live in one page-locked block, so the device writes
// them by DMA at the link's speed (a copy into pageable memory goes through a
// staging buffer and runs several times slower).  Blocks come from a
// process-wide pool of size classes (steps of a quarter of a power of two);
// a freed result's block returns to the pool, which keeps up to 1 GiB of idle
// blocks and releases the rest.  When page-locked memory cannot be had, the
// block is ordinary heap memory.
namespace {

constexpr uint32_t RESULT_MAGIC = 0x4d525331u;   // "MRS1"
constexpr size_t PIN_IDLE_MAX = 1ull << 30;

struct ResultBlock {
    mica_result pub;     // first member: a mica_result * is a ResultBlock *
    uint32_t magic;
    int pinned;
    void *mem;
    size_t bytes;
};

std::mutex g_pin_mu;
std::vector<std::pair<size_t, void *>> g_pin_idle;
size_t g_pin_idle_bytes = 0;

size_t pin_class(size_t bytes)
{
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    if (c <= 16384) return c;
    size_t q = c / 8;                          // quarter steps of the half below c
    size_t r = c / 2;
    while (r < bytes) r += q;
    return r;
}

void *pin_get(size_t bytes, size_t &got, int &pinned)
{
    got = pin_class(bytes);
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        for (size_t i = 0; i < g_pin_idle.size(); i++)
            if (g_pin_idle[i].first == got) {
                void *p = g_pin_idle[i].second;
                g_pin_idle[i] = g_pin_idle.back();
                g_pin_idle.pop_back();
                g_pin_idle_bytes -= got;
                pinned = 1;
                return p;
            }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, got) == cudaSuccess) {
        pinned = 1;
        return p;
    }
    cudaGetLastError();
    pinned = 0;
    got = bytes;
    return malloc(std::max<size_t>(bytes, 1));
}

void pin_put(void *p, size_t bytes)
{
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (g_pin_idle_bytes + bytes <= PIN_IDLE_MAX) {
            g_pin_idle.emplace_back(bytes, p);
            g_pin_idle_bytes += bytes;
            return;
        }
    }
    cudaFreeHost(p);
}

}  // namespace

mica_result *result_new(uint64_t n_reads, uint64_t n_hits)
{
    ResultBlock *b = (ResultBlock *)calloc(1, sizeof(ResultBlock));
    if (!b) return nullptr;
    size_t tb = (std::max<uint64_t>(n_reads, 1) * 8 + 63) & ~63ull;
    size_t ob = ((n_reads + 1) * 8 + 63) & ~63ull;
    size_t hb = std::max<uint64_t>(n_hits, 1) * sizeof(mica_hit);
    b->mem = pin_get(tb + ob + hb, b->bytes, b->pinned);
    if (!b->mem) { free(b); return nullptr; }
    b->magic = RESULT_MAGIC;
    b->pub.n_reads = n_reads;
    b->pub.total = (uint64_t *)b->mem;
    b->pub.offsets = (uint64_t *)((char *)b->mem + tb);
    b->pub.hits = (mica_hit *)((char *)b->mem + tb + ob);
    return &b->pub;
}

void dev_release(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

void free_workspace(Workspace &w)
{
    DevBuf *all[] = {&w.ctl, &w.iv, &w.iv_sorted, &w.iv_cnt, &w.iv_off, &w.total, &w.keep, &w.hit_off,
                     &w.hits, &w.spill, &w.big, &w.scan_tmp, &w.reads_words, &w.reads_off, &w.reads_len,
                     &w.reads_k, &w.spill2, &w.lenlist, &w.lb, &w.spill_seq, &w.deep, &w.redo, &w.frontier};
    for (DevBuf *b : all) dev_release(*b);
    for (auto &e : w.ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    for (auto &e : w.kev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    if (w.gexec) { cudaGraphExecDestroy(w.gexec); w.gexec = nullptr; }
    if (w.gstream) { cudaStreamDestroy(w.gstream); w.gstream = nullptr; }
    if (w.pin_tmpl) { cudaFreeHost(w.pin_tmpl); w.pin_tmpl = nullptr; }
    if (w.pin_status) { cudaFreeHost(w.pin_status); w.pin_status = nullptr; }
}

static int validate_params(const mica_index_params &p)
{
    if (p.kmer_q < 1 || p.kmer_q > MAX_Q) return MICA_EINVAL;
    if (p.sa_sample < 1 || p.sa_sample > 256) return MICA_EINVAL;
    if (p.lower_bounds > 1) return MICA_EINVAL;
    if (p.full_sa > 1) return MICA_EINVAL;
    return 0;
}

// ASCII genome -> base codes (host), rejecting anything but A/C/G/T.
static int encode_genome(const uint8_t *acgt, uint64_t len, std::vector<uint8_t> &codes)
{
    static uint8_t lut[256];
    static std::once_flag once;
    std::call_once(once, [] {
        memset(lut, 0xff, sizeof(lut));
        lut['A'] = lut['a'] = 0; lut['C'] = lut['c'] = 1;
        lut['G'] = lut['g'] = 2; lut['T'] = lut['t'] = 3;
    });
    codes.resize(len);
    for (uint64_t i = 0; i < len; i++) {
        uint8_t c = lut[acgt[i]];
        if (c > 3) return MICA_EINVAL;
        codes[i] = c;
    }
    return 0;
}


// ---- index file ----

static const char MAGIC[8] = {'M', 'I', 'C', 'A', 'I', 'D', 'X', '1'};

struct FileHeader {
    char magic[8];
    uint32_t version, kmer_q, sa_sample;
    uint32_t flags;   // version 5: bit 0 = the index keeps the whole suffix array, its inverse and the text
                      // (rebuilt at load, not stored); 0 before version 5
    uint64_t n, dollar_row;
    uint64_t C[5];
    uint64_t n_occ_blocks, n_super, n_mark_blocks, n_samples, table_len;
    uint32_t nshort, short_pad[MAX_Q], short_len[MAX_Q];
};

// Version 3 follows the header with this block; the reversed genome's
// occurrence blocks and superblocks (same counts as the genome's) follow the
// genome's arrays when has_rev is 1.
struct FileHeaderRev {
    uint32_t has_rev, rev_dollar_row;
    uint64_t rev_C[5];
};

// Version 4 adds this block after FileHeaderRev; when has_rev_table is 1 the
// reversed genome's q-mer table (table_len uint32) follows its superblocks.
struct FileHeaderRevTable {
    uint32_t has_rev_table, rev_nshort;
    uint32_t rev_short_pad[MAX_Q], rev_short_len[MAX_Q];
};

static int write_array(FILE *f, const DevBuf &b, uint64_t bytes)
{
    std::vector<char> h(std::min<uint64_t>(bytes, 1ull << 26));
    for (uint64_t off = 0; off < bytes; off += h.size()) {
        uint64_t c = std::min<uint64_t>(h.size(), bytes - off);
        MICA_CUDA_TRY(cudaMemcpy(h.data(), (const char *)b.p + off, c, cudaMemcpyDeviceToHost));
        if (fwrite(h.data(), 1, c, f) != c) return MICA_EIO;
    }
    return 0;
}

static int read_array(FILE *f, DevBuf &b, uint64_t bytes)
{
    if (int rc = dev_reserve(b, std::max<uint64_t>(bytes, 4))) return rc;
    std::vector<char> h(std::min<uint64_t>(std::max<uint64_t>(bytes, 1), 1ull << 26));
    for (uint64_t off = 0; off < bytes; off += h.size()) {
        uint64_t c = std::min<uint64_t>(h.size(), bytes - off);
        if (fread(h.data(), 1, c, f) != c) return MICA_EIO;
        MICA_CUDA_TRY(cudaMemcpy((char *)b.p + off, h.data(), c, cudaMemcpyHostToDevice));
    }
    return 0;
}

// ---- align orchestration ----

// Prefetching the next round's blocks pays when they are not L2 hits.
static bool use_prefetch(const mica_index *idx)
{
    if (idx->tuning.prefetch >= 0) return idx->tuning.prefetch == 1;
    return idx->n_occ_blocks * 32 > (96ull << 20);
}

// The persistent pipeline as one CUDA graph per batch shape: captured the
// first time a shape (input addresses, read count, cap, kernel shape, buffer
// addresses) is seen, then replayed with a single host synchronisation.  Any
// overflow, error or read with more than 4096 listed hits sets done = false
// and the caller runs the regular path, which recomputes the batch.
//
// align_graph_launch queues the replay on s and returns (launched = false when
// the batch cannot be captured); align_graph_finish waits for it and reads its
// status.
static int align_graph_launch(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
                              const mica_align_params &p, cudaStream_t s, bool &launched)
{
    launched = false;
    uint64_t n = rd.n;
    if (!w.pin_tmpl) {
        MICA_CUDA_TRY(cudaMallocHost(&w.pin_tmpl, 256));
        MICA_CUDA_TRY(cudaMallocHost(&w.pin_status, 256));
    }
    if (!w.gstream) MICA_CUDA_TRY(cudaStreamCreateWithFlags(&w.gstream, cudaStreamNonBlocking));
    SearchCtl tmpl;
    int grid = 0, shape = 0, rc;
    const bool bidir = p.kernel == MICA_KERNEL_BIDIRECTIONAL;
    if (bidir) {
        if ((rc = prepare_bidir(idx, w, n, tmpl, grid))) return rc;
        shape = (1 << 8) | bidir_shape_index(idx);   // the bidirectional kernel and its shape, in the key
    } else if ((rc = prepare_persistent(idx, w, n, idx->tuning.shape, tmpl, grid, shape))) {
        return rc;
    }
    w.hit_capacity = std::max<uint64_t>(w.hit_capacity, 4 * n + 65536);
    if ((rc = reserve_post(w, n, w.iv_cap, w.hit_capacity))) return rc;
    memcpy(w.pin_tmpl, &tmpl, sizeof(tmpl));
    const bool prune = p.prune && idx->has_rev;
    const bool prefetch = use_prefetch(idx);
    // every input, size and workspace buffer the captured kernels use: a
    // buffer grown by any other call since the capture forces a new capture
    uint64_t key[GRAPH_KEY] = {(uint64_t)rd.words, (uint64_t)rd.word_off, (uint64_t)rd.len, (uint64_t)rd.k, n,
                               p.hit_cap, (uint64_t)shape | ((uint64_t)prune << 32) | ((uint64_t)prefetch << 33),
                               (uint64_t)grid,
                               (uint64_t)w.ctl.p, (uint64_t)w.iv.p, (uint64_t)w.iv_cnt.p, (uint64_t)w.spill.p,
                               (uint64_t)w.lb.p, (uint64_t)w.iv_sorted.p, (uint64_t)w.iv_off.p,
                               (uint64_t)w.total.p, (uint64_t)w.keep.p, (uint64_t)w.hit_off.p, (uint64_t)w.hits.p,
                               (uint64_t)w.big.p, (uint64_t)w.scan_tmp.p, w.hit_capacity, (uint64_t)w.iv_cap,
                               (uint64_t)w.spill_cap, (uint64_t)w.spill_seq.p, (uint64_t)w.deep.p,
                               (uint64_t)p.report | ((uint64_t)idx->tuning.bidir_budget << 32),
                               ((uint64_t)idx->idle_limit << 32) | idx->spin_limit,
                               (uint64_t)w.frontier.p, (uint64_t)w.redo.p, (uint64_t)idx->tuning.bidir_verify};
    if (!w.gexec || memcmp(key, w.gkey, sizeof(key)) != 0) {
        if (w.gexec) { cudaGraphExecDestroy(w.gexec); w.gexec = nullptr; }
        uint64_t L = 0;
        MICA_CUDA_TRY(cudaStreamBeginCapture(w.gstream, cudaStreamCaptureModeThreadLocal));
        int crc = bidir ? enqueue_bidir_graph(idx, w, rd, grid, (const SearchCtl *)w.pin_tmpl, w.gstream, L)
                        : enqueue_persistent(idx, w, rd, shape, grid, (const SearchCtl *)w.pin_tmpl, prune, prefetch,
                                             w.gstream, L);
        if (!crc) crc = enqueue_post_device(idx, w, rd, p.hit_cap, p.report, w.hit_capacity, w.gstream,
                                            w.pin_status, L);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(w.gstream, &g);
        if (crc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return 0;   // capture not possible: the regular path runs
        }
        e = cudaGraphInstantiate(&w.gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { w.gexec = nullptr; cudaGetLastError(); return 0; }
        memcpy(w.gkey, key, sizeof(key));
        st.graph_captures++;
        w.glaunches = L;
    }
    MICA_CUDA_TRY(cudaEventRecord(w.ev[0], s));
    MICA_CUDA_TRY(cudaGraphLaunch(w.gexec, s));
    MICA_CUDA_TRY(cudaEventRecord(w.ev[2], s));
    w.g_grid = grid;
    launched = true;
    return 0;
}

static int align_graph_finish(Workspace &w, mica_stats &st, const ReadsView &rd, const mica_align_params &p,
                              uint64_t *nh, bool &done)
{
    done = false;
    const uint64_t n = rd.n;
    const bool bidir = p.kernel == MICA_KERNEL_BIDIRECTIONAL;
    const int grid = w.g_grid;
    MICA_CUDA_TRY(cudaEventSynchronize(w.ev[2]));
    SearchCtl out;
    memcpy(&out, w.pin_status, sizeof(out));
    const char *stp = (const char *)w.pin_status + sizeof(SearchCtl);
    uint64_t nhits, steps;
    unsigned int cnts[2];
    memcpy(&nhits, stp, 8);
    memcpy(&steps, stp + 8, 8);
    memcpy(cnts, stp + 16, 8);
    if (out.error & ERR_TIMEOUT) return MICA_ETIMEOUT;
    if (out.error) {
        // let the regular path grow the buffers and recompute
        return 0;
    }
    if (bidir && (out.redo_reads || out.fr_count)) {
        // reads given up, or nodes still exported after the captured rounds:
        // the regular path runs the rounds to the end and searches the given-up
        // reads again
        w.bd_redo_seen = true;
        return 0;
    }
    if (nhits > w.hit_capacity) { w.hit_capacity = 2 * nhits; return 0; }
    if (cnts[1]) return 0;   // a read above the shared-memory sort size
    st.tasks = 2 * n;
    st.seeds = out.seeds;
    st.nodes = out.nodes;
    st.rank_blocks = out.rank_blocks;
    st.intervals = out.iv_count;
    st.spills = out.spills;
    st.warp_rounds = out.rounds;
    st.lane_ops = out.lane_ops;
    st.rounds_multi = out.rounds_kind[0];
    st.rounds_single = out.rounds_kind[1];
    st.rounds_seed = out.rounds_kind[2];
    st.lb_steps = out.lb_steps;
    st.lb_dead_tasks = out.lb_dead;
    st.queue_wait_ns = out.wait_queue_ns;
    st.idle_wait_ns = out.wait_idle_ns;
    st.overflow_moves = out.deep_moves;
    st.verified = out.verified;
    st.verify_bytes = out.verify_bytes;
    st.verify_sectors = out.verify_sectors;
    st.grid_ctas = (uint64_t)grid;
    st.located = nhits;
    st.lf_steps = steps;
    st.launches += w.glaunches;
    st.graph_replays++;
    st.kernel_ms = elapsed_ms(w.kev[0], w.kev[1]);
    st.search_ms = st.kernel_ms;
    st.total_ms = elapsed_ms(w.ev[0], w.ev[2]);
    *nh = nhits;
    done = true;
    return 0;
}

static int align_graph(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
                       const mica_align_params &p, cudaStream_t s, uint64_t *nh, bool &done)
{
    done = false;
    bool launched = false;
    if (int rc = align_graph_launch(idx, w, st, rd, p, s, launched)) return rc;
    return launched ? align_graph_finish(w, st, rd, p, nh, done) : 0;
}

// The kernel a call runs: an index without the reversed genome's table runs
// the persistent kernel instead of the bidirectional one.
static mica_align_params effective_params(const mica_index *idx, const mica_align_params &p_in)
{
    mica_align_params p = p_in;
    if (p.kernel == MICA_KERNEL_BIDIRECTIONAL && !bidir_available(idx)) p.kernel = MICA_KERNEL_PERSISTENT;
    return p;
}

static int create_events(Workspace &w)
{
    for (auto &e : w.ev)
        if (!e) MICA_CUDA_TRY(cudaEventCreate(&e));
    for (auto &e : w.kev)
        if (!e) MICA_CUDA_TRY(cudaEventCreate(&e));
    return 0;
}

// May the call run as a captured graph?  Best-stratum deepening has host
// steps between its passes; a bidirectional batch that gave reads up needs
// host steps after the kernel, so after one did, this workspace runs
// bidirectional calls uncaptured.  (The budget that gives reads up is part of
// the captured kernel's arguments.)
static bool graph_eligible(const Workspace &w, const mica_align_params &p, const ReadsView &rd)
{
    const bool deepen = p.report == MICA_REPORT_BEST_STRATUM && p.kernel == MICA_KERNEL_PERSISTENT;
    const bool graphable = p.kernel == MICA_KERNEL_PERSISTENT ||
                           (p.kernel == MICA_KERNEL_BIDIRECTIONAL && !w.bd_redo_seen);
    return !deepen && graphable && rd.n > 0;
}

int align_on_device(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
                    const mica_align_params &p_in, cudaStream_t s, uint64_t *nh, bool allow_graph)
{
    const mica_align_params p = effective_params(idx, p_in);
    if (int rc = create_events(w)) return rc;
    uint64_t launches = st.launches;   // the batch check already counted
    st = mica_stats{};
    st.launches = launches;
    const bool deepen = p.report == MICA_REPORT_BEST_STRATUM && p.kernel == MICA_KERNEL_PERSISTENT && rd.n > 0;
    if (allow_graph && graph_eligible(w, p, rd)) {
        bool done = false;
        if (int rc = align_graph(idx, w, st, rd, p, s, nh, done)) return rc;
        if (done) return 0;
        st.graph_fallbacks++;
    }
    MICA_CUDA_TRY(cudaEventRecord(w.ev[0], s));
    SearchConfig cfg{};
    cfg.kernel = p.kernel;
    cfg.shape = idx->tuning.shape;
    cfg.plain_block = idx->tuning.plain_block ? (int)idx->tuning.plain_block : 128;
    cfg.plain_budget = idx->tuning.plain_budget ? idx->tuning.plain_budget : (1u << 16);
    cfg.prune = p.prune && idx->has_rev;
    cfg.prefetch = use_prefetch(idx);
    for (uint32_t c = 0; c < LEN_CLASSES; c++)
        cfg.plain_block_len[c] = idx->tuning.plain_block_len[c] ? (int)idx->tuning.plain_block_len[c] : cfg.plain_block;
    int rc;
    if (p.kernel == MICA_KERNEL_BIDIRECTIONAL) {
        rc = run_search_bidir(idx, w, st, rd, s);
        if (rc == BIDIR_FALLBACK) {
            // a warp's overflow stack filled: the one-directional search (same result)
            st.retries++;
            cfg.kernel = MICA_KERNEL_PERSISTENT;
            rc = run_search(idx, w, st, rd, cfg, s);
        }
    } else {
        rc = deepen ? run_search_stratum(idx, w, st, rd, cfg, s) : run_search(idx, w, st, rd, cfg, s);
        if (rc == STRATUM_FALLBACK) {
            rc = run_search(idx, w, st, rd, cfg, s);   // exhaustive search, filtered after
        }
    }
    if (rc) return rc;
    MICA_CUDA_TRY(cudaEventRecord(w.ev[1], s));
    if ((rc = run_post(idx, w, st, rd, p.hit_cap, p.report, s, nh))) return rc;
    MICA_CUDA_TRY(cudaEventRecord(w.ev[2], s));
    MICA_CUDA_TRY(cudaEventSynchronize(w.ev[2]));
    st.search_ms = elapsed_ms(w.ev[0], w.ev[1]);
    st.kernel_ms = elapsed_ms(w.kev[0], w.kev[1]);
    st.total_ms = elapsed_ms(w.ev[0], w.ev[2]);
    return 0;
}

}  // namespace mica

using namespace mica;

extern "C" {

const char *mica_strerror(int code)
{
    switch (code) {
    case MICA_OK: return "ok";
    case MICA_EINVAL: return "invalid argument";
    case MICA_ENOMEM: return "out of memory";
    case MICA_EIO: return "index file I/O error or malformed file";
    case MICA_ECUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case MICA_ETIMEOUT: return "bounded wait expired";
    case MICA_EINTERNAL: return g_last_internal[0] ? g_last_internal : "internal capacity retry did not converge";
    case MICA_EBUSY: return "request not finished";
    case MICA_ENOTFOUND: return "unknown request";
    default: return "unknown error";
    }
}

void mica_index_params_default(mica_index_params *p)
{
    p->kmer_q = 12;
    p->sa_sample = 16;
    p->lower_bounds = 1;
    p->full_sa = 1;
}

void mica_align_params_default(mica_align_params *p)
{
    p->hit_cap = 1000;
    p->kernel = MICA_KERNEL_BIDIRECTIONAL;
    p->cuda_stream = nullptr;
    p->prune = 1;
    p->report = MICA_REPORT_ALL;
}

int mica_index_build_resident(const uint8_t *genome_acgt, uint64_t len, const mica_index_params *params,
                              int device, mica_index **out)
{
    if (!out || (!genome_acgt && len)) return MICA_EINVAL;
    *out = nullptr;
    mica_index_params p;
    mica_index_params_default(&p);
    if (params) p = *params;
    if (int rc = validate_params(p)) return rc;
    if (len + 1 >= (1ull << 32)) return MICA_EINVAL;
    std::vector<uint8_t> codes;
    if (int rc = encode_genome(genome_acgt, len, codes)) return rc;
    DeviceGuard g(device);
    MICA_CUDA_TRY(cudaSetDevice(device));
    mica_index *idx = new mica_index();
    idx->device = device;
    DevBuf dcodes;
    int rc = dev_reserve(dcodes, std::max<uint64_t>(len, 1));
    if (!rc && len) {
        cudaError_t e = cudaMemcpy(dcodes.p, codes.data(), len, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { set_last_cuda_error(e, "cudaMemcpy genome", __FILE__, __LINE__); rc = MICA_ECUDA; }
    }
    if (!rc) rc = build_index_from_codes((const uint8_t *)dcodes.p, len, p, idx, 0);
    dev_release(dcodes);
    if (rc) { mica_index_free(idx); return rc; }
    *out = idx;
    return 0;
}

int mica_index_build(const uint8_t *genome_acgt, uint64_t len, const mica_index_params *params,
                     const char *out_path)
{
    if (!out_path) return MICA_EINVAL;
    int dev = 0;
    MICA_CUDA_TRY(cudaGetDevice(&dev));
    mica_index *idx = nullptr;
    int rc = mica_index_build_resident(genome_acgt, len, params, dev, &idx);
    if (rc) return rc;
    rc = mica_index_save(idx, out_path);
    mica_index_free(idx);
    return rc;
}

int mica_index_save(const mica_index *idx, const char *path)
{
    if (!idx || !path) return MICA_EINVAL;
    DeviceGuard g(idx->device);
    FILE *f = fopen(path, "wb");
    if (!f) return MICA_EIO;
    FileHeader h{};
    memcpy(h.magic, MAGIC, 8);
    h.version = 5;
    h.kmer_q = idx->params.kmer_q;
    h.sa_sample = idx->params.sa_sample;
    h.flags = idx->has_full_sa ? 1u : 0u;
    h.n = idx->n;
    h.dollar_row = idx->view.dollar_row;
    for (int c = 0; c < 5; c++) h.C[c] = idx->view.C[c];
    h.n_occ_blocks = idx->n_occ_blocks;
    h.n_super = idx->n_super;
    h.n_mark_blocks = idx->n_mark_blocks;
    h.n_samples = idx->n_samples;
    h.table_len = idx->table_len;
    h.nshort = idx->view.nshort;
    for (uint32_t t = 0; t < MAX_Q; t++) {
        h.short_pad[t] = idx->view.short_pad[t];
        h.short_len[t] = idx->view.short_len[t];
    }
    FileHeaderRev hr{};
    hr.has_rev = idx->has_rev ? 1u : 0u;
    hr.rev_dollar_row = idx->view.rev.dollar_row;
    for (int c = 0; c < 5; c++) hr.rev_C[c] = idx->view.rev.C[c];
    FileHeaderRevTable ht{};
    ht.has_rev_table = idx->view.rev.table ? 1u : 0u;
    ht.rev_nshort = idx->view.rev.nshort;
    for (uint32_t t = 0; t < MAX_Q; t++) {
        ht.rev_short_pad[t] = idx->view.rev.short_pad[t];
        ht.rev_short_len[t] = idx->view.rev.short_len[t];
    }
    int rc = fwrite(&h, sizeof(h), 1, f) == 1 ? 0 : MICA_EIO;
    if (!rc && fwrite(&hr, sizeof(hr), 1, f) != 1) rc = MICA_EIO;
    if (!rc && fwrite(&ht, sizeof(ht), 1, f) != 1) rc = MICA_EIO;
    if (!rc) rc = write_array(f, idx->occ, h.n_occ_blocks * 32);
    if (!rc) rc = write_array(f, idx->super, h.n_super * 16);
    if (!rc) rc = write_array(f, idx->marks, h.n_mark_blocks * 64);
    if (!rc) rc = write_array(f, idx->samples, h.n_samples * 4);
    if (!rc) rc = write_array(f, idx->table, h.table_len * 4);
    if (!rc && idx->has_rev) rc = write_array(f, idx->rocc, h.n_occ_blocks * 32);
    if (!rc && idx->has_rev) rc = write_array(f, idx->rsuper, h.n_super * 16);
    if (!rc && ht.has_rev_table) rc = write_array(f, idx->rtable, h.table_len * 4);
    if (fclose(f) != 0 && !rc) rc = MICA_EIO;
    return rc;
}

int mica_index_load(const char *path, int device, mica_index **out)
{
    if (!path || !out) return MICA_EINVAL;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return MICA_EIO;
    FileHeader h{};
    FileHeaderRev hr{};
    FileHeaderRevTable ht{};
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, MAGIC, 8) != 0 || h.version < 2 || h.version > 5 || (h.version < 5 ? h.flags != 0 : h.flags > 1) ||
        (h.version >= 3 && (fread(&hr, sizeof(hr), 1, f) != 1 || hr.has_rev > 1)) ||
        (h.version >= 4 && (fread(&ht, sizeof(ht), 1, f) != 1 || ht.has_rev_table > hr.has_rev ||
                            (ht.has_rev_table && ht.rev_nshort != h.nshort))) ||
        h.kmer_q < 1 || h.kmer_q > MAX_Q || h.sa_sample < 1 || h.n + 1 >= (1ull << 32) ||
        h.n_occ_blocks != (h.n + 1) / OCC_ROWS + 1 ||
        h.n_super != (h.n_occ_blocks + SB_BLOCKS - 1) / SB_BLOCKS || h.n_mark_blocks != (h.n + 1) / MARK_ROWS + 1 ||
        h.table_len != (1ull << (2 * h.kmer_q)) + 1 || h.n_samples > h.n + 1 ||
        h.nshort != std::min<uint64_t>(h.kmer_q, h.n + 1)) {
        fclose(f);
        return MICA_EIO;
    }
    DeviceGuard g(device);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { fclose(f); set_last_cuda_error(e, "cudaSetDevice", __FILE__, __LINE__); return MICA_ECUDA; }
    mica_index *idx = new mica_index();
    idx->device = device;
    idx->params.kmer_q = h.kmer_q;
    idx->params.sa_sample = h.sa_sample;
    idx->n = h.n;
    idx->n_occ_blocks = h.n_occ_blocks;
    idx->n_super = h.n_super;
    idx->n_mark_blocks = h.n_mark_blocks;
    idx->n_samples = h.n_samples;
    idx->table_len = h.table_len;
    int rc = read_array(f, idx->occ, h.n_occ_blocks * 32);
    if (!rc) rc = read_array(f, idx->super, h.n_super * 16);
    if (!rc) rc = read_array(f, idx->marks, h.n_mark_blocks * 64);
    if (!rc) rc = read_array(f, idx->samples, h.n_samples * 4);
    if (!rc) rc = read_array(f, idx->table, h.table_len * 4);
    if (!rc && hr.has_rev) rc = read_array(f, idx->rocc, h.n_occ_blocks * 32);
    if (!rc && hr.has_rev) rc = read_array(f, idx->rsuper, h.n_super * 16);
    if (!rc && ht.has_rev_table) rc = read_array(f, idx->rtable, h.table_len * 4);
    fclose(f);
    idx->has_rev = hr.has_rev != 0;
    idx->params.lower_bounds = hr.has_rev;
    idx->params.full_sa = h.flags & 1u;
    if (!rc) {
        IndexView &v = idx->view;
        v.occ = (const uint4 *)idx->occ.p;
        v.super = (const uint4 *)idx->super.p;
        v.marks = (const uint4 *)idx->marks.p;
        v.samples = (const uint32_t *)idx->samples.p;
        v.table = (const uint32_t *)idx->table.p;
        v.n = h.n;
        v.rows = (uint32_t)(h.n + 1);
        v.dollar_row = (uint32_t)h.dollar_row;
        for (int c = 0; c < 5; c++) v.C[c] = (uint32_t)h.C[c];
        v.q = h.kmer_q;
        v.sa_sample = h.sa_sample;
        v.nshort = h.nshort;
        for (uint32_t t = 0; t < MAX_Q; t++) {
            v.short_pad[t] = h.short_pad[t];
            v.short_len[t] = h.short_len[t];
        }
        v.short_bloom = 0;
        for (uint32_t t = 0; t < v.nshort; t++) v.short_bloom |= 1ull << (v.short_pad[t] & 63);
        v.rev.occ = idx->has_rev ? (const uint4 *)idx->rocc.p : nullptr;
        v.rev.super = idx->has_rev ? (const uint4 *)idx->rsuper.p : nullptr;
        v.rev.dollar_row = hr.rev_dollar_row;
        for (int c = 0; c < 5; c++) v.rev.C[c] = (uint32_t)hr.rev_C[c];
        v.rev.table = ht.has_rev_table ? (const uint32_t *)idx->rtable.p : nullptr;
        v.rev.nshort = ht.rev_nshort;
        v.rev.short_bloom = 0;
        for (uint32_t t = 0; t < MAX_Q; t++) {
            v.rev.short_pad[t] = ht.rev_short_pad[t];
            v.rev.short_len[t] = ht.rev_short_len[t];
        }
        for (uint32_t t = 0; t < v.rev.nshort; t++) v.rev.short_bloom |= 1ull << (v.rev.short_pad[t] & 63);
        rc = upload_variants(idx);
        if (!rc && (h.flags & 1u)) rc = rebuild_full_sa(idx, 0);
        set_full_sa_view(idx);
        if (!rc) rc = build_long_tables(idx, nullptr, 0);
    }
    if (rc) { mica_index_free(idx); return rc; }
    *out = idx;
    return 0;
}

void mica_index_free(mica_index *idx)
{
    if (!idx) return;
    DeviceGuard g(idx->device);
    cudaSetDevice(idx->device);
    // batches still in flight on the pipeline slots finish before anything they read goes
    for (PipeSlot &ps : idx->pipe)
        if (ps.stream) cudaStreamSynchronize(ps.stream);
    dev_release(idx->occ);
    dev_release(idx->super);
    dev_release(idx->marks);
    dev_release(idx->samples);
    dev_release(idx->table);
    dev_release(idx->variants);
    dev_release(idx->rocc);
    dev_release(idx->rsuper);
    dev_release(idx->rtable);
    dev_release(idx->sa_full);
    dev_release(idx->isa);
    dev_release(idx->text);
    dev_release(idx->ltable);
    dev_release(idx->lrtable);
    free_workspace(idx->ws);
    for (PipeSlot &ps : idx->pipe) {
        free_workspace(ps.ws);
        if (ps.stream) cudaStreamDestroy(ps.stream);
    }
    delete idx;
}

int mica_index_get_info(const mica_index *idx, mica_index_info *info)
{
    if (!idx || !info) return MICA_EINVAL;
    info->n = idx->n;
    info->rows = idx->n + 1;
    info->kmer_q = idx->params.kmer_q;
    info->sa_sample = idx->params.sa_sample;
    info->dollar_row = idx->view.dollar_row;
    for (int c = 0; c < 5; c++) info->C[c] = idx->view.C[c];
    info->occ_bytes = idx->n_occ_blocks * 32 + idx->n_super * 16;
    info->mark_bytes = idx->n_mark_blocks * 64;
    info->sample_bytes = idx->n_samples * 4;
    info->table_bytes = idx->table_len * 4;
    info->device = idx->device;
    info->lower_bounds = idx->has_rev ? 1u : 0u;
    info->rev_occ_bytes = idx->has_rev ? idx->n_occ_blocks * 32 + idx->n_super * 16 : 0;
    info->rev_table_bytes = idx->view.rev.table ? idx->table_len * 4 : 0;
    info->full_sa = idx->has_full_sa ? 1u : 0u;
    info->full_sa_bytes = idx->has_full_sa ? full_sa_bytes(idx->n) : 0;
    info->long_q = idx->view.lfwd.table ? idx->view.lfwd.q : 0;
    info->long_table_bytes = idx->view.lfwd.table ? 2 * (((1ull << (2 * idx->view.lfwd.q)) + 1) * 4) : 0;
    return 0;
}

int mica_get_stats(const mica_index *idx, mica_stats *out)
{
    if (!idx || !out) return MICA_EINVAL;
    *out = idx->stats;
    return 0;
}

int mica_tuning_shapes(void) { return search_shape_count(); }

int mica_tuning_shape_info(int shape, int *stack_nodes, int *warps_per_cta, int *min_ctas_per_sm)
{
    return search_shape_info(shape, stack_nodes, warps_per_cta, min_ctas_per_sm);
}

int mica_set_tuning(mica_index *idx, const mica_tuning *t)
{
    if (!idx || !t) return MICA_EINVAL;
    if (t->shape < -1 || t->shape >= search_shape_count()) return MICA_EINVAL;
    if (t->plain_block && (t->plain_block < 32 || t->plain_block > 512 || t->plain_block % 32)) return MICA_EINVAL;
    for (uint32_t c = 0; c < LEN_CLASSES; c++)
        if (t->plain_block_len[c] &&
            (t->plain_block_len[c] < 32 || t->plain_block_len[c] > 512 || t->plain_block_len[c] % 32))
            return MICA_EINVAL;
    if (t->prefetch < -1 || t->prefetch > 1) return MICA_EINVAL;
    if (t->bidir_shape < -1 || t->bidir_shape >= bidir_shape_count()) return MICA_EINVAL;
    idx->tuning = *t;
    return 0;
}

int mica_get_tuning(const mica_index *idx, mica_tuning *t)
{
    if (!idx || !t) return MICA_EINVAL;
    *t = idx->tuning;
    return 0;
}

int mica_set_wait_limits(mica_index *idx, uint32_t idle_rounds, uint32_t ring_spins)
{
    if (!idx) return MICA_EINVAL;
    idx->idle_limit = idle_rounds;
    idx->spin_limit = ring_spins;
    return 0;
}

}  // extern "C"

namespace mica {
namespace {

__global__ void k_validate(ReadsView rd, uint64_t genome_len, unsigned int *bad)
{
    uint64_t total_words = rd.word_off[rd.n];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < rd.n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t m = rd.len[i];
        uint64_t off = rd.word_off[i];
        if (m == 0 || m > MICA_MAX_READ_LEN || m > genome_len || rd.k[i] > MICA_MAX_K ||
            off > total_words || total_words - off < (m + 15) / 16)
            atomicOr(bad, 1u);
    }
}

}  // namespace

int validate_device_batch(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
                          cudaStream_t s)
{
    if (rd.n == 0) return 0;
    if (int rc = dev_reserve(w.ctl, sizeof(SearchCtl) + 64)) return rc;
    unsigned int *bad = (unsigned int *)((char *)w.ctl.p + sizeof(SearchCtl));
    MICA_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, s));
    unsigned g = (unsigned)std::min<uint64_t>((rd.n + 255) / 256, 152 * 32);
    k_validate<<<g, 256, 0, s>>>(rd, idx->n, bad);
    st.launches = 1;
    unsigned int hb = 0;
    MICA_CUDA_TRY(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    return hb ? MICA_EINVAL : 0;
}

int validate_host_batch(const mica_index *idx, const uint64_t *off, const uint16_t *len, const uint8_t *k,
                        uint64_t n)
{
    const uint64_t total = off[n];
    auto bad_in = [&](uint64_t i0, uint64_t i1) {
        for (uint64_t i = i0; i < i1; i++) {
            uint32_t m = len[i];
            if (m == 0 || m > MICA_MAX_READ_LEN || m > idx->n || k[i] > MICA_MAX_K || off[i] > total ||
                total - off[i] < (m + 15) / 16)
                return true;
        }
        return false;
    };
    // a batch of a million reads: chunks on the host threads
    constexpr uint64_t CHUNK = 1u << 16;
    if (n <= 2 * CHUNK) return bad_in(0, n) ? MICA_EINVAL : 0;
    std::atomic<bool> bad{false};
    parallel_chunks((n + CHUNK - 1) / CHUNK, host_threads(), [&](uint64_t c) {
        if (!bad.load(std::memory_order_relaxed) && bad_in(c * CHUNK, std::min(n, (c + 1) * CHUNK)))
            bad.store(true, std::memory_order_relaxed);
    });
    return bad.load() ? MICA_EINVAL : 0;
}

// Defaults filled in and checked for a call with host buffers.
int host_params(const mica_align_params *params, mica_align_params &p)
{
    mica_align_params_default(&p);
    if (params) p = *params;
    if (p.kernel < MICA_KERNEL_PERSISTENT || p.kernel > MICA_KERNEL_BIDIRECTIONAL) return MICA_EINVAL;
    if (p.report > MICA_REPORT_BEST_STRATUM) return MICA_EINVAL;
    return 0;
}

// Copy a batch from host memory into w's staging buffers on stream s; the
// host threads check the batch while the copies run.  Nothing is launched
// before the check passes, and a rejected batch waits for its copies so that
// the caller may free the buffers on return.
int stage_host_batch(const mica_index *idx, Workspace &w, const uint32_t *packed_reads, const uint64_t *word_offsets,
                     const uint16_t *lengths, const uint8_t *k, uint64_t n_reads, cudaStream_t s, ReadsView &rd)
{
    const uint64_t nw = word_offsets[n_reads];
    int rc;
    if ((rc = dev_reserve(w.reads_words, std::max<uint64_t>(nw, 1) * 4)) ||
        (rc = dev_reserve(w.reads_off, (n_reads + 1) * 8)) ||
        (rc = dev_reserve(w.reads_len, std::max<uint64_t>(n_reads, 1) * 2)) ||
        (rc = dev_reserve(w.reads_k, std::max<uint64_t>(n_reads, 1))))
        return rc;
    if (nw) MICA_CUDA_TRY(cudaMemcpyAsync(w.reads_words.p, packed_reads, nw * 4, cudaMemcpyHostToDevice, s));
    MICA_CUDA_TRY(cudaMemcpyAsync(w.reads_off.p, word_offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, s));
    if (n_reads) {
        MICA_CUDA_TRY(cudaMemcpyAsync(w.reads_len.p, lengths, n_reads * 2, cudaMemcpyHostToDevice, s));
        MICA_CUDA_TRY(cudaMemcpyAsync(w.reads_k.p, k, n_reads, cudaMemcpyHostToDevice, s));
    }
    if ((rc = validate_host_batch(idx, word_offsets, lengths, k, n_reads))) {
        cudaStreamSynchronize(s);
        return rc;
    }
    rd = ReadsView{(const uint32_t *)w.reads_words.p, (const uint64_t *)w.reads_off.p,
                   (const uint16_t *)w.reads_len.p, (const uint8_t *)w.reads_k.p, n_reads};
    return 0;
}

// The result of the call just run on w (n reads, nh listed hits) copied into a
// new host result on stream s.
int copy_result(const Workspace &w, uint64_t n_reads, uint64_t nh, cudaStream_t s, mica_result **out)
{
    mica_result *r = result_new(n_reads, nh);
    if (!r) return MICA_ENOMEM;
    cudaError_t e = cudaSuccess;
    if (n_reads) e = cudaMemcpyAsync(r->total, w.total.p, n_reads * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->offsets, w.hit_off.p, (n_reads + 1) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nh) e = cudaMemcpyAsync(r->hits, w.hits.p, nh * sizeof(mica_hit), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "result copy", __FILE__, __LINE__);
        mica_result_free(r);
        return MICA_ECUDA;
    }
    *out = r;
    return 0;
}

}  // namespace mica

extern "C" {

int mica_align_device(mica_index *idx, const uint32_t *d_packed_reads, const uint64_t *d_word_offsets,
                      const uint16_t *d_lengths, const uint8_t *d_k, uint64_t n_reads,
                      const mica_align_params *params, mica_device_result *out)
{
    if (!idx || !out || (n_reads && (!d_packed_reads || !d_word_offsets || !d_lengths || !d_k)))
        return MICA_EINVAL;
    if (n_reads >= (1ull << 31)) return MICA_EINVAL;
    mica_align_params p;
    mica_align_params_default(&p);
    if (params) p = *params;
    if (p.kernel < MICA_KERNEL_PERSISTENT || p.kernel > MICA_KERNEL_BIDIRECTIONAL) return MICA_EINVAL;
    if (p.report > MICA_REPORT_BEST_STRATUM) return MICA_EINVAL;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    cudaStream_t s = (cudaStream_t)p.cuda_stream;
    ReadsView rd{d_packed_reads, d_word_offsets, d_lengths, d_k, n_reads};
    idx->stats.launches = 0;
    if (int rc = validate_device_batch(idx, idx->ws, idx->stats, rd, s)) return rc;
    uint64_t nh = 0;
    if (int rc = align_on_device(idx, idx->ws, idx->stats, rd, p, s, &nh)) return rc;
    out->n_reads = n_reads;
    out->n_hits = nh;
    out->total = (const uint64_t *)idx->ws.total.p;
    out->offsets = (const uint64_t *)idx->ws.hit_off.p;
    out->hits = (const mica_hit *)idx->ws.hits.p;
    return 0;
}

int mica_align_batch(mica_index *idx, const uint32_t *packed_reads, const uint64_t *word_offsets,
                     const uint16_t *lengths, const uint8_t *k, uint64_t n_reads,
                     const mica_align_params *params, mica_result **out)
{
    if (!idx || !out || !word_offsets || (n_reads && (!packed_reads || !lengths || !k))) return MICA_EINVAL;
    *out = nullptr;
    if (n_reads >= (1ull << 31)) return MICA_EINVAL;
    mica_align_params p;
    if (int rc = host_params(params, p)) return rc;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    cudaStream_t s = (cudaStream_t)p.cuda_stream;
    Workspace &w = idx->ws;
    ReadsView rd;
    int rc;
    if ((rc = stage_host_batch(idx, w, packed_reads, word_offsets, lengths, k, n_reads, s, rd))) return rc;
    idx->stats.launches = 0;
    uint64_t nh = 0;
    if ((rc = align_on_device(idx, idx->ws, idx->stats, rd, p, s, &nh))) {
        cudaStreamSynchronize(s);   // the caller's buffers are free to go on return
        return rc;
    }
    return copy_result(w, n_reads, nh, s, out);
}

// ---- pipelined host batches: two slots, each with its own stream and workspace ----

int mica_align_submit(mica_index *idx, const uint32_t *packed_reads, const uint64_t *word_offsets,
                      const uint16_t *lengths, const uint8_t *k, uint64_t n_reads,
                      const mica_align_params *params, uint64_t *ticket)
{
    if (!idx || !ticket || !word_offsets || (n_reads && (!packed_reads || !lengths || !k))) return MICA_EINVAL;
    *ticket = 0;
    if (n_reads >= (1ull << 31)) return MICA_EINVAL;
    mica_align_params p;
    if (int rc = host_params(params, p)) return rc;
    PipeSlot *slot = nullptr;
    for (PipeSlot &ps : idx->pipe)
        if (!ps.busy) { slot = &ps; break; }
    if (!slot) return MICA_EBUSY;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    if (!slot->stream) MICA_CUDA_TRY(cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking));
    Workspace &w = slot->ws;
    ReadsView rd;
    int rc;
    if ((rc = stage_host_batch(idx, w, packed_reads, word_offsets, lengths, k, n_reads, slot->stream, rd))) return rc;
    p = effective_params(idx, p);
    slot->st = mica_stats{};
    slot->launched = false;
    if (graph_eligible(w, p, rd)) {
        if (!(rc = create_events(w))) rc = align_graph_launch(idx, w, slot->st, rd, p, slot->stream, slot->launched);
        if (rc) {
            // no ticket, so the caller may free its buffers on return: let the copies finish first
            cudaStreamSynchronize(slot->stream);
            slot->launched = false;
            return rc;
        }
    }
    slot->busy = true;
    slot->p = p;
    slot->n_reads = n_reads;
    slot->ticket = *ticket = ++idx->next_ticket;
    return 0;
}

int mica_align_collect(mica_index *idx, uint64_t ticket, mica_result **out)
{
    if (!idx || !out) return MICA_EINVAL;
    *out = nullptr;
    PipeSlot *slot = nullptr;
    for (PipeSlot &ps : idx->pipe)
        if (ps.busy && ps.ticket == ticket) { slot = &ps; break; }
    if (!slot) return MICA_ENOTFOUND;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    Workspace &w = slot->ws;
    const uint64_t n = slot->n_reads;
    ReadsView rd{(const uint32_t *)w.reads_words.p, (const uint64_t *)w.reads_off.p,
                 (const uint16_t *)w.reads_len.p, (const uint8_t *)w.reads_k.p, n};
    uint64_t nh = 0;
    bool done = false;
    int rc = 0;
    if (slot->launched) rc = align_graph_finish(w, slot->st, rd, slot->p, &nh, done);
    if (!rc && !done) {
        // not captured, or the replay needs the regular path: run it now
        rc = align_on_device(idx, w, slot->st, rd, slot->p, slot->stream, &nh, false);
        if (slot->launched) slot->st.graph_fallbacks++;
    }
    if (!rc) rc = copy_result(w, n, nh, slot->stream, out);
    else cudaStreamSynchronize(slot->stream);
    idx->stats = slot->st;
    slot->busy = false;
    slot->launched = false;
    return rc;
}

void mica_result_free(mica_result *res)
{
    if (!res) return;
    ResultBlock *b = (ResultBlock *)res;
    if (b->magic != RESULT_MAGIC) return;   // not a result of this library (or freed twice)
    b->magic = 0;
    if (b->pinned) pin_put(b->mem, b->bytes);
    else free(b->mem);
    free(b);
}

int mica_debug_suffix_array(const uint8_t *genome_acgt, uint64_t len, int device, uint32_t *sa_out)
{
    if ((!genome_acgt && len) || !sa_out || len + 1 >= (1ull << 32)) return MICA_EINVAL;
    std::vector<uint8_t> codes;
    if (int rc = encode_genome(genome_acgt, len, codes)) return rc;
    DeviceGuard g(device);
    MICA_CUDA_TRY(cudaSetDevice(device));
    DevBuf dc, dsa;
    int rc = dev_reserve(dc, std::max<uint64_t>(len, 1));
    if (!rc) rc = dev_reserve(dsa, (len + 1) * 4);
    if (!rc && len && cudaMemcpy(dc.p, codes.data(), len, cudaMemcpyHostToDevice) != cudaSuccess) rc = MICA_ECUDA;
    if (!rc) rc = build_suffix_array((const uint8_t *)dc.p, len, (uint32_t *)dsa.p, 0);
    if (!rc && cudaMemcpy(sa_out, dsa.p, (len + 1) * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MICA_ECUDA;
    dev_release(dc);
    dev_release(dsa);
    return rc;
}

static int debug_rows_call(const mica_index *idx, const uint64_t *rows, uint64_t n, uint32_t *out, int per_row,
                           int which)
{
    if (!idx || (n && (!rows || !out))) return MICA_EINVAL;
    // Occ is defined for rows 0..N+1, SA for rows 0..N
    uint64_t limit = which == 0 ? idx->n + 1 : idx->n;
    for (uint64_t i = 0; i < n; i++)
        if (rows[i] > limit) return MICA_EINVAL;
    if (n == 0) return 0;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    DevBuf dr, dout;
    int rc = dev_reserve(dr, n * 8);
    if (!rc) rc = dev_reserve(dout, n * 4 * per_row);
    if (!rc && cudaMemcpy(dr.p, rows, n * 8, cudaMemcpyHostToDevice) != cudaSuccess) rc = MICA_ECUDA;
    if (!rc) rc = which == 0 ? debug_occ(idx, (const uint64_t *)dr.p, n, (uint32_t *)dout.p, 0)
                             : debug_locate(idx, (const uint64_t *)dr.p, n, (uint32_t *)dout.p, 0);
    if (!rc && cudaMemcpy(out, dout.p, n * 4 * per_row, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MICA_ECUDA;
    dev_release(dr);
    dev_release(dout);
    return rc;
}

int mica_debug_occ(const mica_index *idx, const uint64_t *rows, uint64_t n, uint32_t *occ_out)
{
    return debug_rows_call(idx, rows, n, occ_out, 4, 0);
}

int mica_debug_locate(const mica_index *idx, const uint64_t *rows, uint64_t n, uint32_t *pos_out)
{
    return debug_rows_call(idx, rows, n, pos_out, 1, 1);
}

int mica_debug_lower_bounds(mica_index *idx, const uint32_t *packed_reads, const uint64_t *word_offsets,
                            const uint16_t *lengths, const uint8_t *k, uint64_t n_reads, uint64_t *lb_out)
{
    if (!idx || !word_offsets || (n_reads && (!packed_reads || !lengths || !k || !lb_out))) return MICA_EINVAL;
    if (!idx->has_rev || n_reads >= (1ull << 31)) return MICA_EINVAL;
    if (int rc = validate_host_batch(idx, word_offsets, lengths, k, n_reads)) return rc;
    if (n_reads == 0) return 0;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    Workspace &w = idx->ws;
    uint64_t nw = word_offsets[n_reads];
    DevBuf dout;
    int rc;
    if ((rc = dev_reserve(w.reads_words, std::max<uint64_t>(nw, 1) * 4)) ||
        (rc = dev_reserve(w.reads_off, (n_reads + 1) * 8)) || (rc = dev_reserve(w.reads_len, n_reads * 2)) ||
        (rc = dev_reserve(w.reads_k, n_reads)) || (rc = dev_reserve(dout, 2 * n_reads * 8)))
        return rc;
    MICA_CUDA_TRY(cudaMemcpy(w.reads_words.p, packed_reads, std::max<uint64_t>(nw, 1) * 4, cudaMemcpyHostToDevice));
    MICA_CUDA_TRY(cudaMemcpy(w.reads_off.p, word_offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice));
    MICA_CUDA_TRY(cudaMemcpy(w.reads_len.p, lengths, n_reads * 2, cudaMemcpyHostToDevice));
    MICA_CUDA_TRY(cudaMemcpy(w.reads_k.p, k, n_reads, cudaMemcpyHostToDevice));
    ReadsView rd{(const uint32_t *)w.reads_words.p, (const uint64_t *)w.reads_off.p,
                 (const uint16_t *)w.reads_len.p, (const uint8_t *)w.reads_k.p, n_reads};
    rc = debug_lower_bounds(idx, w, rd, (unsigned long long *)dout.p, 0);
    if (!rc && cudaMemcpy(lb_out, dout.p, 2 * n_reads * 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MICA_ECUDA;
    dev_release(dout);
    return rc;
}

int mica_debug_seed_interval(const mica_index *idx, const uint32_t *codes, uint32_t len, uint64_t n,
                             uint32_t *lr_out)
{
    if (!idx || (n && (!codes || !lr_out)) || len < 1 || len > idx->params.kmer_q) return MICA_EINVAL;
    for (uint64_t i = 0; i < n; i++)
        if ((uint64_t)codes[i] >= (1ull << (2 * len))) return MICA_EINVAL;
    if (n == 0) return 0;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    DevBuf dc, dout;
    int rc = dev_reserve(dc, n * 4);
    if (!rc) rc = dev_reserve(dout, n * 8);
    if (!rc && cudaMemcpy(dc.p, codes, n * 4, cudaMemcpyHostToDevice) != cudaSuccess) rc = MICA_ECUDA;
    if (!rc) rc = debug_seed(idx, (const uint32_t *)dc.p, len, n, (uint32_t *)dout.p, 0);
    if (!rc && cudaMemcpy(lr_out, dout.p, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MICA_ECUDA;
    dev_release(dc);
    dev_release(dout);
    return rc;
}

}  // extern "C"
