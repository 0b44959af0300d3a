// Internal definitions shared by the CUDA translation units of libmica_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "mica.h"

namespace mica {

// ---------------------------------------------------------------------------
// Index layout constants
// ---------------------------------------------------------------------------
// Occurrence block: 32 bytes (one sector) for 96 BWT rows =
//   u32 [A | C << 16], u32 [G | T << 16]: Occ(c, block start) minus the
//        counts at the start of the block's superblock (16 bits each);
//   then for rows 0-31, 32-63, 64-95 in turn a low-bit word and a high-bit
//   word (row t at bit t % 32; symbol code = low | high << 1; $ is stored as
//   A and corrected with dollar_row).
// Superblock: SB_BLOCKS consecutive blocks (65,472 rows, so the 16-bit
// relative counts cannot overflow); its 16-byte entry holds Occ(A..T, start).
constexpr uint32_t OCC_ROWS = 96;
constexpr uint32_t OCC_WORDS = 8;         // uint32 per block
constexpr uint32_t SB_BLOCKS = 682;
// Mark block: 64 bytes = uint32 rank of marked rows before the block + 15
// words of mark bits (480 rows).
constexpr uint32_t MARK_ROWS = 480;
constexpr uint32_t MAX_Q = 12;
constexpr uint32_t MAX_LQ = 15;   // longest q-mer of the bidirectional seed tables

// A q-mer table of bounds (4^q + 1 uint32: entry x = suffixes smaller than
// the q-mer x) with the short-suffix corrections that make its bounds exact.
struct QmerView {
    const uint32_t *table;
    uint32_t q, nshort;
    uint32_t short_pad[MAX_LQ];
    uint32_t short_len[MAX_LQ];
    unsigned long long short_bloom;
};
constexpr uint32_t MAX_WORDS = MICA_MAX_READ_LEN / 16;   // packed words per read

// Seed variants: for budget k, every way to substitute <= k of the last q
// bases; ordered so the first V(q', k) entries touch only the last q' bases.
constexpr uint32_t VAR_OFF[5] = {0, 1, 38, 669, 7240};
constexpr uint32_t N_VARIANTS = 7240;
__host__ __device__ __forceinline__ uint32_t var_off(uint32_t k)
{
    return k == 0 ? 0u : k == 1 ? 1u : k == 2 ? 38u : 669u;
}

// Device view of a resident index, passed to kernels by value.
struct IndexView {
    const uint4 *occ;          // blocks * 2 uint4
    const uint4 *super;        // superblocks: Occ(A..T, superblock start)
    const uint4 *marks;        // mark blocks * 4 uint4
    const uint32_t *samples;   // SA values of marked rows, in row order
    const uint32_t *table;     // 4^q + 1 bounds
    const uint32_t *variants;  // N_VARIANTS seed variants: bits 0..23 xor mask, 24..25 d
    uint64_t n;                // genome length
    uint32_t rows;             // n + 1
    uint32_t dollar_row;
    uint32_t C[5];
    uint32_t q;
    uint32_t sa_sample;
    // Suffixes of T shorter than q + 1 symbols (u$ with |u| < q, at most q of
    // them) sort below u padded with A to a q-mer, so the table bound at that
    // padded code counts them.  An interval ending at that code must drop
    // them (they sort after it); an interval of a j-mer starting there must
    // drop those with |u| >= j (they start with the j-mer).
    uint32_t nshort;
    uint32_t short_pad[MAX_Q];
    uint32_t short_len[MAX_Q];
    unsigned long long short_bloom;   // bit (pad & 63) of every short pad: a cheap pre-check
    // Occurrence blocks of the reversed genome G~$ (same block layout; occ is
    // null when the index was built without them).  Backward search of a
    // pattern read left to right on G~ finds whether a substring of G occurs.
    struct {
        const uint4 *occ;
        const uint4 *super;
        uint32_t dollar_row;
        uint32_t C[5];
        // q-mer table of G~$ and its short-suffix corrections (as above);
        // table is null when the index has none (index files before version 4)
        const uint32_t *table;
        uint32_t nshort;
        uint32_t short_pad[MAX_Q];
        uint32_t short_len[MAX_Q];
        unsigned long long short_bloom;
    } rev;
    // The whole suffix array SA[0, n], its inverse ISA[0, n] and the text G at
    // 2 bits per base (16 per word, least-significant first, zero words past
    // the end); all null when the index was built without them.
    const uint32_t *sa_full;
    const uint32_t *isa;
    const uint32_t *text;
    // Seed tables of a longer q (built from the text with full_sa, for the
    // bidirectional kernel's seeds) of G$ and of G~$; table null when absent.
    QmerView lfwd, lrev;
};

// Read batch in device memory.
struct ReadsView {
    const uint32_t *words;
    const uint64_t *word_off;
    const uint16_t *len;
    const uint8_t *k;
    uint64_t n;
};

// Leaf interval found by the search.
struct Interval {
    uint32_t read;
    uint32_t meta;   // bit 0..1 d, bit 2 strand
    uint32_t l, r;
};

// Work item in the device queues: a seed range of a (read, strand) task or a
// continuation node.  meta: bit 30 kind (1 = node), bit 29 strand, bits 0..1
// d, bits 8..16 i (node).  The persistent kernel's spill ring publishes items
// through a separate sequence word per slot.
struct WorkItem {
    uint32_t read;
    uint32_t meta;
    uint32_t a, b;   // node: l, r; seeds: first, end variant
};
constexpr uint32_t WI_NODE = 1u << 30;
constexpr uint32_t WI_MINUS = 1u << 29;

// Hit as written to the output (matches mica_hit).
struct Hit {
    uint32_t pos;
    uint8_t strand, mm;
    uint16_t pad;
};

// Device-global control block of one search launch.
struct SearchCtl {
    unsigned long long task_head;     // next fresh task
    unsigned long long ntasks;
    unsigned int spill_reserve;       // spill ring: positions reserved by producers (plain kernel:
                                      //   items in its re-queue array)
    unsigned int spill_head;          // spill ring: positions claimed by consumers
    unsigned int spill_cap;
    int busy;                         // warps holding work
    unsigned int iv_count;            // intervals written
    unsigned int iv_cap;
    unsigned int error;               // bit 0 interval overflow, bit 1 spill overflow, bit 2 timeout
    unsigned int pad_;
    unsigned long long seeds, nodes, rank_blocks, spills;
    unsigned long long rounds, lane_ops;
    unsigned long long rounds_kind[3];   // multi-row, single-row, seed rounds
    unsigned long long lb_steps, lb_dead; // lower-bound pass: extensions, tasks with no budget left
    unsigned long long wait_queue_ns, wait_idle_ns;   // sleeps in queue waits / by idle warps (summed)
    unsigned long long deep_moves;                    // nodes moved to per-warp overflow stacks
    unsigned int redo_reads;                          // bidirectional search: reads given up, to be re-searched
    unsigned int fr_count;                            // bidirectional search: nodes exported this round
    unsigned long long verified, verify_bytes;        // bidirectional search: one-row intervals checked
                                                      //   against the text, and the bytes that read
    unsigned long long verify_sectors;                // ... and the 32-byte sectors those reads touch
};

constexpr unsigned ERR_IV_OVERFLOW = 1u;
constexpr unsigned ERR_SPILL_OVERFLOW = 2u;
constexpr unsigned ERR_TIMEOUT = 4u;
constexpr unsigned ERR_HIT_OVERFLOW = 8u;
constexpr uint32_t IV_PURGED = 0xffffffffu;   // Interval::read of a leaf dropped after the search

// ---------------------------------------------------------------------------
// Host-side helpers
// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

int dev_reserve(DevBuf &b, size_t bytes);   // grow-only device buffer
void dev_release(DevBuf &b);
// A host result for n_reads reads and n_hits listed hits (arrays in one
// page-locked block from the library's pool); free with mica_result_free.
mica_result *result_new(uint64_t n_reads, uint64_t n_hits);

// Makes `dev` current for a scope and restores the caller's device after.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) { if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev); else prev = -1; }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

constexpr int GRAPH_KEY = 31;   // words identifying a captured batch shape

// Per-index workspace reused across align calls.
struct Workspace {
    DevBuf ctl, iv, iv_sorted, iv_cnt, iv_off, total, keep, hit_off, hits, spill, big, scan_tmp;
    DevBuf lb;   // per (read, strand) task: mismatch lower-bound breakpoints (uint64)
    DevBuf spill_seq;   // spill ring: one sequence word per slot
    DevBuf deep;        // per-warp overflow stacks of the persistent kernel
    DevBuf reads_words, reads_off, reads_len, reads_k;   // staging for host batches
    DevBuf spill2;                                        // plain kernel re-queue ping-pong
    DevBuf lenlist;                                       // plain kernel: reads by length class
    DevBuf redo;                                          // bidirectional search: given-up reads (bits, list)
    DevBuf frontier;                                      // bidirectional search: exported nodes, two rounds
    uint32_t iv_cap = 0, spill_cap = 0;
    uint32_t bd_deep_cap = 0;   // bidirectional search: entries of each warp's overflow stacks
    bool bd_redo_seen = false;  // bidirectional search: the last call gave reads up (no graph replay then)
    uint64_t hit_cap_total = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // call timing
    cudaEvent_t kev[2] = {nullptr, nullptr};                      // search kernel timing
    // captured pipeline for a repeated batch shape (persistent kernel)
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    void *pin_tmpl = nullptr, *pin_status = nullptr;              // pinned host blocks
    uint64_t gkey[GRAPH_KEY] = {};
    uint64_t hit_capacity = 0;
    uint64_t glaunches = 0;   // kernels in the captured graph
    int g_grid = 0;           // grid of the launched replay's search kernel
};

// One of an index's two slots for pipelined host batches
// (mica_align_submit / mica_align_collect).
struct PipeSlot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    bool busy = false;       // submitted and not yet collected
    bool launched = false;   // its captured replay is queued (else collect runs the search)
    uint64_t ticket = 0, n_reads = 0;
    mica_align_params p{};
    mica_stats st{};
};

}  // namespace mica

struct mica_index {
    int device = 0;
    mica_index_params params{};
    mica::IndexView view{};
    uint64_t n = 0;
    uint64_t n_occ_blocks = 0, n_super = 0, n_mark_blocks = 0, n_samples = 0, table_len = 0;
    mica::DevBuf occ, super, marks, samples, table, variants;
    mica::DevBuf rocc, rsuper;   // reversed genome's occurrence blocks (lower bounds, bidirectional search)
    mica::DevBuf rtable;         // reversed genome's q-mer table (bidirectional search)
    mica::DevBuf sa_full, isa, text;   // whole suffix array, its inverse, 2-bit text (full_sa)
    mica::DevBuf ltable, lrtable;      // longer seed tables of G$ and G~$ (with full_sa)
    bool has_rev = false;
    bool has_full_sa = false;
    mica::Workspace ws;
    mica_stats stats{};
    mica_tuning tuning{-1, 0, 0, {0, 0, 0, 0}, -1, 0, 0, -1};
    uint32_t idle_limit = 0, spin_limit = 0;   // persistent kernel wait bounds; 0 = built-in defaults
    mica::PipeSlot pipe[2];                    // pipelined host batches
    uint64_t next_ticket = 0;
};

namespace mica {

#define MICA_CUDA_TRY(call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            mica::set_last_cuda_error(e_, #call, __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? MICA_ENOMEM : MICA_ECUDA; \
        }                                                     \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);
void set_last_internal(const char *msg);   // detail returned by mica_strerror(MICA_EINTERNAL)

// Records a timing event on s.  While s is being captured into a graph a
// plain record is only a dependency marker, so the event becomes an external
// event-record node, recorded on every replay.
inline cudaError_t record_event(cudaEvent_t e, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(s, &cs);
    if (r != cudaSuccess) return r;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                               : cudaEventRecord(e, s);
}

// Milliseconds between two recorded events; 0 (and the error cleared) when
// the pair cannot be timed.
inline float elapsed_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        (void)cudaGetLastError();
        ms = 0.f;
    }
    return ms;
}

// index_build.cu
int build_suffix_array(const uint8_t *d_codes, uint64_t n, uint32_t *d_sa, cudaStream_t s);
// full_sa.cu: the whole suffix array, its inverse and the 2-bit text
uint64_t full_sa_text_words(uint64_t n);   // text words incl. zero padding (a multiple of 4)
uint64_t full_sa_bytes(uint64_t n);
void set_full_sa_view(mica_index *idx);
int build_full_sa(mica_index *idx, DevBuf &sa, const uint8_t *d_codes, uint64_t n, cudaStream_t s);
int rebuild_full_sa(mica_index *idx, cudaStream_t s);
uint32_t long_seed_q(uint64_t n, uint32_t q);   // q of the longer seed tables (== q: none)
// the longer seed tables from the genome's codes (or, when d_codes is null,
// from the resident text)
int build_long_tables(mica_index *idx, const uint8_t *d_codes, cudaStream_t s);

int build_index_from_codes(const uint8_t *d_codes, uint64_t n, const mica_index_params &p,
                           mica_index *idx, cudaStream_t s);
int upload_variants(mica_index *idx);
struct QmerShort {
    uint32_t nshort = 0, pad[MAX_LQ] = {}, len[MAX_LQ] = {};
    unsigned long long bloom = 0;
};
int build_qmer_table(const uint8_t *d_codes, uint64_t n, uint32_t q, DevBuf &table, QmerShort &sh, DevBuf &tmp,
                     cudaStream_t s);
void set_rev_short(IndexView &v, const QmerShort &sh);
void host_variant_table(uint32_t *out);   // N_VARIANTS entries
uint32_t variant_count(uint32_t q, uint32_t k);

// search.cu
struct SearchConfig {
    int kernel;                 // MICA_KERNEL_*
    int shape = -1;             // persistent kernel shape (index into the compiled shapes), -1 = default
    int block_threads;          // persistent: threads per block
    int blocks_per_sm;
    int plain_block;
    uint32_t plain_budget;      // plain: node expansions per task before re-queueing
    int plain_block_len[4] = {0, 0, 0, 0};   // plain by length: block size per class
    bool prune = false;         // compute and use mismatch lower bounds (index has them)
    bool prefetch = false;      // persistent: prefetch the next round's occurrence blocks into L2
};
constexpr uint32_t LEN_CLASSES = 4;   // 1-64, 65-128, 129-192, 193-256 bases
int run_search(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
               const SearchConfig &cfg, cudaStream_t s);
int search_shape_count();
int prepare_persistent(const mica_index *idx, Workspace &w, uint64_t n, int shape_in, SearchCtl &tmpl,
                       int &grid, int &shape);
int debug_lower_bounds(const mica_index *idx, Workspace &w, const ReadsView &rd, unsigned long long *d_out,
                       cudaStream_t s);
int run_search_list(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd, const uint32_t *d_list,
                    uint32_t n_list, uint32_t iv_base, bool prune, cudaStream_t s);
constexpr int STRATUM_FALLBACK = 1;   // run_search_stratum: rerun as an exhaustive search
int run_search_stratum(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
                       const SearchConfig &cfg, cudaStream_t s);
int enqueue_persistent(const mica_index *idx, Workspace &w, const ReadsView &rd, int shape, int grid,
                       const SearchCtl *pinned_tmpl, bool prune, bool prefetch, cudaStream_t s,
                       uint64_t &launches);
int search_shape_info(int shape, int *scap, int *warps, int *minb);
int search_workspace_bytes(const mica_index *idx, uint64_t n, uint64_t *bytes);

// bidir.cu
constexpr int BIDIR_FALLBACK = 2;   // run_search_bidir: an overflow stack filled; run the one-directional search
bool bidir_available(const mica_index *idx);
int bidir_shape_index(const mica_index *idx);   // compiled bidirectional shape a call uses
int bidir_shape_count();
int prepare_bidir(const mica_index *idx, Workspace &w, uint64_t n, SearchCtl &tmpl, int &grid);
int enqueue_bidir_graph(const mica_index *idx, Workspace &w, const ReadsView &rd, int grid, const SearchCtl *tmpl_src,
                        cudaStream_t s, uint64_t &launches);
int run_search_bidir(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd, cudaStream_t s);

// post.cu
int run_post(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd, uint32_t hit_cap,
             uint32_t report, cudaStream_t s, uint64_t *n_hits_out);
// capi.cu: the whole path on one workspace (validation of device batches included)
int align_on_device(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
                    const mica_align_params &p, cudaStream_t s, uint64_t *nh, bool allow_graph = true);
int validate_device_batch(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
                          cudaStream_t s);
int validate_host_batch(const mica_index *idx, const uint64_t *off, const uint16_t *len, const uint8_t *k,
                        uint64_t n);
void free_workspace(Workspace &w);
int enqueue_post_device(const mica_index *idx, Workspace &w, const ReadsView &rd, uint32_t hit_cap,
                        uint32_t report, uint64_t hit_capacity, cudaStream_t s, void *status,
                        uint64_t &launches);
int reserve_post(Workspace &w, uint64_t n, uint32_t iv_cap, uint64_t hit_capacity);
uint64_t post_workspace_bytes(uint64_t n, uint64_t iv_cap, uint64_t hit_capacity);
int exclusive_scan_u64_scratch(const uint64_t *in, uint64_t n, uint64_t *out, unsigned long long *scratch,
                               cudaStream_t s);
int debug_occ(const mica_index *idx, const uint64_t *d_rows, uint64_t n, uint32_t *d_out, cudaStream_t s);
int debug_locate(const mica_index *idx, const uint64_t *d_rows, uint64_t n, uint32_t *d_out, cudaStream_t s);
int debug_seed(const mica_index *idx, const uint32_t *d_codes, uint32_t len, uint64_t n, uint32_t *d_out,
               cudaStream_t s);

}  // namespace mica
