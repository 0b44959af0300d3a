/*
 * mica.h -- C ABI of the GB300 k-mismatch FM-index read search.
 *
 * The operation (MICA, Section 2): every read is first placed on the reference
 * genome by searching a BWT (FM) index with few mismatches; reads that fail
 * go on to a dynamic-programming phase for indels, which this library does not
 * implement.  Here "few mismatches" is a per-read budget k in 0..3 of base
 * substitutions, and the search is exhaustive on both strands:
 *
 *   H(R) = {(p,+,d): d = Ham(R,     G[p,p+m)) <= k}
 *        u {(p,-,d): d = Ham(rc(R), G[p,p+m)) <= k},     0 <= p <= N-m
 *
 * A hit on the - strand reports the leftmost forward-strand coordinate p of
 * the matched window.  A read equal to its own reverse complement reports both
 * (p,+,d) and (p,-,d).  Per read, `total` is the exact size of H(R); at most
 * `hit_cap` hits are listed: when total > hit_cap the listed ones are the first
 * hit_cap in the order (d ascending, + before -, suffix-array row ascending).
 * Listed hits are sorted by (position, strand, d).
 *
 * The index (Section 2: a BWT index of the genome resident in the
 * accelerator's global memory, laid out to cut memory transactions) is built
 * and kept in GPU memory: the BWT as two bit planes interleaved with
 * occurrence counts in 32-byte blocks of 96 rows, a q-mer table of
 * suffix-array interval bounds, a text-sampled suffix array with a
 * row-marking bit vector and, optionally, the occurrence blocks of the
 * reversed genome, from which the search takes a lower bound on the
 * mismatches each pattern prefix needs (Li and Durbin's D array) to prune
 * branches that cannot reach a hit; pruning never changes the result.
 *
 * Conventions.  Every function returning int returns MICA_OK (0) or a negative
 * MICA_E* code; mica_strerror names it.  Input buffers are owned by the caller
 * and only read during the call.  Objects returned through `out` pointers are
 * owned by the library until the matching *_free call.  A mica_index is used
 * by one host thread at a time.  Device pointers are CUDA device addresses on
 * the index's device.  Base codes: A=0, C=1, G=2, T=3.
 *
 * Around the search, host-side layers read references (FASTA, several
 * contigs, ambiguous bases) and reads (FASTQ), and write SAM; they make no
 * CUDA call and work on machines without a GPU.
 */
#ifndef MICA_H
#define MICA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MICA_OK = 0,
    MICA_EINVAL = -1,     /* bad argument: k > 3, read length 0 or > N or > MICA_MAX_READ_LEN,
                             non-ACGT genome byte, bad parameter */
    MICA_ENOMEM = -2,     /* host or device allocation failed */
    MICA_EIO = -3,        /* index file cannot be read or written, or is malformed */
    MICA_ECUDA = -4,      /* a CUDA runtime call failed */
    MICA_ETIMEOUT = -5,   /* a bounded device or host wait expired */
    MICA_EINTERNAL = -6,  /* an internal capacity retry did not converge (should not happen) */
    MICA_EBUSY = -7,      /* serving: the request is not finished yet; pipelined batches: both slots
                             are in flight */
    MICA_ENOTFOUND = -8   /* serving: unknown request id; pipelined batches: unknown ticket */
};

#define MICA_MAX_READ_LEN 256   /* bases per read */
#define MICA_MAX_K 3            /* substitutions per read */

typedef struct mica_index mica_index;

/* Index layout parameters (defaults: 12, 16, 1, 1). */
typedef struct {
    uint32_t kmer_q;     /* q-mer seed table length, 1..12: table of 4^q + 1 uint32 bounds */
    uint32_t sa_sample;  /* text sampling rate s, 1..256: SA[j] kept when SA[j] % s == 0 */
    uint32_t lower_bounds; /* 1: also build the reversed genome's occurrence blocks and q-mer
                              table (one more suffix array at build time, about +1/3 device
                              memory) so searches can prune by mismatch lower bounds and extend
                              patterns in both directions; 0: not */
    uint32_t full_sa;    /* 1: also keep the whole suffix array, its inverse and the genome at
                            2 bits per base on the device (4 (N + 1) + 4 (N + 1) + N / 4 bytes):
                            the bidirectional search then checks an interval of one row
                            against the genome's text instead of extending it base by base, and
                            locating a row is one read; 0: not.  Same results either way */
} mica_index_params;

enum {
    MICA_KERNEL_PERSISTENT = 0,      /* one launch of the warp-cooperative work-pool kernel */
    MICA_KERNEL_PLAIN = 1,           /* one launch of the one-task-per-thread kernel over the batch */
    MICA_KERNEL_PLAIN_BY_LENGTH = 2, /* one plain launch per read-length class (1-64, 65-128,
                                        129-192, 193-256 bases), each with its own block size */
    MICA_KERNEL_BIDIRECTIONAL = 3    /* the default: the warp-pool kernel searching both directions (the
                                        read in k + 1 pieces, one search per leftmost exact piece, over the
                                        genome's and the reversed genome's index), plus further launch
                                        rounds for the nodes of heavy trees.  Same result.  An index built
                                        without lower_bounds (or loaded from a file before format 4) runs
                                        the persistent kernel instead */
};

typedef struct {
    uint32_t hit_cap;    /* listed hits per read; 0 = no cap (every hit listed) */
    int32_t kernel;      /* MICA_KERNEL_* */
    void *cuda_stream;   /* cudaStream_t to run on; NULL = the legacy default stream */
    uint32_t prune;      /* 1 (default): prune by mismatch lower bounds when the index has
                            them; 0: plain exhaustive backtracking.  Same result either way. */
    uint32_t report;     /* MICA_REPORT_*: which placements a read's total and list cover */
} mica_align_params;

enum {
    MICA_REPORT_ALL = 0,          /* H(R): every placement with d <= k (default) */
    MICA_REPORT_BEST_STRATUM = 1  /* the placements of H(R) with the read's smallest d; total = their
                                     number (1 = a unique best placement), cap and order as above */
};

typedef struct {
    uint32_t pos;        /* leftmost forward coordinate of the matched window */
    uint8_t strand;      /* 0 = +, 1 = - */
    uint8_t mm;          /* substitutions d */
    uint16_t pad;
} mica_hit;

/* Host-side result, owned by the library until mica_result_free. */
typedef struct {
    uint64_t n_reads;
    uint64_t *total;     /* n_reads: exact |H(R)| */
    uint64_t *offsets;   /* n_reads + 1: read i's hits are hits[offsets[i], offsets[i+1]) */
    mica_hit *hits;
} mica_result;

/* Device-side result: pointers into the index's workspace on its device,
   valid until the next align call on the same index. */
typedef struct {
    uint64_t n_reads;
    uint64_t n_hits;
    const uint64_t *total;
    const uint64_t *offsets;
    const mica_hit *hits;
} mica_device_result;

/* Work counters of the last align call on an index. */
typedef struct {
    uint64_t tasks;          /* (read, strand) search tasks = 2 * n_reads */
    uint64_t seeds;          /* q-mer table lookups */
    uint64_t nodes;          /* backtracking nodes expanded (one interval extension each) */
    uint64_t rank_blocks;    /* 32-byte occurrence blocks read by the search (incl. lower bounds) */
    uint64_t intervals;      /* leaf SA intervals found */
    uint64_t located;        /* SA rows resolved to positions */
    uint64_t lf_steps;       /* LF-mapping steps taken by the resolution */
    uint64_t spills;         /* work items moved to the device queue (persistent kernel)
                                or re-queued after the per-thread budget (plain kernel) */
    uint64_t retries;        /* internal buffer-growth retries */
    uint64_t launches;       /* CUDA kernels this library launched for the call */
    uint64_t warp_rounds;    /* persistent kernel: work-pool rounds over all warps */
    uint64_t lane_ops;       /* persistent kernel: node extensions + seed lookups done by lanes */
    uint64_t rounds_multi, rounds_single, rounds_seed;   /* persistent kernel rounds by kind of work */
    uint64_t graph_captures;  /* the call captured its pipeline as a CUDA graph (new batch shape) */
    uint64_t graph_replays;   /* the call ran as one replay of a captured graph */
    uint64_t graph_fallbacks; /* a replay overflowed a buffer; the regular path recomputed the call */
    uint64_t lb_steps;       /* lower-bound pass: interval extensions on the reversed genome */
    uint64_t lb_dead_tasks;  /* tasks whose lower bound already exceeds k before any seed */
    uint64_t queue_wait_ns;  /* persistent kernel: nanoseconds slept by warps waiting on the spill ring
                                (summed over warps; compare with kernel_ms x warps) */
    uint64_t idle_wait_ns;   /* persistent kernel: nanoseconds slept by warps with no work */
    uint64_t overflow_moves; /* persistent kernel: nodes moved to a warp's private overflow stack */
    uint64_t grid_ctas;      /* persistent kernel: CTAs of the launch (SMs x resident CTAs per SM) */
    uint64_t fallback_reads; /* bidirectional kernel: reads it gave up on (over the node budget, or on a
                                warp whose overflow stack filled), searched again by the persistent kernel */
    uint64_t verified;       /* bidirectional kernel: one-row intervals checked against the genome's text */
    uint64_t verify_bytes;   /* bytes those checks read: suffix array and inverse entries, text words */
    uint64_t verify_sectors; /* 32-byte sectors those reads touch (one per SA or ISA entry, the text
                                window's span) */
    float search_ms;         /* device time of the search phase (kernel + its control copies) */
    float kernel_ms;         /* device time of the search kernel launch(es) alone, with the
                                lower-bound pass when pruning */
    float total_ms;          /* device time of the whole call */
} mica_stats;

typedef struct {
    uint64_t n;              /* genome length N */
    uint64_t rows;           /* N + 1 */
    uint32_t kmer_q, sa_sample;
    uint64_t dollar_row;     /* BWT row holding $ */
    uint64_t C[5];           /* C[c] = symbols of G$ smaller than c; C[4] = N + 1 */
    uint64_t occ_bytes, mark_bytes, sample_bytes, table_bytes;
    int32_t device;
    uint32_t lower_bounds;   /* 1 if the reversed genome's occurrence blocks are resident */
    uint64_t rev_occ_bytes;  /* their size (0 without them) */
    uint64_t rev_table_bytes; /* the reversed genome's q-mer table (bidirectional search; 0 without it) */
    uint32_t full_sa;        /* 1 if the whole suffix array, its inverse and the 2-bit text are resident */
    uint64_t full_sa_bytes;  /* their size (0 without them) */
    uint32_t long_q;         /* q of the longer seed tables of G$ and G~$ the bidirectional search
                                seeds from (built from the text with full_sa when log4 N + 1 exceeds
                                kmer_q; at most 15); 0 without them */
    uint64_t long_table_bytes; /* their size, both directions (0 without them) */
} mica_index_info;

const char *mica_strerror(int code);

/* Fill *p with the defaults (kmer_q 12, sa_sample 16, lower_bounds 1, full_sa 1). */
void mica_index_params_default(mica_index_params *p);
/* Fill *p with the defaults (hit_cap 1000, bidirectional kernel, default stream, prune 1,
   report MICA_REPORT_ALL). */
void mica_align_params_default(mica_align_params *p);

/*
 * Build the index of genome_acgt[0, len) (ASCII A/C/G/T, either case; anything
 * else is MICA_EINVAL) on the current CUDA device and keep it there.  The
 * suffix array of G$ is built on the GPU by prefix doubling.  params may be
 * NULL (defaults).  *out owns device memory until mica_index_free.
 */
int mica_index_build_resident(const uint8_t *genome_acgt, uint64_t len,
                              const mica_index_params *params, int device, mica_index **out);

/* Build as above on the current device, write it to out_path, free it. */
int mica_index_build(const uint8_t *genome_acgt, uint64_t len,
                     const mica_index_params *params, const char *out_path);

/* Index files (format version 5) hold the reversed genome's blocks and q-mer
   table when the index has them.  The whole suffix array, its inverse and the
   text are not stored: a file records whether the index kept them, and
   loading rebuilds them on the device from the sampled suffix array by LF
   steps (N steps in all, s - 1 at most from each sample).  Version 4 files
   (no such record), version 3 files (blocks, no table) and version 2 files
   (neither) still load. */
int mica_index_save(const mica_index *idx, const char *path);
/* Read an index file and upload it to `device`, where it stays until freed. */
int mica_index_load(const char *path, int device, mica_index **out);
/* Release the index and its device memory; batches submitted and not yet
   collected finish first (their results are dropped).  NULL is a no-op. */
void mica_index_free(mica_index *idx);
int mica_index_get_info(const mica_index *idx, mica_index_info *info);

/*
 * Align a batch given in HOST memory: packed_reads holds 2-bit bases, 16 per
 * uint32 word, least-significant bits first; read i (length lengths[i], budget
 * k[i]) starts at word word_offsets[i] (n_reads + 1 offsets, non-decreasing).
 * Copies the batch to the device, runs the search, copies the result back.
 * The host checks the batch (lengths 1..MICA_MAX_READ_LEN and at most the
 * genome's length, k <= MICA_MAX_K, every read inside packed_reads) while the
 * copies run; a batch that fails returns MICA_EINVAL with no search launched,
 * after its copies have finished.  The input buffers are the caller's and are
 * not used after the call returns.  params may be NULL (defaults).  On
 * success *out is a new mica_result (pinned host memory from a pool).
 */
int mica_align_batch(mica_index *idx, const uint32_t *packed_reads, const uint64_t *word_offsets,
                     const uint16_t *lengths, const uint8_t *k, uint64_t n_reads,
                     const mica_align_params *params, mica_result **out);
void mica_result_free(mica_result *res);

/*
 * Pipelined host batches (Section 2: the host feeds the card the next batch
 * of reads while it works on the current one).  mica_align_submit stages a
 * batch given in host memory (same layout and checks as mica_align_batch) on
 * one of the index's two pipeline slots, each with its own stream and
 * workspace, queues its search and returns without waiting for the device;
 * *ticket names the batch.  mica_align_collect waits for that batch, copies
 * its result back and returns it as a new mica_result (free it with
 * mica_result_free).  While one batch searches, the next one's copies and
 * host checks run and the previous one's result comes back.  At most two
 * batches are in flight per index: a third submit returns MICA_EBUSY;
 * collecting an unknown or already collected ticket returns MICA_ENOTFOUND.
 * The caller's host buffers must stay valid and unchanged until the batch is
 * collected; a submit that fails gives no ticket and returns once its copies
 * (if any were queued) have finished.  params->cuda_stream is not used (each slot has its own stream).
 * Batches may be collected in any order.  Calls on one index are not
 * thread-safe; mica_get_stats reports the last collected batch.
 */
int mica_align_submit(mica_index *idx, const uint32_t *packed_reads, const uint64_t *word_offsets,
                      const uint16_t *lengths, const uint8_t *k, uint64_t n_reads,
                      const mica_align_params *params, uint64_t *ticket);
int mica_align_collect(mica_index *idx, uint64_t ticket, mica_result **out);

/*
 * Align a batch already in DEVICE memory (same layout as mica_align_batch).
 * The result stays on the device (see mica_device_result).  The call returns
 * after the result is complete on the given stream.
 */
int mica_align_device(mica_index *idx, const uint32_t *d_packed_reads, const uint64_t *d_word_offsets,
                      const uint16_t *d_lengths, const uint8_t *d_k, uint64_t n_reads,
                      const mica_align_params *params, mica_device_result *out);

int mica_get_stats(const mica_index *idx, mica_stats *out);

/* ---- tuning of the search launch (no effect on results) ---- */
typedef struct {
    int32_t shape;          /* persistent kernel shape, 0 .. mica_tuning_shapes()-1; -1 = default */
    uint32_t plain_block;   /* plain kernel threads per block (32..512, multiple of 32); 0 = 128 */
    uint32_t plain_budget;  /* plain kernel node expansions per task before its rest is re-queued
                               on the device; 0 = 65536 */
    uint32_t plain_block_len[4];  /* MICA_KERNEL_PLAIN_BY_LENGTH: block size per length class;
                                     0 = plain_block */
    int32_t prefetch;       /* persistent kernel: at the end of a round, prefetch into L2 the
                               occurrence blocks of the next round's nodes.  -1 = automatic (on
                               when the occurrence blocks exceed 96 MiB and so do not stay in
                               L2), 0 = off, 1 = on */
    uint32_t bidir_budget;  /* bidirectional kernel: node expansions a task may take before it hands
                               its pending nodes to the next launch round, where they are tasks of
                               their own on every warp (bounds each round's tail; no effect on
                               results); 0 = 4096 */
    uint32_t bidir_verify;  /* bidirectional kernel with full_sa: an interval of one row whose matched
                               part is at least this many bases (and which has at least 8 bases
                               left to match) is checked against the genome's text in one step
                               instead of being extended base by base; 0 = 12, 256 or more = never */
    int32_t bidir_shape;    /* bidirectional kernel shape: 0 = 64 task slots per warp, 6 warps per CTA
                               (fuller rounds when tasks are short); 1 = 32 slots, 8 warps (more warps
                               to hide HBM latency); -1 = automatic (0 when the occurrence blocks fit in
                               96 MiB and stay in L2, else 1) */
} mica_tuning;

/* Number of compiled persistent kernel shapes; mica_tuning_shape_info
   describes one: shared-memory node stack per warp, warps per CTA, minimum
   resident CTAs per SM the registers were limited for. */
int mica_tuning_shapes(void);
int mica_tuning_shape_info(int shape, int *stack_nodes, int *warps_per_cta, int *min_ctas_per_sm);
int mica_set_tuning(mica_index *idx, const mica_tuning *t);
int mica_get_tuning(const mica_index *idx, mica_tuning *t);

/* Bounds of the persistent kernel's device waits (the paper's thread give-up
   rule of Section 2 turned into bounded waits: no wait on the device is
   endless).  idle_rounds: rounds a warp with no work may wait for work before
   the launch gives up (>= 1 us each; 0 = the default, 2^22); ring_spins:
   waits on one slot of the device spill queue (64-128 ns each; 0 = the
   default, 2^24).  A launch that gives up stops every warp, and the align call
   returns MICA_ETIMEOUT with no result; the index stays usable and the next
   call starts afresh.  Small values exist to exercise that path. */
int mica_set_wait_limits(mica_index *idx, uint32_t idle_rounds, uint32_t ring_spins);

/* Autotuner: time every bidirectional kernel shape with node budgets of 1024
   and 4096 (when the index has the reversed genome's table), every persistent
   kernel shape and the plain kernel's block size (over the batch and per
   read-length class, on that class's reads) on a host sample batch, `repeats`
   timed runs after one warm-up each, and keep the fastest in the index's
   tuning (also copied to *out unless NULL). */
int mica_autotune(mica_index *idx, const uint32_t *packed_reads, const uint64_t *word_offsets,
                  const uint16_t *lengths, const uint8_t *k, uint64_t n_reads, uint32_t hit_cap, uint32_t repeats,
                  mica_tuning *out);
/* Tuning cache file (text, one line per key).  The key is the GPU name, the
   genome length, kmer_q, a bit mask of the read-length classes present and the
   largest k.  lookup returns MICA_ENOTFOUND when the key is absent. */
int mica_tuning_cache_store(const char *path, const mica_index *idx, uint32_t length_classes, uint32_t kmax,
                            const mica_tuning *t);
int mica_tuning_cache_lookup(const char *path, const mica_index *idx, uint32_t length_classes, uint32_t kmax,
                             mica_tuning *t);

/* ---- serving: continuous batching over a resident index ----
 *
 * The paper's host keeps the accelerator busy with batches of about a million
 * reads while it handles the waiting (Section 2, "Pipelining & load
 * balancing").  Here a server owns worker threads (each with its own CUDA
 * stream and workspace).  A request is split on submit into chunks of at most
 * chunk_reads reads.  A worker forms a tick by taking the next chunk of every
 * queued request in arrival order, then their following chunks, round after
 * round, while the tick's reads fit max_tick_reads and the device memory its
 * search needs (mica_server_workspace_bytes) fits the worker's share of
 * max_device_bytes; the tick is one search launch, so the work of its
 * requests interleaves on the device, and with two or more workers one tick's
 * search overlaps another's hit assembly and copies.  A large request so
 * advances a chunk per tick beside later small ones.  A request completes
 * when its last chunk does, and its result is identical to aligning it alone
 * with mica_align_batch.  The index must stay alive until mica_server_stop
 * returns; it may still be used by the caller's own align calls (those use
 * the index's workspace, the server uses its own).
 */
typedef struct mica_server mica_server;

typedef struct {
    uint64_t max_device_bytes;  /* device memory for the workers' workspaces (each worker may use an equal
                                   share); 0 = half the free memory at start */
    uint64_t max_tick_reads;    /* reads per search launch; 0 = 2^20 */
    uint32_t hit_cap;           /* as mica_align_params.hit_cap, for every request */
    int32_t kernel;             /* MICA_KERNEL_* (default: bidirectional) */
    int32_t workers;            /* concurrent ticks, 1..8; 0 = 2 */
    int32_t start_paused;       /* nonzero: queue requests but admit none until mica_server_resume */
    uint64_t chunk_reads;       /* largest piece of a request in one tick; 0 = 2^18 (smaller when a
                                   worker's share of the memory cannot hold it) */
} mica_server_params;

typedef struct {
    uint64_t submitted, completed, failed, cancelled;
    uint64_t ticks;             /* search launches run */
    uint64_t reads;             /* reads of completed requests */
    uint64_t pending;           /* requests with chunks not yet admitted */
    uint64_t device_bytes_in_use, device_budget;   /* workspace the workers' ticks have needed (each
                                                      worker's largest; workspaces only grow), budget */
    double busy_s;              /* summed wall time of ticks over all workers */
} mica_server_stats;

void mica_server_params_default(mica_server_params *p);
/* Start the worker threads on idx's device.  params may be NULL (defaults). */
int mica_server_start(mica_index *idx, const mica_server_params *params, mica_server **out);
/* Device bytes a worker's workspace needs to run one tick of n_reads reads
   held in n_words packed words (the staged batch, the search's buffers incl.
   the persistent grid's overflow stacks, and the hit assembly's at 4 hits per
   read): what admission charges against a worker's share. */
int mica_server_workspace_bytes(const mica_index *idx, uint64_t n_reads, uint64_t n_words, uint64_t *bytes);
/* Queue a host batch (same layout as mica_align_batch; copied before return).
   MICA_EINVAL for a bad batch, MICA_ENOMEM if a worker's share of the budget
   cannot hold even a one-read tick (nothing could ever be admitted),
   MICA_EBUSY after stop. */
int mica_server_submit(mica_server *srv, const uint32_t *packed_reads, const uint64_t *word_offsets,
                       const uint16_t *lengths, const uint8_t *k, uint64_t n_reads, uint64_t *req_id);
/* MICA_EBUSY while queued or running.  Once done, returns the request's status
   and hands *out (a mica_result to free with mica_result_free; NULL if out is
   NULL or the request failed) and *latency_ms (submit to completion, host
   clock; may be NULL) to the caller; the id is then forgotten. */
int mica_server_poll(mica_server *srv, uint64_t req_id, mica_result **out, double *latency_ms);
/* As poll, waiting up to timeout_ms; MICA_ETIMEOUT if still not done. */
int mica_server_wait(mica_server *srv, uint64_t req_id, uint32_t timeout_ms, mica_result **out,
                     double *latency_ms);
/* Drop a queued request (MICA_EBUSY once a tick has taken one of its chunks). */
int mica_server_cancel(mica_server *srv, uint64_t req_id);
void mica_server_resume(mica_server *srv);
int mica_server_get_stats(mica_server *srv, mica_server_stats *out);
/* Finish the ticks in flight and the requests they have started, drop the
   queued requests no tick has taken, join the workers, free uncollected
   results. */
void mica_server_stop(mica_server *srv);

/* ---- mate pairing (after the search; no effect on its result) ----
 *
 * The paper benchmarks paired-end reads and reports the share of properly
 * paired ones (Section 3, Table 1).  Reads 2i and 2i + 1 of a batch are the
 * two mates of pair i.  A concordant placement of pair i is a listed hit a of
 * one mate on the + strand and a listed hit b of the other mate on the -
 * strand with fragment length L = b.pos + m_b - a.pos (m_b the length of b's
 * mate) in [insert_min, insert_max] -- the forward/reverse orientation of
 * paired-end sequencing.  Only listed hits are paired: a mate whose total
 * exceeds the cap contributes its listed hits alone.
 *
 * Per pair: n_concordant = number of such (a, b) combinations; mm = the
 * smallest a.mm + b.mm among them and n_best = how many reach it (1 = a
 * unique best placement); pos_plus / pos_minus / plus_mate describe the best
 * one, ties broken by smallest pos_plus, then mate 1 before mate 2 on the +
 * strand, then smallest pos_minus.  With no concordant placement n_concordant
 * = n_best = 0 and the other fields are 0.
 */
typedef struct {
    uint32_t n_concordant;
    uint32_t n_best;
    uint32_t pos_plus;    /* + strand hit of the best placement (fragment start) */
    uint32_t pos_minus;   /* - strand hit of the best placement */
    uint8_t plus_mate;    /* 0: mate 1 is on the + strand, 1: mate 2 */
    uint8_t mm;           /* substitutions of both mates together */
    uint16_t pad;
} mica_pair;

/* Pair the device result of a batch of 2 * n_pairs reads (d_offsets: 2 *
   n_pairs + 1 CSR offsets, d_hits: hits sorted by (pos, strand) per read as
   mica_align_device returns them, d_lengths: read lengths) into d_out[n_pairs]
   on cuda_stream (NULL = legacy default stream) of the current device;
   returns without waiting.  MICA_EINVAL if insert_min > insert_max. */
int mica_pair_device(const uint64_t *d_offsets, const mica_hit *d_hits, const uint16_t *d_lengths,
                     uint64_t n_pairs, uint32_t insert_min, uint32_t insert_max, mica_pair *d_out,
                     void *cuda_stream);
/* The same on host arrays (copied to `device` and back; synchronous). */
int mica_pair_batch(int device, const uint64_t *offsets, const mica_hit *hits, const uint16_t *lengths,
                    uint64_t n_pairs, uint32_t insert_min, uint32_t insert_max, mica_pair *out);

/* ---- reference sequences: contigs, ambiguous bases (host-side) ----
 *
 * The paper aligns reads against a reference genome and hands the BWT
 * phase's placements on to SAM-producing stages (Section 2); a real
 * reference is a set of named contigs whose bytes may hold N or other IUPAC
 * codes.  The index has one text over {A,C,G,T}, so a mica_reference maps the
 * two onto each other, entirely on the host (no CUDA call):
 *
 *   - contig i (in input order) occupies [start_i, start_i + length_i) of the
 *     concatenated text G, start_0 = 0, start_{i+1} = start_i + length_i;
 *   - a byte other than A/C/G/T (either case) is ambiguous: in G it becomes
 *     the base given by the top two bits of SplitMix64 (Steele, Lea and
 *     Flood, 2014) of its coordinate in G, and it is recorded in a maximal
 *     run [s, e) of ambiguous coordinates;
 *   - a placement (p, strand, d) of a read of length m is a placement on the
 *     reference when [p, p + m) lies inside one contig and holds no ambiguous
 *     coordinate.  The others (windows across a contig boundary or over a
 *     replaced base) exist only in G and are dropped by mica_reference_filter
 *     and by the SAM writer.
 *
 * Feed mica_reference_text() to mica_index_build.  The text must stay below
 * 2^32 - 1 bases (the index's limit); contigs are non-empty; names follow
 * SAM's reference-name rule (printable, no whitespace, none of "'(),<>[\]`{},
 * not starting with * or =) and are unique.  A mica_reference is read-only
 * after creation and may be shared between threads.
 */
typedef struct mica_reference mica_reference;

typedef struct {
    uint64_t length;           /* bases of the concatenated text G */
    uint64_t n_contigs;
    uint64_t n_ambiguous_runs; /* maximal runs of ambiguous coordinates */
    uint64_t ambiguous_bases;  /* their total length */
} mica_reference_info;

/* From memory: `sequence` holds the contigs' bytes back to back (len bytes),
   contig i has contig_lengths[i] of them (sum = len).  names[i] is contig i's
   name (NUL-terminated); names = NULL names them contig1, contig2, ....
   MICA_EINVAL on a zero-length contig, lengths that do not sum to len, a bad
   or repeated name, or a text too long for the index. */
int mica_reference_create(const uint8_t *sequence, uint64_t len, const uint64_t *contig_lengths,
                          const char *const *names, uint64_t n_contigs, mica_reference **out);
/* From a FASTA file: each record starts with a '>' line whose first
   whitespace-delimited word is the contig name; the sequence lines that
   follow hold letters (any non-ACGT letter is ambiguous) and whitespace,
   which is skipped; lines starting with ';' are comments.  MICA_EIO when the
   file cannot be read or is malformed (bytes before the first record, a
   character other than a letter or whitespace, an empty record, an empty,
   invalid or repeated name); MICA_EINVAL when the text is too long. */
int mica_reference_read_fasta(const char *path, mica_reference **out);
/* Binary copy (contig table, ambiguous runs, G at 2 bits per base). */
int mica_reference_save(const mica_reference *ref, const char *path);
int mica_reference_load(const char *path, mica_reference **out);   /* MICA_EIO when malformed */
void mica_reference_free(mica_reference *ref);

int mica_reference_get_info(const mica_reference *ref, mica_reference_info *info);
/* *acgt = G as 'A','C','G','T' bytes (owned by ref), *len = its length. */
int mica_reference_text(const mica_reference *ref, const uint8_t **acgt, uint64_t *len);
/* Contig i: *name (owned by ref), *start, *length; MICA_EINVAL when i is out
   of range.  Any output pointer may be NULL. */
int mica_reference_contig(const mica_reference *ref, uint64_t i, const char **name, uint64_t *start,
                          uint64_t *length);
/* Ambiguous run j as [*start, *start + *length) of G; MICA_EINVAL when j is
   out of range. */
int mica_reference_ambiguous_run(const mica_reference *ref, uint64_t j, uint64_t *start, uint64_t *length);

/* For each window [pos[i], pos[i] + span[i]) of G: contig[i] = its contig
   when it is a placement on the reference (inside one contig, no ambiguous
   coordinate), else -1; local[i] = pos[i] - that contig's start (0 for -1).
   MICA_EINVAL when a span is 0 or a window ends past G. */
int mica_reference_locate(const mica_reference *ref, const uint32_t *pos, const uint16_t *span, uint64_t n,
                          int32_t *contig, uint32_t *local);
/* In place on a host result of n_reads reads (read i of length lengths[i]):
   removes the listed hits that are not placements on the reference, keeping
   the others in order, rewrites offsets[0..n_reads] and lowers total[i] by
   the number removed from read i.  total[i] is then exact for every read
   whose hits were all listed (total <= hit cap); for a capped read it is an
   upper bound, since unlisted hits were never located.  *n_dropped
   (optional) = hits removed.  MICA_EINVAL when offsets decrease, a listed
   count exceeds total, or a hit ends past G. */
int mica_reference_filter(const mica_reference *ref, const uint16_t *lengths, uint64_t n_reads, uint64_t *total,
                          uint64_t *offsets, mica_hit *hits, uint64_t *n_dropped);

/* ---- reads from FASTQ (host-side) ----
 *
 * The paper's input is sequencer reads in FASTQ (Section 3: paired-end
 * lanes).  A mica_fastq reads one file, or two files of mates, into batches
 * in the layout mica_align_batch takes, keeping names and qualities for SAM.
 * Each record is four lines: '@' and the name (its first word is kept; a
 * trailing "/1" or "/2" is dropped for mates), the bases, a line starting
 * with '+', and one quality character (33..126) per base; CRLF is accepted
 * and blank lines between records are skipped.  A base other than A/C/G/T
 * (either case; N, IUPAC codes, '.') is ambiguous: the packed read holds the
 * base given by the top two bits of SplitMix64(2^8 * r + j) for read number
 * r of the file (mates numbered 2i, 2i + 1) and offset j, and its offset is
 * recorded.
 *
 * N in reads.  An ambiguous read base matches no reference base, so a
 * placement's substitutions d' count it always.  The search over the packed
 * read never counts it more than that (its stand-in base costs 0 or 1), so
 * every placement with d' <= k is among the search's hits, and
 * mica_read_batch_filter_n keeps exactly those, with d' as their mm: the
 * result is {(p, s, d'): d' <= k}.  For a read listed in full (total <= hit
 * cap) this is exact; for a capped read the cap chose among the search's d
 * and total is an upper bound.
 */
typedef struct mica_fastq mica_fastq;
typedef struct mica_read_batch mica_read_batch;

/* path2 = NULL: single reads; else mates of path1 and path2 interleaved as
   reads 2i and 2i + 1.  MICA_EIO when a file cannot be opened. */
int mica_fastq_open(const char *path1, const char *path2, mica_fastq **out);
/* The next batch: up to max_reads reads (rounded down to even when paired,
   at least 2), each with budget k.  *out = a batch of 0 reads at the end of
   the file(s).  MICA_EIO on a malformed record, names of mates that differ,
   or files of mates of different lengths; MICA_EINVAL on a read of length 0
   or above MICA_MAX_READ_LEN, or k > MICA_MAX_K; after an error the
   reader's position is unspecified (close it).  Records are checked and
   packed on all host threads. */
int mica_fastq_read(mica_fastq *fq, uint64_t max_reads, uint8_t k, mica_read_batch **out);
void mica_fastq_close(mica_fastq *fq);

typedef struct {
    uint64_t n_reads;
    const uint32_t *packed_reads;  /* the layout mica_align_batch takes, owned by the batch */
    const uint64_t *word_offsets;
    const uint16_t *lengths;
    const uint8_t *k;
    uint64_t n_ambiguous_reads;    /* reads with at least one ambiguous base */
    uint32_t paired;               /* 1: reads 2i and 2i + 1 are mates */
} mica_read_batch_view;

int mica_read_batch_get_view(const mica_read_batch *b, mica_read_batch_view *v);
/* Read i's name (owned by the batch), qualities (lengths[i] bytes, not
   NUL-terminated) and ambiguous offsets (ascending).  Any output pointer may
   be NULL. */
int mica_read_batch_read(const mica_read_batch *b, uint64_t i, const char **name, const char **qualities,
                         const uint16_t **ambiguous, uint32_t *n_ambiguous);
void mica_read_batch_free(mica_read_batch *b);

/* In place on the host result of this batch (as mica_reference_filter):
   for every read with ambiguous bases, each listed hit's mm becomes d'
   (mismatches against the reference text plus ambiguous bases) and hits
   with d' > k are removed, total falling by their number.  Idempotent.
   MICA_EINVAL on inconsistent input (offsets, totals, a hit past the text,
   or an mm that is neither the hit's d nor its d'); nothing changes then. */
int mica_read_batch_filter_n(const mica_read_batch *b, const mica_reference *ref, uint64_t *total,
                             uint64_t *offsets, mica_hit *hits, uint64_t *n_dropped);

/* ---- SAM output (host-side) ----
 *
 * Writes the search's placements as SAM 1.6 text (header @HD, one @SQ per
 * contig, @PG).  Per read (numbered from 0 across calls; pairs numbered by
 * pair), of length m, V = its listed hits that are placements on the
 * reference:
 *
 *   - V empty: one unmapped record (FLAG 4, SEQ the read as given);
 *   - else the primary record is the first hit of V (listed order: position,
 *     strand) with the fewest substitutions dmin: RNAME/POS its contig and
 *     1-based contig coordinate, CIGAR mM, FLAG 16 on the - strand with SEQ
 *     the reverse complement (SAM stores the forward strand), QUAL *, tags
 *     NM:i (substitutions, recomputed against G and required to equal the
 *     hit's d), MD:Z (the reference bases at the substitutions), X0:i (hits
 *     of V with dmin), X1:i (hits of V with dmin + 1) and ZT:i (the read's
 *     total less the listed hits dropped, as mica_reference_filter gives);
 *   - MAPQ: 0 unless the best placement is unique (X0 = 1, and the list is
 *     complete or holds a hit with d > dmin, so the cap cut no dmin hit);
 *     then 37 when no placement with dmin + 1 exists (X1 = 0 and the list is
 *     complete or holds a hit with d > dmin + 1), else 25;
 *   - with `secondary`, every other hit of V follows as FLAG 256, MAPQ 0,
 *     SEQ *, with NM and MD.
 *
 * Pairs (mates 2i and 2i + 1, `pairs` from mica_pair_batch on the same
 * result): FLAG 1, and 64 / 128 for mate 1 / 2.  When pairs[i] names a best
 * concordant placement whose two hits are both in V and in the same contig,
 * those hits are the mates' primaries and FLAG 2 (properly paired) is set,
 * with MAPQ 0 when n_best > 1, 37 when the placement is the only concordant
 * one and both mates' lists are complete, else 25.  Otherwise each mate
 * takes its own primary as above.  Mate fields follow SAM: FLAG 8 / 32 for
 * an unmapped / reverse-strand mate, RNEXT = or the mate's contig, PNEXT the
 * mate's POS; an unmapped mate of a mapped read takes that read's RNAME and
 * POS; TLEN = +-(rightmost end - leftmost start) when both are in one
 * contig, + on the mate that starts first (mate 1 on a tie), else 0.
 *
 * A mica_sam_writer keeps a pointer to `ref`: free the reference only after
 * mica_sam_close.  One host thread at a time.
 */
typedef struct mica_sam_writer mica_sam_writer;

typedef struct {
    const char *qname_prefix;  /* QNAME = prefix + read (or pair) number; NULL = "r" */
    uint32_t secondary;        /* 1: also write the other placements of V as secondary records */
    const char *command_line;  /* written as @PG CL: when not NULL */
    uint32_t threads;          /* host threads checking and formatting records, <= 256;
                                  0 = the hardware's thread count */
} mica_sam_params;

void mica_sam_params_default(mica_sam_params *p);
/* Creates or truncates `path` and writes the header.  MICA_EIO when the file
   cannot be written; MICA_EINVAL on a prefix with whitespace or a command
   line with a tab or newline, or more than 256 threads. */
int mica_sam_open(const char *path, const mica_reference *ref, const mica_sam_params *params,
                  mica_sam_writer **out);
/* Appends the records of a batch of n_reads reads (host arrays, the layout
   mica_align_batch takes and returns).  pairs = NULL: single reads;
   otherwise n_reads is even and pairs holds n_reads / 2 entries.  MICA_EINVAL
   on inconsistent input (offsets decrease, more listed hits than total, a hit
   that ends past G, or a hit whose d differs from its substitutions against
   G, which means the result does not belong to these reads and this
   reference); nothing of the batch is written then.  MICA_EIO on a write
   error and MICA_ENOMEM when a formatting buffer cannot grow; part of the
   batch may have been written then.  Records come out in read order
   whatever the thread count. */
int mica_sam_write(mica_sam_writer *w, const uint32_t *packed_reads, const uint64_t *word_offsets,
                   const uint16_t *lengths, uint64_t n_reads, const uint64_t *total, const uint64_t *offsets,
                   const mica_hit *hits, const mica_pair *pairs);
/* As mica_sam_write for a batch from mica_fastq_read, with its names,
   qualities and ambiguous bases: QNAME is the read's name (mate 1's for a
   pair), SEQ shows ambiguous bases as N, QUAL holds the read's qualities
   (reversed on the - strand), NM and MD count ambiguous bases as
   substitutions (d'), and hits with d' > k are left out as
   mica_read_batch_filter_n leaves them out; the hits may be given before or
   after that filter.  pairs: the pairing of a paired batch's result
   (mica_pair_batch), or NULL, which writes its mates as pairs with none
   properly paired; must be NULL for a batch of single reads.  The numbering
   of mica_sam_write is not used or advanced. */
int mica_sam_write_batch(mica_sam_writer *w, const mica_read_batch *b, const uint64_t *total,
                         const uint64_t *offsets, const mica_hit *hits, const mica_pair *pairs);
/* Flushes and closes the file and frees the writer (also on error).
   MICA_EIO when the final write fails. */
int mica_sam_close(mica_sam_writer *w);

/* ---- hit-list offsets for callers that cannot allocate device memory ----
 *
 * The paper has no counterpart: this serves callers that may not call
 * cudaMalloc (code running during CUDA graph capture, services whose device
 * memory belongs to another allocator or pool, processes that must keep a
 * fixed footprint after start-up).  mica_offsets_noalloc turns n per-read hit
 * counts (device, uint64) into the n + 1 CSR offsets (device, uint64):
 * d_offsets[0] = 0, d_offsets[i+1] = d_offsets[i] + d_counts[i] -- the
 * offsets a mica_device_result holds for its listed hits.  It allocates
 * nothing: its scratch is a fixed 64 KiB array that every GPU loading the
 * library holds until exit.  n may be at most MICA_NOALLOC_MAX_COUNTS; larger
 * n returns MICA_EINVAL before any work.  It runs on cuda_stream (NULL = the
 * legacy default stream) on the current device and returns without waiting.
 * The first call on a device looks the scratch up on that device, and so does
 * the first call after the device's context was replaced (a device reset);
 * make such a call before any stream capture.  All calls share the one scratch
 * array, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race: serialise them.
 */
#define MICA_NOALLOC_MAX_COUNTS (1ull << 24)
int mica_offsets_noalloc(const uint64_t *d_counts, uint64_t n, uint64_t *d_offsets, void *cuda_stream);

/* ---- random-gather ceiling (measurement) ----
 *
 * The paper locates the BWT phase's bottleneck in access to the index in
 * memory (Section 3); the search reads one 32-byte occurrence block per
 * dependent step at a random row.  mica_gather_ceiling measures what this GPU
 * sustains for that pattern: every thread of a full-occupancy grid makes
 * independent loads of load_bytes (16, 32, 64 or 128) at uniformly random
 * load_bytes-aligned offsets of a fresh device buffer of buffer_bytes (a
 * multiple of load_bytes, >= 4096), about `loads` loads per launch.  *gbs
 * (required) = bytes loaded / best launch time over `repeats` timed launches
 * (0 = 1) after one warm-up, in 1e9 bytes/s; *ms (optional) = that time.
 * A buffer well above L2 gives the HBM random-sector ceiling, one the size
 * of a small index the L2 one.  The buffer is allocated and freed inside the
 * call on `device`; MICA_ENOMEM if it does not fit, MICA_EINVAL on bad sizes.
 * Synchronous on the legacy default stream.
 */
int mica_gather_ceiling(int device, uint64_t buffer_bytes, uint32_t load_bytes, uint64_t loads, uint32_t repeats,
                        double *gbs, double *ms);

/* ---- parity probes: each exposes one step of the path on the GPU ---- */

/* Suffix array of G$ (len + 1 entries, host output) built on the GPU by the
   same prefix-doubling code the index builder uses. */
int mica_debug_suffix_array(const uint8_t *genome_acgt, uint64_t len, int device, uint32_t *sa_out);

/* occ_out[4*i + c] = Occ(c, rows[i]) from the interleaved blocks (host in/out). */
int mica_debug_occ(const mica_index *idx, const uint64_t *rows, uint64_t n, uint32_t *occ_out);

/* pos_out[i] = SA[rows[i]] resolved by LF walks to the sampled rows (host in/out),
   whether or not the index keeps the whole suffix array. */
int mica_debug_locate(const mica_index *idx, const uint64_t *rows, uint64_t n, uint32_t *pos_out);

/* Copy entries [first, first + n) of one of the full_sa arrays to out (host):
   which = 0: the suffix array SA[0, N]; 1: its inverse ISA[0, N] (ISA[SA[j]]
   = j); 2: the genome as 2-bit codes, 16 per uint32 word, least-significant
   bits first (word w holds G[16 w, 16 w + 16), zero past N).  MICA_EINVAL
   for an index without them or a range past the array. */
int mica_debug_full_sa(const mica_index *idx, uint32_t which, uint64_t first, uint64_t n, uint32_t *out);

/* SA interval of each len-mer (len <= kmer_q) given by its code (first base
   most significant, codes[i] < 4^len), looked up in the q-mer table on the
   GPU as the search's seed step does: lr_out[2i] = l, lr_out[2i+1] = r
   (host in/out; l == r when the len-mer does not occur). */
int mica_debug_seed_interval(const mica_index *idx, const uint32_t *codes, uint32_t len, uint64_t n,
                             uint32_t *lr_out);

/* The same from one of the index's seed tables: which = 0 the q-mer table of
   G$, 1 that of the reversed genome G~$ (intervals of the reversed string's
   rows), 2 and 3 the longer seed tables of G$ and G~$ (mica_index_info
   long_q; built with full_sa); len <= that table's q.  MICA_EINVAL for a
   table the index does not have. */
int mica_debug_table_interval(const mica_index *idx, uint32_t which, const uint32_t *codes, uint32_t len,
                              uint64_t n, uint32_t *lr_out);

/* Mismatch lower bounds of every (read, strand) task as the pruned search
   computes them (host in/out; the index must have lower_bounds).  Task
   2i + s is read i on strand s (0 = the read, 1 = its reverse complement):
   P = that strand's pattern, m = |P|, q' = min(m, kmer_q).  Scanning
   P[0, m - q') left to right, a piece P[s, j] that does not occur in the
   genome ends at j and the next piece starts at j + 1; 9-bit field t of
   lb_out[task] (t = 0..3) is j + 1 for the (t+1)-th such piece, 511 where
   there is none, and the scan stops after k + 1 pieces.  D(i), the number of
   fields <= i, bounds from below the substitutions P[0, i) needs. */
int mica_debug_lower_bounds(mica_index *idx, const uint32_t *packed_reads, const uint64_t *word_offsets,
                            const uint16_t *lengths, const uint8_t *k, uint64_t n_reads, uint64_t *lb_out);

#ifdef __cplusplus
}
#endif
#endif /* MICA_H */
