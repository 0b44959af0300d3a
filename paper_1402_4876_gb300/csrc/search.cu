// k-mismatch backward search over the resident FM index (MICA, Section 2:
// "align with few mismatches" using the BWT index; the paper's load-balancing
// rule that a thread may give up on resource-demanding repetitive reads is
// kept, but the work goes back to a device queue, never to the host).
//
// A (read, strand) task searches pattern P = R or rc(R) right to left.  Its
// last qe = min(q, m) bases are looked up directly in the q-mer table for
// every way of substituting at most k of them (the "seed variants"); each
// non-empty interval continues base by base: a node (i, [l, r), d) has a
// child for every symbol c with l' = C[c] + Occ(c, l) < r' = C[c] + Occ(c, r)
// and d + [c != P[i-1]] <= k; nodes with i = 0 are leaf intervals.  With
// lower bounds (k_lower_bounds, from the reversed genome) a child at depth i
// must also satisfy d + D(i) <= k, and the seed window takes at most
// k - D(m - qe) substitutions: branches that cannot reach a hit are dropped,
// the leaf set is unchanged.
//
// Two kernels produce the same leaf set:
//   * k_plain:      one task per thread, depth-first with a stack in local
//                   memory; a task over its node budget pushes its pending
//                   nodes (and untried seeds) to a re-queue that the next
//                   launch drains.
//   * k_persistent: one CTA per SM slot, each warp a work pool of up to 32
//                   tasks.  Every round the 32 lanes take the newest nodes
//                   of one kind from the warp's shared-memory stacks (or
//                   seed lookups of one task), extend them in parallel, and
//                   compact the children back with ballot/shuffle prefix
//                   sums.  Full stacks move their oldest nodes to the warp's
//                   overflow stacks in global memory; near the end of a batch
//                   warps donate nodes through a bounded ring to idle warps.
#include <algorithm>
#include <mutex>

#include "search_common.cuh"

namespace mica {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void emit_interval(SearchCtl *ctl, Interval *iv, uint32_t *iv_cnt,
                                              uint32_t read, uint32_t strand, uint32_t d,
                                              uint32_t l, uint32_t r)
{
    uint32_t at = atomicAdd(&ctl->iv_count, 1u);
    atomicAdd(&iv_cnt[read], 1u);
    if (at < ctl->iv_cap) {
        Interval x;
        x.read = read;
        x.meta = d | (strand << 2);
        x.l = l;
        x.r = r;
        iv[at] = x;
    } else {
        atomicOr(&ctl->error, ERR_IV_OVERFLOW);
    }
}

__device__ __forceinline__ uint32_t sel4(const uint32_t (&v)[4], uint32_t c)
{
    return c == 0 ? v[0] : c == 1 ? v[1] : c == 2 ? v[2] : v[3];
}

// Build the strand's pattern for read `read` into pat[0..W).
__device__ __forceinline__ void thread_pattern(const ReadsView &rd, uint32_t read, uint32_t minus,
                                               uint32_t m, uint32_t *pat)
{
    const uint32_t *w = rd.words + rd.word_off[read];
    uint32_t W = (m + 15) >> 4;
    if (!minus) {
        for (uint32_t j = 0; j < W; j++) pat[j] = w[j];
    } else {
        for (uint32_t j = 0; j < W; j++) {
            uint32_t hi = w[W - 1 - j];
            uint32_t lo = (j + 1 < W) ? w[W - 2 - j] : 0u;
            pat[j] = rc_word(hi, lo, m);
        }
    }
}

// --------------------------------------------------------------------------
// Mismatch lower bounds (Li and Durbin's D array, from the reversed genome)
// --------------------------------------------------------------------------
//
// The search consumes a task's pattern P from its last base; a node at depth
// i has P[0, i) still to match with at most k - d mismatches.  Cutting P[0, i)
// left to right into maximal pieces that occur in G, every piece that does
// not occur forces one mismatch in any placement, so the number D(i) of such
// failed pieces bounds the mismatches P[0, i) needs from below, and a node
// with d + D(i) > k cannot reach a hit.  Whether P[s, j] occurs in G is one
// backward-search step per base on the reversed genome, P read left to right.
// The bound is kept as its breakpoints: field t (9 bits) of a task's word is
// the prefix length at which D reaches t + 1 (511 = never), so
// D(i) = #{t : field t <= i}; at most k + 1 fields are set.

constexpr unsigned long long LB_NONE = ~0ull;   // every field 511: D = 0

__device__ __forceinline__ uint32_t lb_at(unsigned long long v, uint32_t i)
{
    return ((uint32_t)(v & 511u) <= i) + ((uint32_t)((v >> 9) & 511u) <= i) +
           ((uint32_t)((v >> 18) & 511u) <= i) + ((uint32_t)((v >> 27) & 511u) <= i);
}

// Budget left for P[0, i) at d mismatches used: k - D(i), negative = dead.
__device__ __forceinline__ int lb_budget(unsigned long long v, uint32_t k, uint32_t i)
{
    return (int)k - (int)lb_at(v, i);
}

// Occ(c, l) and Occ(c, r) for one symbol c (one block read when l and r share
// it); returns the 32-byte blocks touched.
__device__ __forceinline__ uint32_t occ_single_pair(const IndexView &ix, uint32_t l, uint32_t r, uint32_t c,
                                                    uint32_t &ol, uint32_t &orr)
{
    uint32_t bl = l / OCC_ROWS, xl = l - bl * OCC_ROWS;
    uint32_t br = r / OCC_ROWS, xr = r - br * OCC_ROWS;
    uint4 sl = ld_nc(ix.super + bl / SB_BLOCKS);
    OccBlock a;
    if (bl == br) {
        load_block(ix, bl, xr, a);
        ol = occ_single(ix, bl, xl, sl, a, c);
        orr = occ_single(ix, br, xr, sl, a, c);
        return 1;
    }
    uint4 sr = ld_nc(ix.super + br / SB_BLOCKS);
    OccBlock b;
    load_block(ix, bl, xl, a);
    load_block(ix, br, xr, b);
    ol = occ_single(ix, bl, xl, sl, a, c);
    orr = occ_single(ix, br, xr, sr, b, c);
    return 2;
}

__global__ void __launch_bounds__(256) k_lower_bounds(const IndexView ix, const ReadsView rd,
                                                      unsigned long long *__restrict__ lb, SearchCtl *ctl,
                                                      const uint32_t *__restrict__ read_list = nullptr,
                                                      uint64_t n_list = 0)
{
    IndexView rv = ix;            // the reversed genome's blocks through the same helpers
    rv.occ = ix.rev.occ;
    rv.super = ix.rev.super;
    rv.dollar_row = ix.rev.dollar_row;
#pragma unroll
    for (int c = 0; c < 5; c++) rv.C[c] = ix.rev.C[c];
    const uint64_t ntasks = 2 * (read_list ? n_list : rd.n);
    uint32_t steps = 0, blocks = 0, dead = 0;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < ntasks;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t rid = read_list ? read_list[t >> 1] : (uint32_t)(t >> 1), minus = (uint32_t)(t & 1);
        const uint32_t m = rd.len[rid], k = rd.k[rid];
        const uint32_t qe = m < ix.q ? m : ix.q, lim = m - qe;
        const uint32_t *w = rd.words + rd.word_off[rid];
        unsigned long long v = LB_NONE;
        uint32_t z = 0, l = 0, r = 0;
        bool fresh = true;
        for (uint32_t j = 0; j < lim; j++) {
            uint32_t jj = minus ? m - 1 - j : j;
            uint32_t c = (__ldg(w + (jj >> 4)) >> (2 * (jj & 15))) & 3u;
            if (minus) c = 3u - c;
            const uint32_t cbase = C_of(rv, c);
            if (fresh) {
                l = cbase;
                r = c == 0 ? rv.C[1] : c == 1 ? rv.C[2] : c == 2 ? rv.C[3] : rv.C[4];
                fresh = false;
            } else {
                uint32_t ol, orr;
                blocks += occ_single_pair(rv, l, r, c, ol, orr);
                steps++;
                l = cbase + ol;
                r = cbase + orr;
            }
            if (l >= r) {
                // P[s, j] does not occur: one more forced mismatch from prefix j + 1 on
                v = (v & ~(511ull << (9 * z))) | ((unsigned long long)(j + 1) << (9 * z));
                fresh = true;
                if (++z > k) break;
            }
        }
        lb[2ull * rid + minus] = v;
        dead += z > k;
    }
    unsigned mask = __activemask();
    unsigned s1 = __reduce_add_sync(mask, steps), s2 = __reduce_add_sync(mask, blocks),
             s3 = __reduce_add_sync(mask, dead);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
        if (s1) atomicAdd(&ctl->lb_steps, (unsigned long long)s1);
        if (s2) atomicAdd(&ctl->rank_blocks, (unsigned long long)s2);
        if (s3) atomicAdd(&ctl->lb_dead, (unsigned long long)s3);
    }
}

// --------------------------------------------------------------------------
// Plain kernel: one work item per thread
// --------------------------------------------------------------------------

constexpr int PLAIN_STACK = 48;

struct PlainArgs {
    IndexView ix;
    ReadsView rd;
    const uint32_t *read_list;   // optional: task t -> read_list[t >> 1]
    const WorkItem *items;       // optional: items mode
    uint64_t ntasks;
    SearchCtl *ctl;
    Interval *iv;
    uint32_t *iv_cnt;
    WorkItem *requeue;           // output re-queue
    unsigned int *requeue_count;
    uint32_t requeue_cap;
    uint32_t budget;             // node expansions before re-queueing the rest
    const unsigned long long *lb;   // optional: lower-bound breakpoints per (read, strand)
};

__device__ __forceinline__ void requeue_push(const PlainArgs &a, uint32_t read, uint32_t meta,
                                             uint32_t x, uint32_t y)
{
    uint32_t at = atomicAdd(a.requeue_count, 1u);
    if (at < a.requeue_cap) {
        WorkItem it;
        it.read = read;
        it.meta = meta;   // a plain array: the persistent kernel's ring publishes through sequence words
        it.a = x;
        it.b = y;
        a.requeue[at] = it;
    } else {
        atomicOr(&a.ctl->error, ERR_SPILL_OVERFLOW);
    }
}

__global__ void __launch_bounds__(512) k_plain(PlainArgs a)
{
    uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= a.ntasks) return;
    const IndexView &ix = a.ix;
    uint32_t read, minus, vbeg, vend, kind_node = 0, n_l = 0, n_r = 0, n_i = 0, n_d = 0;
    if (a.items) {
        WorkItem it = a.items[t];
        read = it.read;
        minus = (it.meta & WI_MINUS) ? 1u : 0u;
        if (it.meta & WI_NODE) {
            kind_node = 1;
            n_l = it.a; n_r = it.b; n_i = (it.meta >> 8) & 511u; n_d = it.meta & 3u;
            vbeg = vend = 0;
        } else {
            vbeg = it.a; vend = it.b;
        }
    } else {
        read = a.read_list ? a.read_list[t >> 1] : (uint32_t)(t >> 1);
        minus = (uint32_t)(t & 1);
        vbeg = 0;
        vend = 0xffffffffu;   // resolved below
    }
    uint32_t m = a.rd.len[read], k = a.rd.k[read];
    uint32_t qe = m < ix.q ? m : ix.q;
    const unsigned long long lbv = a.lb ? a.lb[2ull * read + minus] : LB_NONE;
    // seeds: the window's substitutions may use only what the rest cannot need
    const int keff = lb_budget(lbv, k, m - qe);
    uint32_t V = keff < 0 ? 0u : n_variants(qe, (uint32_t)keff);
    if (vend > V) vend = V;
    uint32_t pat[MAX_WORDS];
    thread_pattern(a.rd, read, minus, m, pat);
    uint32_t code = window_code(pat, m, qe);
    const uint32_t *var = ix.variants + var_off(keff < 0 ? 0u : (uint32_t)keff);

    uint32_t st_l[PLAIN_STACK], st_r[PLAIN_STACK], st_m[PLAIN_STACK];
    int sp = 0;
    uint32_t spent = 0;
    unsigned long long seeds = 0, nodes = 0, blocks = 0, spills = 0;
    uint32_t smeta = (minus ? WI_MINUS : 0u);

    if (kind_node) {
        st_l[0] = n_l; st_r[0] = n_r; st_m[0] = n_i | (n_d << 9); sp = 1;
    }
    uint32_t v = vbeg;
    for (;;) {
        if (sp == 0) {
            // next seed variant
            if (v >= vend) break;
            if (spent >= a.budget) {
                requeue_push(a, read, smeta, v, vend);
                spills++;
                break;
            }
            uint32_t w = __ldg(var + v);
            v++;
            seeds++;
            uint32_t l, r;
            seed_interval(ix, code ^ (w & 0xffffffu), qe, l, r);
            if (l >= r) continue;
            uint32_t d = w >> 24, i = m - qe;
            if (i == 0) { emit_interval(a.ctl, a.iv, a.iv_cnt, read, minus, d, l, r); continue; }
            st_l[0] = l; st_r[0] = r; st_m[0] = i | (d << 9); sp = 1;
            continue;
        }
        if (spent >= a.budget) {
            // over budget: re-queue every pending node and the untried seeds
            for (int s = 0; s < sp; s++) {
                requeue_push(a, read, smeta | WI_NODE | ((st_m[s] & 511u) << 8) | (st_m[s] >> 9),
                             st_l[s], st_r[s]);
                spills++;
            }
            if (v < vend) { requeue_push(a, read, smeta, v, vend); spills++; }
            break;
        }
        sp--;
        uint32_t l = st_l[sp], r = st_r[sp], i = st_m[sp] & 511u, d = st_m[sp] >> 9;
        uint32_t ol[4], orr[4];
        blocks += occ_pair(ix, l, r, ol, orr);
        nodes++;
        spent++;
        uint32_t base = pat_base(pat, i - 1);
        const int kb = lb_budget(lbv, k, i - 1);   // mismatches children may hold
        // mismatching children first, the matching child last (popped next)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            uint32_t cc = (uint32_t)c;
            if (cc == base || (int)d + 1 > kb) continue;
            uint32_t l2 = ix.C[c] + ol[c], r2 = ix.C[c] + orr[c];
            if (l2 >= r2) continue;
            if (i == 1) { emit_interval(a.ctl, a.iv, a.iv_cnt, read, minus, d + 1, l2, r2); continue; }
            if (sp < PLAIN_STACK) {
                st_l[sp] = l2; st_r[sp] = r2; st_m[sp] = (i - 1) | ((d + 1) << 9); sp++;
            } else {
                requeue_push(a, read, smeta | WI_NODE | ((i - 1) << 8) | (d + 1), l2, r2);
                spills++;
            }
        }
        if ((int)d <= kb) {
            uint32_t l2 = ix.C[base] + sel4(ol, base), r2 = ix.C[base] + sel4(orr, base);
            if (l2 < r2) {
                if (i == 1) {
                    emit_interval(a.ctl, a.iv, a.iv_cnt, read, minus, d, l2, r2);
                } else if (sp < PLAIN_STACK) {
                    st_l[sp] = l2; st_r[sp] = r2; st_m[sp] = (i - 1) | (d << 9); sp++;
                } else {
                    requeue_push(a, read, smeta | WI_NODE | ((i - 1) << 8) | d, l2, r2);
                    spills++;
                }
            }
        }
    }
    // counters, aggregated over the lanes that reach this point together
    unsigned mask = __activemask();
    unsigned s_seeds = __reduce_add_sync(mask, (unsigned)seeds);
    unsigned s_nodes = __reduce_add_sync(mask, (unsigned)nodes);
    unsigned s_blocks = __reduce_add_sync(mask, (unsigned)blocks);
    unsigned s_spills = __reduce_add_sync(mask, (unsigned)spills);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
        atomicAdd(&a.ctl->seeds, (unsigned long long)s_seeds);
        atomicAdd(&a.ctl->nodes, (unsigned long long)s_nodes);
        atomicAdd(&a.ctl->rank_blocks, (unsigned long long)s_blocks);
        if (s_spills) atomicAdd(&a.ctl->spills, (unsigned long long)s_spills);
    }
}

// reads grouped by length class for per-length plain launches
__device__ __forceinline__ uint32_t len_class(uint32_t m) { return m <= 64 ? 0u : m <= 128 ? 1u : m <= 192 ? 2u : 3u; }

__global__ void k_len_count(ReadsView rd, unsigned int *counts)
{
    __shared__ unsigned int c[LEN_CLASSES];
    if (threadIdx.x < LEN_CLASSES) c[threadIdx.x] = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < rd.n; i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&c[len_class(rd.len[i])], 1u);
    __syncthreads();
    if (threadIdx.x < LEN_CLASSES && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
}

__global__ void k_len_scatter(ReadsView rd, const unsigned int *base, unsigned int *cursor, uint32_t *list)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < rd.n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c = len_class(rd.len[i]);
        list[base[c] + atomicAdd(&cursor[c], 1u)] = (uint32_t)i;
    }
}

// Best-stratum deepening: pass j searches the reads of `list` with budget
// min(k, j) (written into k_pass); the reads that found nothing and allow
// more mismatches form the next pass's list.
__global__ void k_stratum_pass(const uint32_t *__restrict__ list, uint32_t n_list, const uint8_t *__restrict__ k,
                               uint32_t j, uint8_t *__restrict__ k_pass)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_list; t += gridDim.x * blockDim.x) {
        uint32_t r = list[t];
        k_pass[r] = (uint8_t)min((uint32_t)k[r], j);
    }
}

__global__ void k_stratum_next(const uint32_t *__restrict__ list, uint32_t n_list,
                               const uint32_t *__restrict__ iv_cnt, const uint8_t *__restrict__ k, uint32_t j,
                               uint32_t *__restrict__ next, unsigned int *__restrict__ n_next)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_list; t += gridDim.x * blockDim.x) {
        uint32_t r = list[t];
        if (iv_cnt[r] == 0 && k[r] > j) next[atomicAdd(n_next, 1u)] = r;
    }
}

__global__ void k_iota(uint32_t *list, uint32_t n)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) list[t] = t;
}

// The spill ring's sequence words for a fresh launch: slot i expects
// position i.
__global__ void k_ring_init(uint32_t *seq, uint32_t cap)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) seq[i] = i;
}

// --------------------------------------------------------------------------
// Persistent warp-pool kernel
// --------------------------------------------------------------------------

constexpr uint32_t ADMIT_LOW = 64;          // admit tasks when pending work < this
// ... and, while holding work, once at least PersistArgs::admit_min_free slots
// are free: an admission costs a few memory round trips whatever it takes, so
// it should fill several slots -- 8, or 16 when the index lives in HBM and
// the round trips are longer (measured faster on each genome)
// Bounded waits: the defaults of PersistArgs::idle_limit (idle rounds of
// >= 1 us each before the kernel gives up with ERR_TIMEOUT) and
// PersistArgs::spin_limit (waits of 64-128 ns on one ring slot: ~1-2 s);
// mica_set_wait_limits overrides both.
constexpr uint32_t IDLE_LIMIT = 1u << 22;
constexpr uint32_t SPIN_LIMIT = 1u << 24;
constexpr uint32_t RESERVE_LIMIT = 1u << 20; // spill reservation attempts (lost races back off)
constexpr uint32_t FULL_WAITS = 1024;        // waits on a full ring before a room spill gives up
constexpr uint32_t DONATE_TRIES = 8;         // reservation attempts of a donation under contention
constexpr uint32_t DEEP_CAP = 8192;          // entries of each per-warp overflow stack
constexpr uint32_t DONATE_MIN = 96;          // stack depth that makes a warp share work
constexpr uint32_t DONATE_N = 128;
constexpr int DEFAULT_SHAPE = 0;   // 256-node stacks, 8 warps, 3 CTAs per SM: fastest measured
                                   // on both the 64 Mbp and the 3.1 Gbp genome

struct PersistArgs {
    IndexView ix;
    ReadsView rd;
    const uint32_t *read_list;
    uint64_t ntasks;
    SearchCtl *ctl;
    Interval *iv;
    uint32_t *iv_cnt;
    WorkItem *spill;
    uint32_t *seq;                  // spill ring: one sequence word per slot
    uint4 *deep_m;                  // per-warp overflow stacks in global memory: multi-row nodes
    uint2 *deep_s;                  //   and single-row nodes, DEEP_CAP entries per warp each
    int total_warps;
    bool prefetch;                  // warm the next round's occurrence blocks in L2
    int admit_min_free;             // free slots that make a warp holding work admit more
    const unsigned long long *lb;   // optional: lower-bound breakpoints per (read, strand)
    uint32_t idle_limit;            // idle rounds before ERR_TIMEOUT
    uint32_t spin_limit;            // waits on one spill-ring slot before ERR_TIMEOUT
};

template <int SCAP>
struct WarpSmem {
    uint32_t ml[SCAP];                    // multi-row nodes [l, r), r - l > 1
    uint32_t mr[SCAP];
    uint16_t mm[SCAP];                    // slot | i << 5 | d << 14
    uint32_t sl[SCAP];                    // single-row nodes [l, l + 1)
    uint16_t sm[SCAP];
    uint32_t pat[32][MAX_WORDS + 1];      // pattern of each task slot
    unsigned long long lb[32];            // lower-bound breakpoints of each slot
    int live[32];                         // nodes of each slot in the two stacks
    uint8_t rank_lane[32];                // admission: the slot of the j-th new task
};

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t x, int lane)
{
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
    }
    return v - x;
}

__device__ __forceinline__ uint32_t vload(const unsigned int *p) { return *(const volatile unsigned int *)p; }
__device__ __forceinline__ unsigned long long vload64(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

__device__ __forceinline__ uint16_t node_meta(uint32_t slot, uint32_t i, uint32_t d)
{
    return (uint16_t)(slot | (i << 5) | (d << 14));
}

// Move the `nsp` oldest nodes of one stack to the device spill queue, a
// bounded ring of spill_cap (a power of two) work items with one sequence
// word per slot (Vyukov's bounded multi-producer multi-consumer queue):
// slot p % cap may be written for position p when its sequence is p, is
// readable when it is p + 1, and is released for position p + cap after the
// read.  Slots are reserved only while the items reserved and not yet
// claimed fit in the ring, so a producer waits (bounded) only for a consumer
// that has already claimed the previous item and is reading it.  A full ring refuses a donation (returns false, stack unchanged);
// when the nodes must go to make room, they are dropped and the overflow flag
// makes the host rerun the batch with a larger ring.
template <int SCAP, bool SINGLE>
__device__ __forceinline__ bool spill_bottom(WarpSmem<SCAP> &W, const PersistArgs &a, uint32_t &bot,
                                             uint32_t nsp, uint32_t s_read, uint32_t s_info, int lane,
                                             uint32_t &c_spills, bool donation)
{
    SearchCtl *ctl = a.ctl;
    const uint32_t cap = ctl->spill_cap;
    uint32_t at0 = 0;
    int ok = 0;
    if (lane == 0) {
        uint32_t full_waits = 0;
        unsigned long long waited = 0;
        for (uint32_t tries = 0; tries < RESERVE_LIMIT; tries++) {
            // both counters only grow and claims never pass reservations: with
            // H read first R - H >= 0 over-estimates the backlog at the CAS
            // below (a negative difference is a stale read, treated as full)
            uint32_t H = atomicAdd(&ctl->spill_head, 0u);
            uint32_t R = atomicAdd(&ctl->spill_reserve, 0u);
            if ((int)(R - H) < 0 || (R - H) + nsp > cap) {
                // full: a donation gives up, room waits a little for readers
                if (donation || ++full_waits > FULL_WAITS) break;
                __nanosleep(256);
                waited += 256;
                continue;
            }
            if (atomicCAS(&ctl->spill_reserve, R, R + nsp) == R) { at0 = R; ok = 1; break; }
            if (donation && tries + 1 >= DONATE_TRIES) break;   // contended: the donor keeps its nodes
            __nanosleep(32 + 8 * (tries & 31));     // lost the race to another producer: back off
            waited += 32 + 8 * (tries & 31);
        }
        if (waited) atomicAdd(&ctl->wait_queue_ns, waited);
        if (!ok && !donation) atomicOr(&ctl->error, ERR_SPILL_OVERFLOW);
    }
    ok = __shfl_sync(FULL, ok, 0);
    at0 = __shfl_sync(FULL, at0, 0);
    if (!ok && donation) return false;
    for (uint32_t r0 = 0; r0 < nsp; r0 += 32) {
        uint32_t j = r0 + lane;
        bool act = j < nsp;
        uint32_t p = (bot + j) & (SCAP - 1);
        uint32_t l = 0, r = 0, mm = 0;
        if (act) {
            if (SINGLE) { l = W.sl[p]; r = l + 1; mm = W.sm[p]; }
            else { l = W.ml[p]; r = W.mr[p]; mm = W.mm[p]; }
        }
        uint32_t sl = mm & 31u;
        uint32_t rid = __shfl_sync(FULL, s_read, sl);
        uint32_t info = __shfl_sync(FULL, s_info, sl);
        if (act) {
            if (ok) {
                const uint32_t pos = at0 + j, slot_i = pos & (cap - 1);
                WorkItem *it = a.spill + slot_i;
                volatile uint32_t *sq = a.seq + slot_i;
                uint32_t spin = 0;
                bool free_ = true;
                while (*sq != pos) {               // previous lap's item not read yet
                    if (++spin > a.spin_limit) { atomicOr(&ctl->error, ERR_TIMEOUT); free_ = false; break; }
                    __nanosleep(64);
                }
                if (spin) atomicAdd(&ctl->wait_queue_ns, 64ull * spin);
                if (free_) {
                    __threadfence();
                    it->read = rid;
                    it->a = l;
                    it->b = r;
                    it->meta = WI_NODE | (((info >> 11) & 1u) ? WI_MINUS : 0u) | (((mm >> 5) & 511u) << 8) |
                               (mm >> 14);
                    __threadfence();
                    *sq = pos + 1;                 // published
                }
            }
            atomicAdd(&W.live[sl], -1);
        }
    }
    bot += nsp;
    if (lane == 0) c_spills += nsp;
    __syncwarp();
    return true;
}

// The warp's private overflow stacks: when a shared-memory stack is full its
// oldest nodes move to global memory (coalesced, no atomics, no other warp
// involved) and come back under the stack's bottom when it runs low, so the
// order stays depth-first and the nodes keep their task slots.
__device__ __forceinline__ uint4 *deep_m_of(const PersistArgs &a, int warp_global)
{
    return a.deep_m + (size_t)warp_global * DEEP_CAP;
}
__device__ __forceinline__ uint2 *deep_s_of(const PersistArgs &a, int warp_global)
{
    return a.deep_s + (size_t)warp_global * DEEP_CAP;
}

// Move the `n` oldest nodes of a stack to its overflow stack (n fits).
template <int SCAP, bool SINGLE>
__device__ __forceinline__ void deep_push(WarpSmem<SCAP> &W, const PersistArgs &a, int wg, uint32_t &dtop,
                                          uint32_t &bot, uint32_t n, int lane)
{
    for (uint32_t r0 = 0; r0 < n; r0 += 32) {
        uint32_t j = r0 + (uint32_t)lane;
        if (j < n) {
            uint32_t p = (bot + j) & (SCAP - 1);
            if (SINGLE) deep_s_of(a, wg)[dtop + j] = make_uint2(W.sl[p], W.sm[p]);
            else deep_m_of(a, wg)[dtop + j] = make_uint4(W.ml[p], W.mr[p], W.mm[p], 0u);
        }
    }
    dtop += n;
    bot += n;
    __syncwarp();
}

// Bring the `n` most recently moved nodes back under the stack's bottom.
template <int SCAP, bool SINGLE>
__device__ __forceinline__ void deep_pop(WarpSmem<SCAP> &W, const PersistArgs &a, int wg, uint32_t &dtop,
                                         uint32_t &bot, uint32_t n, int lane)
{
    for (uint32_t r0 = 0; r0 < n; r0 += 32) {
        uint32_t j = r0 + (uint32_t)lane;
        if (j < n) {
            uint32_t p = (bot - n + j) & (SCAP - 1);
            if (SINGLE) {
                uint2 v = deep_s_of(a, wg)[dtop - n + j];
                W.sl[p] = v.x;
                W.sm[p] = (uint16_t)v.y;
            } else {
                uint4 v = deep_m_of(a, wg)[dtop - n + j];
                W.ml[p] = v.x;
                W.mr[p] = v.y;
                W.mm[p] = (uint16_t)v.z;
            }
        }
    }
    dtop -= n;
    bot -= n;
    __syncwarp();
}

// Make room for `add` more nodes on a stack: its oldest nodes go to the
// warp's overflow stack, or to the shared spill ring when that is full.
template <int SCAP, bool SINGLE>
__device__ __forceinline__ void make_room(WarpSmem<SCAP> &W, const PersistArgs &a, int wg, uint32_t &dtop,
                                          uint32_t &bot, uint32_t top, uint32_t add, uint32_t s_read,
                                          uint32_t s_info, int lane, uint32_t &c_spills, uint32_t &c_deep)
{
    if ((top - bot) + add > (uint32_t)SCAP) {
        uint32_t nsp = (top - bot) + add - SCAP + SCAP / 4;
        nsp = min((nsp + 31) & ~31u, top - bot);
        if (dtop + nsp <= DEEP_CAP) {
            deep_push<SCAP, SINGLE>(W, a, wg, dtop, bot, nsp, lane);
            c_deep += nsp;
        } else {
            spill_bottom<SCAP, SINGLE>(W, a, bot, nsp, s_read, s_info, lane, c_spills, false);
        }
    }
}

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Ask L2 for the occurrence blocks of the nodes the next round will take
// (the top 32 of each stack), so that round's dependent loads find them
// there instead of in HBM.  No register waits on a prefetch.
template <int SCAP>
__device__ __forceinline__ void prefetch_next(const WarpSmem<SCAP> &W, const IndexView &ix, uint32_t mbot,
                                              uint32_t mtop, uint32_t sbot, uint32_t stop, int lane)
{
    if ((uint32_t)lane < mtop - mbot) {
        uint32_t p = (mtop - 1 - (uint32_t)lane) & (SCAP - 1);
        uint32_t bl = W.ml[p] / OCC_ROWS, br = W.mr[p] / OCC_ROWS;
        prefetch_l2(ix.occ + (size_t)bl * 2);
        if (br != bl) prefetch_l2(ix.occ + (size_t)br * 2);
    }
    if ((uint32_t)lane < stop - sbot) {
        uint32_t p = (stop - 1 - (uint32_t)lane) & (SCAP - 1);
        prefetch_l2(ix.occ + (size_t)(W.sl[p] / OCC_ROWS) * 2);
    }
}

// Write at most one leaf interval per lane with one warp-wide atomic.
__device__ __forceinline__ void emit_one(const PersistArgs &a, bool leaf, uint32_t rid, uint32_t d, uint32_t minus,
                                         uint32_t l, uint32_t r, int lane, unsigned lt)
{
    unsigned bl = __ballot_sync(FULL, leaf);
    if (!bl) return;
    uint32_t at0 = 0;
    if (lane == 0) at0 = atomicAdd(&a.ctl->iv_count, (unsigned)__popc(bl));
    at0 = __shfl_sync(FULL, at0, 0);
    if (leaf) {
        atomicAdd(&a.iv_cnt[rid], 1u);
        uint32_t q = at0 + __popc(bl & lt);
        if (q < a.ctl->iv_cap) {
            Interval x;
            x.read = rid; x.meta = d | (minus << 2); x.l = l; x.r = r;
            a.iv[q] = x;
        } else {
            atomicOr(&a.ctl->error, ERR_IV_OVERFLOW);
        }
    }
}

// Copy the packed words of `nnew` newly admitted slots into their pattern
// rows (word-reversed for the minus strand), four lanes per slot: lane g of a
// quad loads the 16-byte-aligned chunks g and g + 4 of the slot's read.
// woff / info are read from the slot's own lane by shuffle.
template <int SCAP>
__device__ __forceinline__ void stage_patterns(WarpSmem<SCAP> &W, const uint32_t *words, const uint32_t *words_end,
                                               uint64_t woff, uint32_t info, uint32_t nnew, int lane)
{
    const uint32_t quad = (uint32_t)lane >> 2, g = (uint32_t)lane & 3u;
    for (uint32_t base = 0; base < nnew; base += 8) {
        const uint32_t r = base + quad;
        const int src = r < nnew ? W.rank_lane[r] : 0;
        const uint64_t off = __shfl_sync(FULL, woff, src);
        const uint32_t inf = __shfl_sync(FULL, info, src);
        if (r >= nnew) continue;
        const uint32_t m = inf & 511u, minus = (inf >> 11) & 1u, Wn = (m + 15) >> 4;
        const uint32_t *p0 = words + off, *pend = p0 + Wn;
        const uint32_t *a0 = (const uint32_t *)((uintptr_t)p0 & ~(uintptr_t)15);
        uint32_t *row = W.pat[src];
#pragma unroll
        for (uint32_t c = g; c < 8; c += 4) {
            const uint32_t *cp = a0 + 4 * c;
            if (cp >= pend) break;
            uint32_t v[4];
            if (cp >= words && cp + 4 <= words_end) {
                uint4 x = __ldg((const uint4 *)cp);
                v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++) v[e] = (cp + e >= p0 && cp + e < pend) ? __ldg(cp + e) : 0u;
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t *wp = cp + e;
                if (wp >= p0 && wp < pend) {
                    const uint32_t t = (uint32_t)(wp - p0);
                    row[minus ? Wn - 1 - t : t] = v[e];
                }
            }
        }
    }
}

// Push at most one node per lane onto the stack its size selects.  Callers
// guarantee room: admission runs with fewer than 64 nodes held and seed
// rounds with fewer than 32 on each stack, so 32 more always fit.
template <int SCAP>
__device__ __forceinline__ void push_one(WarpSmem<SCAP> &W, bool push, uint32_t l, uint32_t r, uint16_t meta,
                                         uint32_t &mtop, uint32_t &stop, unsigned lt)
{
    bool single = r - l == 1;
    unsigned bm = __ballot_sync(FULL, push && !single), bs = __ballot_sync(FULL, push && single);
    if (push && !single) {
        uint32_t p = (mtop + __popc(bm & lt)) & (SCAP - 1);
        W.ml[p] = l; W.mr[p] = r; W.mm[p] = meta;
    }
    if (push && single) {
        uint32_t p = (stop + __popc(bs & lt)) & (SCAP - 1);
        W.sl[p] = l; W.sm[p] = meta;
    }
    mtop += __popc(bm);
    stop += __popc(bs);
}

template <int SCAP, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) k_persistent(PersistArgs a)
{
    extern __shared__ uint4 smem_raw[];
    WarpSmem<SCAP> *all = reinterpret_cast<WarpSmem<SCAP> *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<SCAP> &W = all[warp];
    const IndexView &ix = a.ix;
    SearchCtl *ctl = a.ctl;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t spill_cap = ctl->spill_cap;

    W.live[lane] = 0;
    // task slot `lane`: read id, info = m | k << 9 | minus << 11 | qe << 12,
    // window code, next and end seed variant
    uint32_t s_read = 0, s_info = 0, s_code = 0, s_vnext = 0, s_vend = 0;
    uint64_t s_woff = 0;          // admission only: word offset of the slot's read
    bool s_used = false;
    const uint32_t *words_end = a.rd.words + a.rd.word_off[a.rd.n];   // end of the batch's packed words
    uint32_t mbot = 0, mtop = 0, sbot = 0, stop = 0;
    uint32_t dmt = 0, dst = 0;    // entries in the warp's overflow stacks (multi-row, single-row)
    const int wg = (int)blockIdx.x * WARPS + warp;
    bool busy = false;
    uint32_t idle_rounds = 0;   // consecutive rounds without work; the sleep grows with it
    uint32_t c_seeds = 0, c_nodes = 0, c_blocks = 0, c_spills = 0;   // per lane
    unsigned long long c_idle_ns = 0;                                 // warp-uniform
    uint32_t c_deep = 0;                                              // warp-uniform
    uint32_t c_km = 0, c_ks = 0, c_kq = 0;                           // rounds by kind (warp-uniform)
    __syncwarp();

    for (uint32_t iter = 0;; iter++) {
        if ((iter & 15) == 0 && vload(&ctl->error) != 0) break;

        if (s_used && W.live[lane] == 0 && s_vnext >= s_vend) s_used = false;
        unsigned used = __ballot_sync(FULL, s_used);
        uint32_t mc = mtop - mbot, sc = stop - sbot;
        // refill a low stack from the warp's overflow stack (mc, sc < 32: room for 64)
        if (mc < 32 && dmt > 0) {
            uint32_t k = min(dmt, 64u);
            deep_pop<SCAP, false>(W, a, wg, dmt, mbot, k, lane);
            mc += k;
        }
        if (sc < 32 && dst > 0) {
            uint32_t k = min(dst, 64u);
            deep_pop<SCAP, true>(W, a, wg, dst, sbot, k, lane);
            sc += k;
        }
        uint32_t cnt = mc + sc;
        uint32_t avail = s_used ? s_vend - s_vnext : 0u;
        uint32_t seeds_total = __reduce_add_sync(FULL, avail);
        unsigned freem = ~used;

        // ---- admission of new work into free slots (not while the overflow stacks hold
        // work; a warp that still has work tries only every fourth iteration and
        // once several slots are free or its work runs low, so the queue counters
        // are not hammered and each admission fills several slots)
        if (freem != 0 && cnt + seeds_total + dmt + dst < ADMIT_LOW &&
            (cnt + seeds_total == 0 ||
             ((iter & 3) == 0 && (__popc(freem) >= a.admit_min_free || cnt + seeds_total < ADMIT_LOW / 4)))) {
            bool idle = (cnt + seeds_total == 0) && used == 0;
            // an idle warp first peeks without atomics
            if (idle && !busy) {
                int pw = 0;
                if (lane == 0) {
                    uint32_t h = vload(&ctl->spill_head);
                    uint32_t R = vload(&ctl->spill_reserve);
                    pw = (R != h) || (vload64(&ctl->task_head) < a.ntasks);
                    if (!pw) {
                        // nothing queued: finished once no warp holds work
                        if (vload((const unsigned *)&ctl->busy) == 0) {
                            __threadfence();
                            h = vload(&ctl->spill_head);
                            R = vload(&ctl->spill_reserve);
                            if (R == h && vload64(&ctl->task_head) >= a.ntasks) pw = -1;
                        }
                    }
                }
                pw = __shfl_sync(FULL, pw, 0);
                if (pw < 0) break;
                if (pw == 0) {
                    if (++idle_rounds > a.idle_limit) {
                        if (lane == 0) atomicOr(&ctl->error, ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(256u << min(idle_rounds, 5u));
                    c_idle_ns += 256u << min(idle_rounds, 5u);
                    continue;
                }
            }
            uint32_t want = __popc(freem);
            uint32_t h0 = 0, take = 0, got = 0;
            unsigned long long t0 = 0;
            if (lane == 0) {
                if (!busy) atomicAdd(&ctl->busy, 1);
                // a plain read first: the ring is usually empty, and then no atomic is spent
                bool ring = vload(&ctl->spill_reserve) != vload(&ctl->spill_head);
                for (int tries = 0; ring && tries < 4; tries++) {   // contended: try again later
                    // claims up to R, both counters only grow: R - h <= 0 is a stale read
                    uint32_t h = atomicAdd(&ctl->spill_head, 0u);
                    uint32_t R = atomicAdd(&ctl->spill_reserve, 0u);
                    if ((int)(R - h) <= 0) break;
                    uint32_t n = min(R - h, want);
                    if (atomicCAS(&ctl->spill_head, h, h + n) == h) { h0 = h; take = n; break; }
                }
                if (take < want && vload64(&ctl->task_head) < a.ntasks) {
                    t0 = atomicAdd(&ctl->task_head, (unsigned long long)(want - take));
                    if (t0 < a.ntasks) got = (uint32_t)min((unsigned long long)(want - take), a.ntasks - t0);
                }
            }
            busy = true;
            h0 = __shfl_sync(FULL, h0, 0);
            take = __shfl_sync(FULL, take, 0);
            got = __shfl_sync(FULL, got, 0);
            t0 = __shfl_sync(FULL, t0, 0);
            if (take + got > 0) {
                uint32_t j = __popc(freem & lt);
                bool mine = ((freem >> lane) & 1u) && j < take + got;
                bool is_node = false;
                uint32_t nd_l = 0, nd_r = 0, nd_i = 0, nd_d = 0;
                if (mine) {
                    uint32_t rid, minus, vb, ve;
                    if (j < take) {
                        const uint32_t pos = h0 + j, slot_i = pos & (spill_cap - 1);
                        WorkItem *it = a.spill + slot_i;
                        volatile uint32_t *sq = a.seq + slot_i;
                        uint32_t spin = 0;
                        bool ready = true;
                        while (*sq != pos + 1) {          // written by its producer?
                            if (++spin > a.spin_limit) { atomicOr(&ctl->error, ERR_TIMEOUT); ready = false; break; }
                            __nanosleep(128);
                        }
                        if (spin) atomicAdd(&ctl->wait_queue_ns, 128ull * spin);
                        __threadfence();
                        rid = *(volatile uint32_t *)&it->read;
                        uint32_t meta = *(volatile uint32_t *)&it->meta;
                        uint32_t xa = *(volatile uint32_t *)&it->a, xb = *(volatile uint32_t *)&it->b;
                        __threadfence();
                        if (ready) *sq = pos + spill_cap;   // the slot is free for the next lap
                        else { rid = 0; meta = WI_NODE; xa = xb = 0; }   // timed out
                        minus = (meta & WI_MINUS) ? 1u : 0u;
                        if (meta & WI_NODE) {
                            is_node = xa < xb;
                            nd_l = xa; nd_r = xb;
                            nd_i = (meta >> 8) & 511u;
                            nd_d = meta & 3u;
                            vb = ve = 0;
                        } else {
                            vb = xa; ve = xb;
                        }
                    } else {
                        unsigned long long t = t0 + (j - take);
                        rid = a.read_list ? a.read_list[t >> 1] : (uint32_t)(t >> 1);
                        minus = (uint32_t)(t & 1);
                        vb = 0; ve = 0xffffffffu;
                    }
                    uint32_t m = a.rd.len[rid], k = a.rd.k[rid];
                    uint32_t qe = min(m, ix.q);
                    unsigned long long lbv = a.lb ? a.lb[2ull * rid + minus] : LB_NONE;
                    // the seed window may hold only the mismatches the rest cannot need
                    int keff = lb_budget(lbv, k, m - qe);
                    s_read = rid;
                    s_info = m | (k << 9) | (minus << 11) | (qe << 12) | ((uint32_t)max(keff, 0) << 16);
                    s_vnext = vb;
                    s_vend = keff < 0 ? 0u : min(ve, n_variants(qe, (uint32_t)keff));
                    s_used = true;
                    W.live[lane] = is_node ? 1 : 0;
                    W.lb[lane] = lbv;
                }
                // stage the new tasks' patterns cooperatively: four lanes per
                // new slot, eight slots per pass, each lane moving 16-byte
                // vector loads of the slot's packed words (consecutive lanes on
                // consecutive chunks, so a read costs its two or three sectors
                // once).  Chunks are aligned down to 16 bytes; the bytes of
                // neighbouring reads they cover are dropped, and a chunk that
                // would reach outside the batch's words array (its first or
                // last read only) is read word by word.  A minus-strand pattern
                // is stored word-reversed and then turned into the reverse
                // complement in place by the slot's own lane (word j needs
                // stored words j and j + 1, and only word j is overwritten).
                if (mine) {
                    W.rank_lane[j] = (uint8_t)lane;
                    s_woff = a.rd.word_off[s_read];
                }
                __syncwarp();
                stage_patterns<SCAP>(W, a.rd.words, words_end, s_woff, s_info, take + got, lane);
                __syncwarp();
                if (mine && ((s_info >> 11) & 1u)) {
                    const uint32_t m = s_info & 511u, Wn = (m + 15) >> 4;
                    uint32_t *row = W.pat[lane];
                    for (uint32_t q = 0; q < Wn; q++) {
                        uint32_t hi = row[q], lo = q + 1 < Wn ? row[q + 1] : 0u;
                        row[q] = rc_word(hi, lo, m);
                    }
                }
                __syncwarp();
                if (mine) s_code = window_code(W.pat[lane], s_info & 511u, (s_info >> 12) & 15u);
                push_one<SCAP>(W, is_node, nd_l, nd_r, node_meta((uint32_t)lane, nd_i, nd_d), mtop, stop, lt);
                __syncwarp();
                idle_rounds = 0;
                continue;
            }
            if (idle) {
                // claimed nothing and hold nothing: leave the busy set
                int done = 0;
                if (lane == 0) {
                    __threadfence();
                    int old = atomicSub(&ctl->busy, 1);
                    if (old == 1) {
                        uint32_t h = atomicAdd(&ctl->spill_head, 0u);
                        uint32_t R = atomicAdd(&ctl->spill_reserve, 0u);
                        if (R == h && vload64(&ctl->task_head) >= a.ntasks) done = 1;
                    }
                }
                busy = false;
                if (__shfl_sync(FULL, done, 0)) break;
                if (++idle_rounds > a.idle_limit) {
                    if (lane == 0) atomicOr(&ctl->error, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(256u << min(idle_rounds, 5u));
                c_idle_ns += 256u << min(idle_rounds, 5u);
                continue;
            }
        }
        if (cnt + seeds_total == 0) {
            // slots still held but no work: cannot happen while the per-slot
            // node counts are right; bounded so a bug cannot spin forever
            if (++idle_rounds > a.idle_limit) {
                if (lane == 0) atomicOr(&ctl->error, ERR_TIMEOUT);
                break;
            }
            continue;
        }

        // ---- one round over one kind of work: multi-row nodes, single-row
        // nodes or seed lookups, so that no lane runs another kind's code
        int kind;
        if (mc >= 32) kind = 0;
        else if (sc >= 32) kind = 1;
        else if (seeds_total >= 32) kind = 2;
        else kind = (mc >= sc && mc >= seeds_total) ? 0 : (sc >= seeds_total ? 1 : 2);
        c_km += kind == 0;
        c_ks += kind == 1;
        c_kq += kind == 2;

        if (kind == 1) {
            // single-row node [l, l+1): its only possible child is c = BWT[l]
            uint32_t npop = min(sc, 32u);
            bool has = (uint32_t)lane < npop;
            uint32_t l = 0, meta = 0;
            if (has) {
                uint32_t p = (stop - 1 - lane) & (SCAP - 1);
                l = W.sl[p];
                meta = W.sm[p];
            }
            stop -= npop;
            __syncwarp();
            uint32_t slot = meta & 31u;
            uint32_t info = __shfl_sync(FULL, s_info, slot);
            uint32_t rid = __shfl_sync(FULL, s_read, slot);
            uint32_t i = (meta >> 5) & 511u, d = meta >> 14, k = (info >> 9) & 3u, minus = (info >> 11) & 1u;
            bool child = false;
            uint32_t l2 = 0, dd = 0;
            if (has) {
                c_nodes++;
                if (l != ix.dollar_row) {
                    uint32_t b = l / OCC_ROWS, o = l - b * OCC_ROWS;
                    uint4 sup = ld_nc(ix.super + b / SB_BLOCKS);
                    OccBlock blk;
                    load_block(ix, b, o + 1, blk);
                    c_blocks++;
                    uint32_t c = block_symbol(blk, o);
                    uint32_t base = pat_base(W.pat[slot], i - 1);
                    dd = d + (c != base);
                    if ((int)dd <= lb_budget(W.lb[slot], k, i - 1)) {
                        l2 = C_of(ix, c) + occ_single(ix, b, o, sup, blk, c);
                        child = true;
                    }
                }
            }
            emit_one(a, child && i == 1, rid, dd, minus, l2, l2 + 1, lane, lt);
            // a single-row round pops n nodes and pushes at most n: no room check
            bool push = child && i > 1;
            unsigned bs = __ballot_sync(FULL, push);
            if (push) {
                uint32_t p = (stop + __popc(bs & lt)) & (SCAP - 1);
                W.sl[p] = l2;
                W.sm[p] = node_meta(slot, i - 1, dd);
            }
            stop += __popc(bs);
            if (has && !push) atomicAdd(&W.live[slot], -1);
        } else if (kind == 0) {
            // multi-row node: counts of all four symbols at l and r
            uint32_t npop = min(mc, 32u);
            bool has = (uint32_t)lane < npop;
            uint32_t l = 0, r = 0, meta = 0;
            if (has) {
                uint32_t p = (mtop - 1 - lane) & (SCAP - 1);
                l = W.ml[p];
                r = W.mr[p];
                meta = W.mm[p];
            }
            mtop -= npop;
            __syncwarp();
            uint32_t slot = meta & 31u;
            uint32_t info = __shfl_sync(FULL, s_info, slot);
            uint32_t rid = __shfl_sync(FULL, s_read, slot);
            uint32_t i = (meta >> 5) & 511u, d = meta >> 14, k = (info >> 9) & 3u, minus = (info >> 11) & 1u;
            uint32_t cl[4], cr[4], cd[4];
            uint32_t valid = 0;
#pragma unroll
            for (int c = 0; c < 4; c++) cl[c] = cr[c] = cd[c] = 0;
            if (has) {
                uint32_t ol[4], orr[4];
                c_blocks += occ_pair(ix, l, r, ol, orr);
                c_nodes++;
                uint32_t base = pat_base(W.pat[slot], i - 1);
                const int kb = lb_budget(W.lb[slot], k, i - 1);   // mismatches children may hold
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    cl[c] = ix.C[c] + ol[c];
                    cr[c] = ix.C[c] + orr[c];
                    cd[c] = d + ((uint32_t)c != base);
                    if ((int)cd[c] <= kb && cl[c] < cr[c]) valid |= 1u << c;
                }
            }
            bool leafs = (i == 1);
            // leaves: up to four per lane
            uint32_t nleaf = leafs ? (uint32_t)__popc(valid) : 0u;
            if (__ballot_sync(FULL, nleaf != 0)) {
                uint32_t pre = warp_excl_scan(nleaf, lane);
                uint32_t tot = __shfl_sync(FULL, pre + nleaf, 31);
                uint32_t at0 = 0;
                if (lane == 0) at0 = atomicAdd(&ctl->iv_count, tot);
                at0 = __shfl_sync(FULL, at0, 0);
                if (nleaf) {
                    atomicAdd(&a.iv_cnt[rid], nleaf);
                    uint32_t q = at0 + pre;
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        if (valid >> c & 1u) {
                            if (q < ctl->iv_cap) {
                                Interval x;
                                x.read = rid; x.meta = cd[c] | (minus << 2); x.l = cl[c]; x.r = cr[c];
                                a.iv[q] = x;
                            } else {
                                atomicOr(&ctl->error, ERR_IV_OVERFLOW);
                            }
                            q++;
                        }
                    }
                }
            }
            // children onto the stack their size selects
            uint32_t nm = 0, ns = 0;
            if (!leafs) {
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if (valid >> c & 1u) {
                        if (cr[c] - cl[c] == 1) ns++;
                        else nm++;
                    }
            }
            uint32_t packed = nm | (ns << 8);
            uint32_t pre = warp_excl_scan(packed, lane);
            uint32_t tot = __shfl_sync(FULL, pre + packed, 31);
            uint32_t tm = tot & 0xffu, ts = tot >> 8;
            if (tm) make_room<SCAP, false>(W, a, wg, dmt, mbot, mtop, tm, s_read, s_info, lane, c_spills, c_deep);
            if (ts) make_room<SCAP, true>(W, a, wg, dst, sbot, stop, ts, s_read, s_info, lane, c_spills, c_deep);
            if (nm | ns) {
                uint32_t pm = mtop + (pre & 0xffu), ps = stop + (pre >> 8);
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    if (valid >> c & 1u) {
                        uint16_t mt = node_meta(slot, i - 1, cd[c]);
                        if (cr[c] - cl[c] == 1) {
                            uint32_t q = ps++ & (SCAP - 1);
                            W.sl[q] = cl[c];
                            W.sm[q] = mt;
                        } else {
                            uint32_t q = pm++ & (SCAP - 1);
                            W.ml[q] = cl[c];
                            W.mr[q] = cr[c];
                            W.mm[q] = mt;
                        }
                    }
                }
            }
            mtop += tm;
            stop += ts;
            int delta = (int)(nm + ns) - 1;
            if (has && delta) atomicAdd(&W.live[slot], delta);
        } else {
            // seed lookups, all from one slot
            int s = __ffs(__ballot_sync(FULL, avail > 0)) - 1;
            uint32_t av = __shfl_sync(FULL, avail, s), vn = __shfl_sync(FULL, s_vnext, s);
            uint32_t info = __shfl_sync(FULL, s_info, s);
            uint32_t rid = __shfl_sync(FULL, s_read, s);
            uint32_t code = __shfl_sync(FULL, s_code, s);
            if (lane == s) s_vnext += min(av, 32u);
            bool has = (uint32_t)lane < av;
            uint32_t minus = (info >> 11) & 1u, m = info & 511u, qe = (info >> 12) & 15u;
            uint32_t l = 0, r = 0, dd = 0;
            bool child = false;
            if (has) {
                uint32_t w = __ldg(ix.variants + var_off((info >> 16) & 3u) + vn + lane);
                seed_interval(ix, code ^ (w & 0xffffffu), qe, l, r);
                c_seeds++;
                dd = w >> 24;
                child = l < r;
            }
            uint32_t i0 = m - qe;
            emit_one(a, child && i0 == 0, rid, dd, minus, l, r, lane, lt);
            bool push = child && i0 > 0;
            push_one<SCAP>(W, push, l, r, node_meta((uint32_t)s, i0, dd), mtop, stop, lt);
            unsigned bp = __ballot_sync(FULL, push);
            if (lane == 0 && bp) atomicAdd(&W.live[s], __popc(bp));
        }
        __syncwarp();
        if (a.prefetch) prefetch_next<SCAP>(W, ix, mbot, mtop, sbot, stop, lane);

        // ---- share work with idle warps near the end of the batch
        if ((iter & 31) == 31 && (mtop - mbot) + (stop - sbot) + dmt + dst > DONATE_MIN) {
            int give = 0;
            if (lane == 0) {
                uint32_t h = vload(&ctl->spill_head);
                uint32_t R = vload(&ctl->spill_reserve);
                give = R == h && vload64(&ctl->task_head) >= a.ntasks &&
                       (int)vload((const unsigned *)&ctl->busy) < a.total_warps;
            }
            if (__shfl_sync(FULL, give, 0)) {
                if (stop - sbot >= mtop - mbot)
                    spill_bottom<SCAP, true>(W, a, sbot, min(DONATE_N, stop - sbot), s_read, s_info, lane, c_spills,
                                             true);
                else
                    spill_bottom<SCAP, false>(W, a, mbot, min(DONATE_N, mtop - mbot), s_read, s_info, lane, c_spills,
                                              true);
            }
        }
    }

    // counters
    unsigned long long v;
    v = c_seeds;  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->seeds, v);
    v = c_nodes;  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->nodes, v);
    v = c_blocks; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->rank_blocks, v);
    v = c_spills; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->spills, v);
    if (lane == 0 && c_idle_ns) atomicAdd(&ctl->wait_idle_ns, c_idle_ns);
    if (lane == 0 && c_deep) atomicAdd(&ctl->deep_moves, (unsigned long long)c_deep);
    if (lane == 0) atomicAdd(&ctl->rounds, (unsigned long long)c_km + c_ks + c_kq);
    v = (unsigned long long)c_seeds + c_nodes; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->lane_ops, v);
    if (lane == 0) {
        atomicAdd(&ctl->rounds_kind[0], (unsigned long long)c_km);
        atomicAdd(&ctl->rounds_kind[1], (unsigned long long)c_ks);
        atomicAdd(&ctl->rounds_kind[2], (unsigned long long)c_kq);
    }
}


}  // namespace

// --------------------------------------------------------------------------
// Host launcher
// --------------------------------------------------------------------------

static uint32_t ring_capacity(uint64_t n);

// Persistent kernel shapes: (stack capacity, warps per CTA, min CTAs per SM).
struct PersistShape {
    void (*fn)(PersistArgs);
    int scap, warps, minb;
    size_t smem;
    int blocks_per_sm;
};

#define MICA_SHAPE(S, W, B) {k_persistent<S, W, B>, S, W, B, sizeof(WarpSmem<S>) * W, 0}
static PersistShape g_shapes[] = {
    MICA_SHAPE(256, 8, 3),
    MICA_SHAPE(256, 8, 4),
    MICA_SHAPE(256, 4, 8),
    MICA_SHAPE(128, 8, 4),
};
#undef MICA_SHAPE
constexpr int N_SHAPES = sizeof(g_shapes) / sizeof(g_shapes[0]);

static int g_num_sms = 0;
static std::mutex g_grid_mu;

static int persistent_grid(int device, int shape, int &blocks_per_sm)
{
    std::lock_guard<std::mutex> lk(g_grid_mu);
    if (g_num_sms == 0)
        MICA_CUDA_TRY(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, device));
    PersistShape &sh = g_shapes[shape];
    if (sh.blocks_per_sm == 0) {
        MICA_CUDA_TRY(cudaFuncSetAttribute(sh.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
        MICA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh.blocks_per_sm, sh.fn, sh.warps * 32,
                                                                    sh.smem));
        if (sh.blocks_per_sm < 1) sh.blocks_per_sm = 1;
    }
    blocks_per_sm = sh.blocks_per_sm;
    return 0;
}

int search_shape_count() { return N_SHAPES; }

// Device bytes the persistent search reserves for a batch of n reads (grow-
// only workspace buffers at their first-call sizes): per-read counters, the
// interval buffer (4 per read + 65,536), lower-bound words, the spill ring
// (a power of two >= max(n, 2^20) items) and the grid's per-warp overflow
// stacks, which do not depend on n.
int search_workspace_bytes(const mica_index *idx, uint64_t n, uint64_t *bytes)
{
    int shape = (idx->tuning.shape >= 0 && idx->tuning.shape < N_SHAPES) ? idx->tuning.shape : DEFAULT_SHAPE;
    int bps = 0;
    if (int rc = persistent_grid(idx->device, shape, bps)) return rc;
    uint64_t warps = (uint64_t)g_num_sms * bps * g_shapes[shape].warps;
    uint64_t iv_cap = std::min<uint64_t>(4 * n + 65536, 1ull << 30);
    uint64_t ring = ring_capacity(n);
    *bytes = sizeof(SearchCtl) + 64 + 4 * std::max<uint64_t>(n, 1) + iv_cap * sizeof(Interval) +
             16 * std::max<uint64_t>(n, 1) + ring * (sizeof(WorkItem) + 4) + warps * DEEP_CAP * 24;
    return 0;
}

int search_shape_info(int shape, int *scap, int *warps, int *minb)
{
    if (shape < 0 || shape >= N_SHAPES) return MICA_EINVAL;
    if (scap) *scap = g_shapes[shape].scap;
    if (warps) *warps = g_shapes[shape].warps;
    if (minb) *minb = g_shapes[shape].minb;
    return 0;
}

// Admission threshold (see k_persistent): 16 free slots when the occurrence
// blocks do not stay in L2 (over 96 MiB), else 8.
static int admit_min_free_for(const mica_index *idx)
{
    return idx->n_occ_blocks * 32 > (96ull << 20) ? 16 : 8;
}

static void set_wait_limits(const mica_index *idx, PersistArgs &pa)
{
    pa.idle_limit = idx->idle_limit ? idx->idle_limit : IDLE_LIMIT;
    pa.spin_limit = idx->spin_limit ? idx->spin_limit : SPIN_LIMIT;
}

// Spill ring capacity for a batch of n reads: a power of two >= max(n, 2^20).
static uint32_t ring_capacity(uint64_t n)
{
    uint64_t c = 1u << 20;
    while (c < n && c < (1ull << 28)) c <<= 1;
    return (uint32_t)c;
}

// Per-warp overflow stacks for a grid of `total_warps` warps: DEEP_CAP multi-row
// entries (16 B) then DEEP_CAP single-row entries (8 B) per warp.
static int reserve_deep(Workspace &w, int total_warps)
{
    return dev_reserve(w.deep, (size_t)total_warps * DEEP_CAP * 24);
}

static void deep_ptrs(const Workspace &w, int total_warps, uint4 *&dm, uint2 *&ds)
{
    dm = (uint4 *)w.deep.p;
    ds = (uint2 *)((char *)w.deep.p + (size_t)total_warps * DEEP_CAP * 16);
}

// Fresh sequence words for the spill ring (w.spill_seq, spill_cap entries).
static int launch_ring_init(Workspace &w, cudaStream_t s)
{
    unsigned g = (unsigned)std::min<uint64_t>((w.spill_cap + 255) / 256, 152ull * 8);
    k_ring_init<<<g, 256, 0, s>>>((uint32_t *)w.spill_seq.p, w.spill_cap);
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

// The lower-bound pass over all 2n tasks into w.lb (reserved by the caller).
static int launch_lower_bounds(const mica_index *idx, Workspace &w, const ReadsView &rd, SearchCtl *d_ctl,
                               cudaStream_t s)
{
    if (rd.n == 0) return 0;
    unsigned g = (unsigned)std::min<uint64_t>((2 * rd.n + 255) / 256, 152ull * 64);
    k_lower_bounds<<<g, 256, 0, s>>>(idx->view, rd, (unsigned long long *)w.lb.p, d_ctl);
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

// Parity probe: the lower-bound words of all 2n tasks into d_out.
int debug_lower_bounds(const mica_index *idx, Workspace &w, const ReadsView &rd, unsigned long long *d_out,
                       cudaStream_t s)
{
    if (!idx->has_rev) return MICA_EINVAL;
    int rc;
    if ((rc = dev_reserve(w.ctl, sizeof(SearchCtl) + 64))) return rc;
    MICA_CUDA_TRY(cudaMemsetAsync(w.ctl.p, 0, sizeof(SearchCtl), s));
    if (rd.n) {
        unsigned g = (unsigned)std::min<uint64_t>((2 * rd.n + 255) / 256, 152ull * 64);
        k_lower_bounds<<<g, 256, 0, s>>>(idx->view, rd, d_out, (SearchCtl *)w.ctl.p);
        MICA_CUDA_TRY(cudaGetLastError());
    }
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}

// Reserve the search buffers for n reads and prepare the persistent launch;
// fills the control-block template (to be copied to the device) and the grid.
int prepare_persistent(const mica_index *idx, Workspace &w, uint64_t n, int shape_in, SearchCtl &tmpl,
                       int &grid, int &shape)
{
    int rc;
    if ((rc = dev_reserve(w.ctl, sizeof(SearchCtl) + 64))) return rc;
    if ((rc = dev_reserve(w.iv_cnt, std::max<uint64_t>(n, 1) * 4))) return rc;
    // room for 4 leaf intervals per read, kept when a smaller batch follows
    w.iv_cap = (uint32_t)std::max<uint64_t>(w.iv_cap, std::min<uint64_t>(4 * n + 65536, 1ull << 30));
    if (w.spill_cap == 0) w.spill_cap = ring_capacity(n);
    if ((rc = dev_reserve(w.iv, (size_t)w.iv_cap * sizeof(Interval)))) return rc;
    if ((rc = dev_reserve(w.spill, (size_t)w.spill_cap * sizeof(WorkItem)))) return rc;
    if ((rc = dev_reserve(w.lb, std::max<uint64_t>(2 * n, 1) * 8))) return rc;
    if ((rc = dev_reserve(w.spill_seq, (size_t)w.spill_cap * 4))) return rc;
    shape = (shape_in >= 0 && shape_in < N_SHAPES) ? shape_in : DEFAULT_SHAPE;
    int bps = 0;
    if ((rc = persistent_grid(idx->device, shape, bps))) return rc;
    grid = g_num_sms * bps;
    if ((rc = reserve_deep(w, grid * g_shapes[shape].warps))) return rc;
    tmpl = SearchCtl{};
    tmpl.ntasks = 2 * n;
    tmpl.spill_cap = w.spill_cap;
    tmpl.iv_cap = w.iv_cap;
    return 0;
}

// Enqueue one persistent search (control-block reset from the pinned
// template, zeroed per-read counters, the kernel between timing events);
// no host reads, so it can be captured in a CUDA graph.
int enqueue_persistent(const mica_index *idx, Workspace &w, const ReadsView &rd, int shape, int grid,
                       const SearchCtl *pinned_tmpl, bool prune, bool prefetch, cudaStream_t s,
                       uint64_t &launches)
{
    SearchCtl *d_ctl = (SearchCtl *)w.ctl.p;
    const PersistShape &sh = g_shapes[shape];
    MICA_CUDA_TRY(cudaMemcpyAsync(d_ctl, pinned_tmpl, sizeof(SearchCtl), cudaMemcpyHostToDevice, s));
    MICA_CUDA_TRY(cudaMemsetAsync(w.iv_cnt.p, 0, std::max<uint64_t>(rd.n, 1) * 4, s));
    PersistArgs pa;
    pa.ix = idx->view; pa.rd = rd; pa.read_list = nullptr; pa.ntasks = 2 * rd.n;
    pa.ctl = d_ctl; pa.iv = (Interval *)w.iv.p; pa.iv_cnt = (uint32_t *)w.iv_cnt.p;
    pa.spill = (WorkItem *)w.spill.p;
    pa.total_warps = grid * sh.warps;
    pa.lb = prune ? (const unsigned long long *)w.lb.p : nullptr;
    pa.seq = (uint32_t *)w.spill_seq.p;
    pa.prefetch = prefetch;
    pa.admit_min_free = admit_min_free_for(idx);
    deep_ptrs(w, pa.total_warps, pa.deep_m, pa.deep_s);
    set_wait_limits(idx, pa);
    if (rd.n) {
        if (int rc = launch_ring_init(w, s)) return rc;
        launches++;
    }
    MICA_CUDA_TRY(record_event(w.kev[0], s));
    if (prune && rd.n) {
        if (int rc = launch_lower_bounds(idx, w, rd, d_ctl, s)) return rc;
        launches++;
    }
    if (rd.n) { sh.fn<<<grid, sh.warps * 32, sh.smem, s>>>(pa); launches++; }
    MICA_CUDA_TRY(cudaGetLastError());
    MICA_CUDA_TRY(record_event(w.kev[1], s));
    return 0;
}

int run_search(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
               const SearchConfig &cfg, cudaStream_t s)
{
    uint64_t n = rd.n;
    int rc;
    if ((rc = dev_reserve(w.ctl, sizeof(SearchCtl) + 64))) return rc;
    if ((rc = dev_reserve(w.iv_cnt, std::max<uint64_t>(n, 1) * 4))) return rc;
    // room for 4 leaf intervals per read, kept when a smaller batch follows
    w.iv_cap = (uint32_t)std::max<uint64_t>(w.iv_cap, std::min<uint64_t>(4 * n + 65536, 1ull << 30));
    if (w.spill_cap == 0) w.spill_cap = ring_capacity(n);
    SearchCtl *d_ctl = (SearchCtl *)w.ctl.p;
    int shape = (cfg.shape >= 0 && cfg.shape < N_SHAPES) ? cfg.shape : DEFAULT_SHAPE;
    if (cfg.prune && (rc = dev_reserve(w.lb, std::max<uint64_t>(2 * n, 1) * 8))) return rc;
    const unsigned long long *d_lb = cfg.prune ? (const unsigned long long *)w.lb.p : nullptr;
    for (int attempt = 0; attempt < 8; attempt++) {
        if ((rc = dev_reserve(w.iv, (size_t)w.iv_cap * sizeof(Interval)))) return rc;
        if ((rc = dev_reserve(w.spill, (size_t)w.spill_cap * sizeof(WorkItem)))) return rc;
        SearchCtl h{};
        h.ntasks = 2 * n;
        h.spill_cap = w.spill_cap;
        h.iv_cap = w.iv_cap;
        MICA_CUDA_TRY(cudaMemcpyAsync(d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s));
        MICA_CUDA_TRY(cudaMemsetAsync(w.iv_cnt.p, 0, std::max<uint64_t>(n, 1) * 4, s));
        if (n > 0) {
            if (cfg.kernel == MICA_KERNEL_PERSISTENT) {
                int bps = 0;
                if ((rc = persistent_grid(idx->device, shape, bps))) return rc;
                const PersistShape &sh = g_shapes[shape];
                PersistArgs pa;
                pa.ix = idx->view; pa.rd = rd; pa.read_list = nullptr; pa.ntasks = 2 * n;
                pa.ctl = d_ctl; pa.iv = (Interval *)w.iv.p; pa.iv_cnt = (uint32_t *)w.iv_cnt.p;
                pa.spill = (WorkItem *)w.spill.p;
                int grid = g_num_sms * bps;
                pa.total_warps = grid * sh.warps;
                if ((rc = reserve_deep(w, pa.total_warps))) return rc;
                deep_ptrs(w, pa.total_warps, pa.deep_m, pa.deep_s);
                pa.prefetch = cfg.prefetch;
                pa.admit_min_free = admit_min_free_for(idx);
                pa.lb = d_lb;
                set_wait_limits(idx, pa);
                if ((rc = dev_reserve(w.spill_seq, (size_t)w.spill_cap * 4))) return rc;
                pa.seq = (uint32_t *)w.spill_seq.p;
                if ((rc = launch_ring_init(w, s))) return rc;
                st.launches++;
                MICA_CUDA_TRY(record_event(w.kev[0], s));
                if (cfg.prune) {
                    if ((rc = launch_lower_bounds(idx, w, rd, d_ctl, s))) return rc;
                    st.launches++;
                }
                sh.fn<<<grid, sh.warps * 32, sh.smem, s>>>(pa);
                MICA_CUDA_TRY(cudaGetLastError());
                MICA_CUDA_TRY(record_event(w.kev[1], s));
                st.launches++;
                st.grid_ctas = (uint64_t)grid;
            } else {
                // plain: one task per thread, then drain the re-queue in rounds
                if ((rc = dev_reserve(w.spill2, (size_t)w.spill_cap * sizeof(WorkItem)))) return rc;
                PlainArgs pa;
                pa.ix = idx->view; pa.rd = rd; pa.read_list = nullptr; pa.items = nullptr;
                pa.ntasks = 2 * n; pa.ctl = d_ctl; pa.iv = (Interval *)w.iv.p;
                pa.iv_cnt = (uint32_t *)w.iv_cnt.p;
                pa.requeue = (WorkItem *)w.spill.p;
                pa.requeue_count = &d_ctl->spill_reserve;
                pa.requeue_cap = w.spill_cap;
                pa.budget = cfg.plain_budget;
                pa.lb = d_lb;
                int blk = cfg.plain_block > 0 ? cfg.plain_block : 128;
                if (cfg.kernel == MICA_KERNEL_PLAIN_BY_LENGTH) {
                    // one launch per length class, each with its own block size
                    if ((rc = dev_reserve(w.lenlist, std::max<uint64_t>(n, 1) * 4 + 64))) return rc;
                    unsigned int *cnt = (unsigned int *)((char *)w.lenlist.p + ((std::max<uint64_t>(n, 1) * 4 + 15) & ~15ull));
                    MICA_CUDA_TRY(cudaMemsetAsync(cnt, 0, 3 * LEN_CLASSES * 4, s));
                    unsigned g = (unsigned)std::min<uint64_t>((n + 255) / 256, 152 * 16);
                    k_len_count<<<g, 256, 0, s>>>(rd, cnt);
                    unsigned int hc[LEN_CLASSES], hb[LEN_CLASSES];
                    MICA_CUDA_TRY(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
                    MICA_CUDA_TRY(cudaStreamSynchronize(s));
                    unsigned int acc = 0;
                    for (uint32_t c = 0; c < LEN_CLASSES; c++) { hb[c] = acc; acc += hc[c]; }
                    MICA_CUDA_TRY(cudaMemcpyAsync(cnt + LEN_CLASSES, hb, sizeof(hb), cudaMemcpyHostToDevice, s));
                    k_len_scatter<<<g, 256, 0, s>>>(rd, cnt + LEN_CLASSES, cnt + 2 * LEN_CLASSES, (uint32_t *)w.lenlist.p);
                    st.launches += 2;
                    MICA_CUDA_TRY(record_event(w.kev[0], s));
                    if (cfg.prune) {
                        if ((rc = launch_lower_bounds(idx, w, rd, d_ctl, s))) return rc;
                        st.launches++;
                    }
                    for (uint32_t c = 0; c < LEN_CLASSES; c++) {
                        if (!hc[c]) continue;
                        int bc = cfg.plain_block_len[c] > 0 ? cfg.plain_block_len[c] : blk;
                        PlainArgs pc = pa;
                        pc.read_list = (const uint32_t *)w.lenlist.p + hb[c];
                        pc.ntasks = 2ull * hc[c];
                        k_plain<<<(unsigned)((pc.ntasks + bc - 1) / bc), bc, 0, s>>>(pc);
                        MICA_CUDA_TRY(cudaGetLastError());
                        st.launches++;
                    }
                    MICA_CUDA_TRY(record_event(w.kev[1], s));
                } else {
                    MICA_CUDA_TRY(record_event(w.kev[0], s));
                    if (cfg.prune) {
                        if ((rc = launch_lower_bounds(idx, w, rd, d_ctl, s))) return rc;
                        st.launches++;
                    }
                    k_plain<<<(unsigned)((pa.ntasks + blk - 1) / blk), blk, 0, s>>>(pa);
                    MICA_CUDA_TRY(cudaGetLastError());
                    MICA_CUDA_TRY(record_event(w.kev[1], s));
                    st.launches++;
                }
                WorkItem *bufs[2] = {(WorkItem *)w.spill.p, (WorkItem *)w.spill2.p};
                for (int round = 0; round < 64; round++) {
                    unsigned int cnt = 0, err = 0;
                    MICA_CUDA_TRY(cudaMemcpyAsync(&cnt, &d_ctl->spill_reserve, 4, cudaMemcpyDeviceToHost, s));
                    MICA_CUDA_TRY(cudaMemcpyAsync(&err, &d_ctl->error, 4, cudaMemcpyDeviceToHost, s));
                    MICA_CUDA_TRY(cudaStreamSynchronize(s));
                    if (cnt == 0 || err) break;
                    cnt = std::min(cnt, w.spill_cap);
                    pa.items = bufs[round & 1];
                    pa.requeue = bufs[(round + 1) & 1];
                    pa.ntasks = cnt;
                    pa.budget = pa.budget > (1u << 28) ? 0xffffffffu : pa.budget << 2;
                    MICA_CUDA_TRY(cudaMemsetAsync(&d_ctl->spill_reserve, 0, 4, s));
                    k_plain<<<(cnt + blk - 1) / blk, blk, 0, s>>>(pa);
                    MICA_CUDA_TRY(cudaGetLastError());
                    MICA_CUDA_TRY(record_event(w.kev[1], s));
                    st.launches++;
                }
            }
        }
        SearchCtl out;
        MICA_CUDA_TRY(cudaMemcpyAsync(&out, d_ctl, sizeof(out), cudaMemcpyDeviceToHost, s));
        MICA_CUDA_TRY(cudaStreamSynchronize(s));
        if (out.error & ERR_TIMEOUT) return MICA_ETIMEOUT;
        if (out.error & (ERR_IV_OVERFLOW | ERR_SPILL_OVERFLOW)) {
            st.retries++;
            char msg[256];
            snprintf(msg, sizeof(msg),
                     "internal capacity retry did not converge (last error bits 0x%x, %u intervals for %u, "
                     "%llu spills, ring %u)", out.error, out.iv_count, w.iv_cap, out.spills, w.spill_cap);
            set_last_internal(msg);
            if (out.error & ERR_IV_OVERFLOW)
                w.iv_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(2ull * out.iv_count, 2ull * w.iv_cap), 0xfffffff0ull);
            if (out.error & ERR_SPILL_OVERFLOW)
                w.spill_cap = (uint32_t)std::min<uint64_t>(4ull * w.spill_cap, 1ull << 30);
            continue;
        }
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
        return 0;
    }
    return MICA_EINTERNAL;
}

// The persistent search of the reads d_list[0, n_list) of a batch (both
// strands of each), appending to the interval buffer after iv_base leaves
// already there (their per-read counts must be 0 for the listed reads).  Used
// for the reads the bidirectional search gave up on.  Returns
// BIDIR_FALLBACK when a buffer overflows (the caller then searches the whole
// batch with the persistent kernel).
int run_search_list(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd, const uint32_t *d_list,
                    uint32_t n_list, uint32_t iv_base, bool prune, cudaStream_t s)
{
    int rc;
    if (w.spill_cap == 0) w.spill_cap = ring_capacity(rd.n);
    if ((rc = dev_reserve(w.spill, (size_t)w.spill_cap * sizeof(WorkItem))) ||
        (rc = dev_reserve(w.spill_seq, (size_t)w.spill_cap * 4)))
        return rc;
    if (prune && (rc = dev_reserve(w.lb, std::max<uint64_t>(2 * rd.n, 1) * 8))) return rc;
    const int shape = (idx->tuning.shape >= 0 && idx->tuning.shape < N_SHAPES) ? idx->tuning.shape : DEFAULT_SHAPE;
    int bps = 0;
    if ((rc = persistent_grid(idx->device, shape, bps))) return rc;
    const PersistShape &sh = g_shapes[shape];
    const int grid = g_num_sms * bps;
    if ((rc = reserve_deep(w, grid * sh.warps))) return rc;
    SearchCtl *d_ctl = (SearchCtl *)w.ctl.p;
    SearchCtl h{};
    h.ntasks = 2ull * n_list;
    h.spill_cap = w.spill_cap;
    h.iv_cap = w.iv_cap;
    h.iv_count = iv_base;
    MICA_CUDA_TRY(cudaMemcpyAsync(d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    if (prune) {
        unsigned g = (unsigned)std::min<uint64_t>((2ull * n_list + 255) / 256, 152ull * 64);
        k_lower_bounds<<<g, 256, 0, s>>>(idx->view, rd, (unsigned long long *)w.lb.p, d_ctl, d_list, n_list);
        st.launches++;
    }
    if ((rc = launch_ring_init(w, s))) return rc;
    st.launches++;
    PersistArgs pa;
    pa.ix = idx->view; pa.rd = rd; pa.read_list = d_list; pa.ntasks = 2ull * n_list;
    pa.ctl = d_ctl; pa.iv = (Interval *)w.iv.p; pa.iv_cnt = (uint32_t *)w.iv_cnt.p;
    pa.spill = (WorkItem *)w.spill.p;
    pa.seq = (uint32_t *)w.spill_seq.p;
    pa.total_warps = grid * sh.warps;
    deep_ptrs(w, pa.total_warps, pa.deep_m, pa.deep_s);
    pa.prefetch = idx->n_occ_blocks * 32 > (96ull << 20);
    pa.admit_min_free = admit_min_free_for(idx);
    pa.lb = prune ? (const unsigned long long *)w.lb.p : nullptr;
    set_wait_limits(idx, pa);
    sh.fn<<<grid, sh.warps * 32, sh.smem, s>>>(pa);
    MICA_CUDA_TRY(cudaGetLastError());
    st.launches++;
    SearchCtl out;
    MICA_CUDA_TRY(cudaMemcpyAsync(&out, d_ctl, sizeof(out), cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    if (out.error & ERR_TIMEOUT) return MICA_ETIMEOUT;
    if (out.error) return BIDIR_FALLBACK;
    st.seeds += out.seeds;
    st.nodes += out.nodes;
    st.rank_blocks += out.rank_blocks;
    st.intervals = out.iv_count;
    st.spills += out.spills;
    st.lb_steps += out.lb_steps;
    return 0;
}

// Best-stratum search by iterative deepening (persistent kernel): pass j =
// 0, 1, ... searches, with budget min(k, j), only the reads that found
// nothing at a smaller budget; a read's first pass with hits finds exactly
// its best stratum (every hit of that pass has d = j), so the result equals
// the exhaustive search filtered to the best stratum, with less work.  The
// intervals of all passes accumulate in one buffer.  Returns
// STRATUM_FALLBACK when a pass overflows a buffer: the caller then runs the
// exhaustive search with the stratum filter.
int run_search_stratum(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
                       const SearchConfig &cfg, cudaStream_t s)
{
    const uint64_t n = rd.n;
    int rc;
    if (n == 0 || n >= (1ull << 31)) return STRATUM_FALLBACK;
    if ((rc = dev_reserve(w.ctl, sizeof(SearchCtl) + 64))) return rc;
    if ((rc = dev_reserve(w.iv_cnt, n * 4))) return rc;
    w.iv_cap = (uint32_t)std::max<uint64_t>(w.iv_cap, std::min<uint64_t>(4 * n + 65536, 1ull << 30));
    if (w.spill_cap == 0) w.spill_cap = ring_capacity(n);
    if ((rc = dev_reserve(w.iv, (size_t)w.iv_cap * sizeof(Interval))) ||
        (rc = dev_reserve(w.spill, (size_t)w.spill_cap * sizeof(WorkItem))) ||
        (rc = dev_reserve(w.spill_seq, (size_t)w.spill_cap * 4)) ||
        (rc = dev_reserve(w.lb, 2 * n * 8)) ||
        (rc = dev_reserve(w.lenlist, 2 * n * 4 + n + 64)))
        return rc;
    uint32_t *lists[2] = {(uint32_t *)w.lenlist.p, (uint32_t *)w.lenlist.p + n};
    uint8_t *k_pass = (uint8_t *)((uint32_t *)w.lenlist.p + 2 * n);
    unsigned int *d_next = (unsigned int *)((char *)w.lenlist.p + ((2 * n * 4 + n + 15) & ~15ull));
    SearchCtl *d_ctl = (SearchCtl *)w.ctl.p;
    const int shape = (cfg.shape >= 0 && cfg.shape < N_SHAPES) ? cfg.shape : DEFAULT_SHAPE;
    int bps = 0;
    if ((rc = persistent_grid(idx->device, shape, bps))) return rc;
    const PersistShape &sh = g_shapes[shape];
    const int grid = g_num_sms * bps;
    if ((rc = reserve_deep(w, grid * sh.warps))) return rc;
    const unsigned g1 = (unsigned)std::min<uint64_t>((n + 255) / 256, 152ull * 16);

    MICA_CUDA_TRY(cudaMemsetAsync(w.iv_cnt.p, 0, n * 4, s));
    k_iota<<<g1, 256, 0, s>>>(lists[0], (uint32_t)n);
    MICA_CUDA_TRY(record_event(w.kev[0], s));
    st.launches++;
    {   // pass 0's control block, then the lower bounds (their counters land in
        // it) with the reads' own budgets: valid for every smaller budget
        SearchCtl h{};
        h.ntasks = 2ull * n;
        h.spill_cap = w.spill_cap;
        h.iv_cap = w.iv_cap;
        MICA_CUDA_TRY(cudaMemcpyAsync(d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s));
        if (cfg.prune) {
            if ((rc = launch_lower_bounds(idx, w, rd, d_ctl, s))) return rc;
            st.launches++;
        }
    }
    ReadsView rp = rd;
    rp.k = k_pass;
    uint32_t n_list = (uint32_t)n, iv_base = 0, cur = 0;
    SearchCtl total{};
    for (uint32_t j = 0; j <= MICA_MAX_K && n_list > 0; j++) {
        k_stratum_pass<<<g1, 256, 0, s>>>(lists[cur], n_list, rd.k, j, k_pass);
        if (j > 0) {
            SearchCtl h{};
            h.ntasks = 2ull * n_list;
            h.spill_cap = w.spill_cap;
            h.iv_cap = w.iv_cap;
            h.iv_count = iv_base;
            MICA_CUDA_TRY(cudaMemcpyAsync(d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s));
        }
        if ((rc = launch_ring_init(w, s))) return rc;
        PersistArgs pa;
        pa.ix = idx->view; pa.rd = rp; pa.read_list = lists[cur]; pa.ntasks = 2ull * n_list;
        pa.ctl = d_ctl; pa.iv = (Interval *)w.iv.p; pa.iv_cnt = (uint32_t *)w.iv_cnt.p;
        pa.spill = (WorkItem *)w.spill.p;
        pa.seq = (uint32_t *)w.spill_seq.p;
        pa.total_warps = grid * sh.warps;
        deep_ptrs(w, pa.total_warps, pa.deep_m, pa.deep_s);
        pa.prefetch = cfg.prefetch;
        pa.admit_min_free = admit_min_free_for(idx);
        pa.lb = cfg.prune ? (const unsigned long long *)w.lb.p : nullptr;
        set_wait_limits(idx, pa);
        sh.fn<<<grid, sh.warps * 32, sh.smem, s>>>(pa);
        MICA_CUDA_TRY(cudaGetLastError());
        MICA_CUDA_TRY(cudaMemsetAsync(d_next, 0, 4, s));
        k_stratum_next<<<g1, 256, 0, s>>>(lists[cur], n_list, (const uint32_t *)w.iv_cnt.p, rd.k, j,
                                          lists[cur ^ 1], d_next);
        st.launches += 4;
        SearchCtl out;
        unsigned int nn = 0;
        MICA_CUDA_TRY(cudaMemcpyAsync(&out, d_ctl, sizeof(out), cudaMemcpyDeviceToHost, s));
        MICA_CUDA_TRY(cudaMemcpyAsync(&nn, d_next, 4, cudaMemcpyDeviceToHost, s));
        MICA_CUDA_TRY(cudaStreamSynchronize(s));
        if (out.error & ERR_TIMEOUT) return MICA_ETIMEOUT;
        if (out.error) return STRATUM_FALLBACK;
        iv_base = out.iv_count;
        total.seeds += out.seeds; total.nodes += out.nodes; total.rank_blocks += out.rank_blocks;
        total.spills += out.spills; total.rounds += out.rounds; total.lane_ops += out.lane_ops;
        for (int q = 0; q < 3; q++) total.rounds_kind[q] += out.rounds_kind[q];
        total.wait_queue_ns += out.wait_queue_ns; total.wait_idle_ns += out.wait_idle_ns;
        total.deep_moves += out.deep_moves;
        if (j == 0) { total.lb_steps = out.lb_steps; total.lb_dead = out.lb_dead; }
        n_list = nn;
        cur ^= 1;
    }
    MICA_CUDA_TRY(record_event(w.kev[1], s));
    // the post kernels read the interval count from the control block
    SearchCtl fin{};
    fin.iv_count = iv_base;
    fin.iv_cap = w.iv_cap;
    MICA_CUDA_TRY(cudaMemcpyAsync(d_ctl, &fin, sizeof(fin), cudaMemcpyHostToDevice, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    st.tasks = 2 * n;
    st.seeds = total.seeds;
    st.nodes = total.nodes;
    st.rank_blocks = total.rank_blocks;
    st.intervals = iv_base;
    st.spills = total.spills;
    st.warp_rounds = total.rounds;
    st.lane_ops = total.lane_ops;
    st.rounds_multi = total.rounds_kind[0];
    st.rounds_single = total.rounds_kind[1];
    st.rounds_seed = total.rounds_kind[2];
    st.lb_steps = total.lb_steps;
    st.lb_dead_tasks = total.lb_dead;
    st.queue_wait_ns = total.wait_queue_ns;
    st.idle_wait_ns = total.wait_idle_ns;
    st.overflow_moves = total.deep_moves;
    st.grid_ctas = (uint64_t)grid;
    return 0;
}

}  // namespace mica
