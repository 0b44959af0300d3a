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
// and d + [c != P[i-1]] <= k; nodes with i = 0 are leaf intervals.
//
// Two kernels produce the same leaf set:
//   * k_plain:      one task per thread, depth-first with a stack in local
//                   memory; a task over its node budget pushes its pending
//                   nodes (and untried seeds) to a re-queue that the next
//                   launch drains.
//   * k_persistent: one CTA per SM slot, each warp a work pool of up to 32
//                   tasks.  Every round the 32 lanes take the 32 newest nodes
//                   of the warp's shared-memory stack (topped up with seed
//                   lookups), extend them in parallel, and compact the
//                   children back with ballot/shuffle prefix sums.  Excess
//                   nodes spill to a device queue that idle warps drain.
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
};

__device__ __forceinline__ void requeue_push(const PlainArgs &a, uint32_t read, uint32_t meta,
                                             uint32_t x, uint32_t y)
{
    uint32_t at = atomicAdd(a.requeue_count, 1u);
    if (at < a.requeue_cap) {
        WorkItem it;
        it.read = read;
        it.meta = meta | WI_VALID;
        it.a = x;
        it.b = y;
        a.requeue[at] = it;
    } else {
        atomicOr(&a.ctl->error, ERR_SPILL_OVERFLOW);
    }
}

__global__ void __launch_bounds__(128) k_plain(PlainArgs a)
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
    uint32_t V = n_variants(qe, k);
    if (vend > V) vend = V;
    uint32_t pat[MAX_WORDS];
    thread_pattern(a.rd, read, minus, m, pat);
    uint32_t code = window_code(pat, m, qe);
    const uint32_t *var = ix.variants + var_off(k);

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
        // mismatching children first, the matching child last (popped next)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            uint32_t cc = (uint32_t)c;
            if (cc == base || d + 1 > k) continue;
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
        {
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

// --------------------------------------------------------------------------
// Persistent warp-pool kernel
// --------------------------------------------------------------------------

constexpr uint32_t ADMIT_LOW = 64;          // admit tasks when pending work < this
constexpr uint32_t IDLE_LIMIT = 1u << 22;    // idle rounds (>= 1 us each) before timing out
constexpr uint32_t SPIN_LIMIT = 1u << 22;    // waits for a reserved queue entry
constexpr uint32_t DONATE_MIN = 96;          // stack depth that makes a warp share work
constexpr uint32_t DONATE_N = 64;

struct PersistArgs {
    IndexView ix;
    ReadsView rd;
    const uint32_t *read_list;
    uint64_t ntasks;
    SearchCtl *ctl;
    Interval *iv;
    uint32_t *iv_cnt;
    WorkItem *spill;
    int total_warps;
};

template <int SCAP>
struct WarpSmem {
    uint32_t nl[SCAP];
    uint32_t nr[SCAP];
    uint16_t nm[SCAP];                    // slot | i << 5 | d << 14
    uint32_t pat[32][MAX_WORDS + 1];      // pattern of each task slot
    int live[32];                         // nodes of each slot in the stack
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

template <int SCAP>
__device__ __forceinline__ void spill_bottom(WarpSmem<SCAP> &sm, const PersistArgs &a, uint32_t &bot,
                                             uint32_t nsp, uint32_t s_read, uint32_t s_info, int lane,
                                             unsigned long long &c_spills)
{
    SearchCtl *ctl = a.ctl;
    uint32_t at0 = 0;
    if (lane == 0) at0 = atomicAdd(&ctl->spill_reserve, nsp);
    at0 = __shfl_sync(FULL, at0, 0);
    uint32_t cap = ctl->spill_cap;
    if (at0 + nsp > cap && lane == 0) atomicOr(&ctl->error, ERR_SPILL_OVERFLOW);
    for (uint32_t r0 = 0; r0 < nsp; r0 += 32) {
        uint32_t j = r0 + lane;
        bool act = j < nsp;
        uint32_t p = (bot + j) & (SCAP - 1);
        uint32_t l = act ? sm.nl[p] : 0u, r = act ? sm.nr[p] : 0u, mm = act ? (uint32_t)sm.nm[p] : 0u;
        uint32_t sl = mm & 31u;
        uint32_t rid = __shfl_sync(FULL, s_read, sl);
        uint32_t info = __shfl_sync(FULL, s_info, sl);
        if (act) {
            if (at0 + j < cap) {
                WorkItem *it = a.spill + at0 + j;
                it->read = rid;
                it->a = l;
                it->b = r;
                __threadfence();
                uint32_t meta = WI_VALID | WI_NODE | (((info >> 11) & 1u) ? WI_MINUS : 0u) |
                                (((mm >> 5) & 511u) << 8) | (mm >> 14);
                *(volatile uint32_t *)&it->meta = meta;
            }
            atomicAdd(&sm.live[sl], -1);
        }
    }
    bot += nsp;
    if (lane == 0) c_spills += nsp;
    __syncwarp();
}

template <int SCAP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_persistent(PersistArgs a)
{
    extern __shared__ uint4 smem_raw[];
    WarpSmem<SCAP> *all = reinterpret_cast<WarpSmem<SCAP> *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<SCAP> &sm = all[warp];
    const IndexView &ix = a.ix;
    SearchCtl *ctl = a.ctl;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t spill_cap = ctl->spill_cap;

    sm.live[lane] = 0;
    // task slot `lane`: read id, info = m | k << 9 | minus << 11 | qe << 12,
    // window code, next and end seed variant
    uint32_t s_read = 0, s_info = 0, s_code = 0, s_vnext = 0, s_vend = 0;
    bool s_used = false;
    uint32_t bot = 0, top = 0;
    bool busy = false;
    uint32_t idle_rounds = 0, backoff = 256;
    unsigned long long c_seeds = 0, c_nodes = 0, c_blocks = 0, c_spills = 0, c_rounds = 0;
    __syncwarp();

    for (uint32_t iter = 0;; iter++) {
        if ((iter & 15) == 0 && vload(&ctl->error) != 0) break;

        if (s_used && sm.live[lane] == 0 && s_vnext >= s_vend) s_used = false;
        unsigned used = __ballot_sync(FULL, s_used);
        uint32_t cnt = top - bot;
        uint32_t avail = s_used ? s_vend - s_vnext : 0u;
        uint32_t seeds_total = __reduce_add_sync(FULL, avail);
        unsigned freem = ~used;

        // ---- admission of new work into free slots
        if (freem != 0 && cnt + seeds_total < ADMIT_LOW) {
            bool idle = (cnt + seeds_total == 0) && used == 0;
            // an idle warp first peeks without atomics
            int peek_work = 1;
            if (idle && !busy) {
                int pw = 0;
                if (lane == 0) {
                    uint32_t h = vload(&ctl->spill_head);
                    uint32_t R = min(vload(&ctl->spill_reserve), spill_cap);
                    pw = (h < R) || (vload64(&ctl->task_head) < a.ntasks);
                    if (!pw) {
                        // nothing queued: finished once no warp holds work
                        if (vload((const unsigned *)&ctl->busy) == 0) {
                            __threadfence();
                            h = vload(&ctl->spill_head);
                            R = min(vload(&ctl->spill_reserve), spill_cap);
                            if (h >= R && vload64(&ctl->task_head) >= a.ntasks) pw = -1;
                        }
                    }
                }
                peek_work = __shfl_sync(FULL, pw, 0);
                if (peek_work < 0) break;
                if (peek_work == 0) {
                    if (++idle_rounds > IDLE_LIMIT) {
                        if (lane == 0) atomicOr(&ctl->error, ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(backoff);
                    backoff = min(backoff * 2, 8192u);
                    continue;
                }
            }
            uint32_t want = __popc(freem);
            uint32_t h0 = 0, take = 0, got = 0;
            unsigned long long t0 = 0;
            if (lane == 0) {
                if (!busy) atomicAdd(&ctl->busy, 1);
                for (int tries = 0; tries < 32; tries++) {
                    uint32_t h = atomicAdd(&ctl->spill_head, 0u);
                    uint32_t R = min(atomicAdd(&ctl->spill_reserve, 0u), spill_cap);
                    if (h >= R) break;
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
                uint32_t nd_l = 0, nd_r = 0, nd_m = 0;
                if (mine) {
                    uint32_t rid, minus, vb, ve;
                    if (j < take) {
                        WorkItem *it = a.spill + h0 + j;
                        volatile uint32_t *vm = &it->meta;
                        uint32_t meta = *vm;
                        uint32_t spin = 0;
                        while (!(meta & WI_VALID)) {
                            if (++spin > SPIN_LIMIT) { atomicOr(&ctl->error, ERR_TIMEOUT); break; }
                            __nanosleep(128);
                            meta = *vm;
                        }
                        __threadfence();
                        rid = *(volatile uint32_t *)&it->read;
                        uint32_t xa = *(volatile uint32_t *)&it->a, xb = *(volatile uint32_t *)&it->b;
                        *vm = 0u;
                        if (!(meta & WI_VALID)) { rid = 0; meta = WI_NODE; xa = xb = 0; }   // timed out
                        minus = (meta & WI_MINUS) ? 1u : 0u;
                        if (meta & WI_NODE) {
                            is_node = xa < xb;
                            nd_l = xa; nd_r = xb;
                            nd_m = (uint32_t)lane | (((meta >> 8) & 511u) << 5) | ((meta & 3u) << 14);
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
                    s_read = rid;
                    s_info = m | (k << 9) | (minus << 11) | (qe << 12);
                    s_vnext = vb;
                    s_vend = min(ve, n_variants(qe, k));
                    s_used = true;
                    sm.live[lane] = is_node ? 1 : 0;
                }
                // stage the new tasks' patterns: one coalesced word per lane
                unsigned newm = __ballot_sync(FULL, mine);
                unsigned todo = newm;
                while (todo) {
                    int s = __ffs(todo) - 1;
                    todo &= todo - 1;
                    uint32_t rid = __shfl_sync(FULL, s_read, s), info = __shfl_sync(FULL, s_info, s);
                    uint32_t m = info & 511u, minus = (info >> 11) & 1u;
                    uint32_t W = (m + 15) >> 4;
                    unsigned long long off = a.rd.word_off[rid];
                    uint32_t raw = (uint32_t)lane < W ? a.rd.words[off + lane] : 0u;
                    uint32_t hi = __shfl_sync(FULL, raw, (int)((W - 1 - lane) & 31u));
                    uint32_t lo = __shfl_sync(FULL, raw, (int)((W - 2 - lane) & 31u));
                    if ((uint32_t)lane + 1 >= W) lo = 0u;
                    uint32_t out = minus ? rc_word(hi, lo, m) : raw;
                    if ((uint32_t)lane < W) sm.pat[s][lane] = out;
                }
                __syncwarp();
                if (mine) s_code = window_code(sm.pat[lane], s_info & 511u, (s_info >> 12) & 15u);
                unsigned nodem = __ballot_sync(FULL, is_node);
                if (is_node) {
                    uint32_t p = (top + __popc(nodem & lt)) & (SCAP - 1);
                    sm.nl[p] = nd_l; sm.nr[p] = nd_r; sm.nm[p] = (uint16_t)nd_m;
                }
                top += __popc(nodem);
                __syncwarp();
                idle_rounds = 0;
                backoff = 256;
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
                        uint32_t R = min(atomicAdd(&ctl->spill_reserve, 0u), spill_cap);
                        if (h >= R && vload64(&ctl->task_head) >= a.ntasks) done = 1;
                    }
                }
                busy = false;
                if (__shfl_sync(FULL, done, 0)) break;
                if (++idle_rounds > IDLE_LIMIT) {
                    if (lane == 0) atomicOr(&ctl->error, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(backoff);
                backoff = min(backoff * 2, 8192u);
                continue;
            }
        }

        // ---- lanes take the newest nodes, the rest take seed variants
        uint32_t npop = min(cnt, 32u);
        bool has_node = (uint32_t)lane < npop;
        uint32_t x_l = 0, x_r = 0, x_m = 0;
        if (has_node) {
            uint32_t p = (top - 1 - lane) & (SCAP - 1);
            x_l = sm.nl[p]; x_r = sm.nr[p]; x_m = sm.nm[p];
        }
        top -= npop;
        __syncwarp();
        bool has_seed = false;
        uint32_t sslot = 0, sv = 0;
        if (seeds_total > 0 && npop < 32) {
            uint32_t lanes_free = 32 - npop;
            uint32_t excl = warp_excl_scan(avail, lane);
            uint32_t incl = excl + avail;
            uint32_t g = (uint32_t)lane - npop;
            int s = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                uint32_t e = __shfl_sync(FULL, incl, s + step - 1);
                if (e <= g) s += step;
            }
            s &= 31;
            uint32_t ex_s = __shfl_sync(FULL, excl, s), vn_s = __shfl_sync(FULL, s_vnext, s);
            has_seed = !has_node && g < seeds_total;
            sslot = (uint32_t)s;
            sv = vn_s + (g - ex_s);
            uint32_t taken = lanes_free > excl ? min(avail, lanes_free - excl) : 0u;
            s_vnext += taken;
        }

        // ---- extend
        if (lane == 0) c_rounds++;
        uint32_t slot = has_node ? (x_m & 31u) : sslot;
        uint32_t info = __shfl_sync(FULL, s_info, slot);
        uint32_t rid = __shfl_sync(FULL, s_read, slot);
        uint32_t code = __shfl_sync(FULL, s_code, slot);
        uint32_t k = (info >> 9) & 3u, minus = (info >> 11) & 1u, m = info & 511u, qe = (info >> 12) & 15u;
        uint32_t cl[4], cr[4], cd[4];
        uint32_t valid = 0, ci = 0;
        if (has_node) {
            uint32_t i = (x_m >> 5) & 511u, d = x_m >> 14;
            uint32_t ol[4], orr[4];
            c_blocks += occ_pair(ix, x_l, x_r, ol, orr);
            c_nodes++;
            uint32_t base = pat_base(sm.pat[slot], i - 1);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                uint32_t dd = d + ((uint32_t)c != base);
                cl[c] = ix.C[c] + ol[c];
                cr[c] = ix.C[c] + orr[c];
                cd[c] = dd;
                if (dd <= k && cl[c] < cr[c]) valid |= 1u << c;
            }
            ci = i - 1;
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++) { cl[c] = cr[c] = cd[c] = 0; }
            if (has_seed) {
                uint32_t w = __ldg(ix.variants + var_off(k) + sv);
                uint32_t l, r;
                seed_interval(ix, code ^ (w & 0xffffffu), qe, l, r);
                c_seeds++;
                cl[0] = l; cr[0] = r; cd[0] = w >> 24;
                if (l < r) valid = 1u;
                ci = m - qe;
            }
        }
        bool leaf = (ci == 0);

        // ---- leaves: SA intervals of matches
        uint32_t nleaf = leaf ? (uint32_t)__popc(valid) : 0u;
        uint32_t leaf_total = __reduce_add_sync(FULL, nleaf);
        if (leaf_total) {
            uint32_t pre = warp_excl_scan(nleaf, lane);
            uint32_t at0 = 0;
            if (lane == 0) at0 = atomicAdd(&ctl->iv_count, leaf_total);
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

        // ---- children back onto the stack
        uint32_t nc = leaf ? 0u : (uint32_t)__popc(valid);
        uint32_t pre = warp_excl_scan(nc, lane);
        uint32_t ch_total = __shfl_sync(FULL, pre + nc, 31);
        if ((top - bot) + ch_total > (uint32_t)SCAP) {
            uint32_t nsp = (top - bot) + ch_total - SCAP + SCAP / 4;
            nsp = min((nsp + 31) & ~31u, top - bot);
            spill_bottom(sm, a, bot, nsp, s_read, s_info, lane, c_spills);
        }
        if (nc) {
            uint32_t p = top + pre;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                if (valid >> c & 1u) {
                    uint32_t q = p & (SCAP - 1);
                    sm.nl[q] = cl[c];
                    sm.nr[q] = cr[c];
                    sm.nm[q] = (uint16_t)(slot | (ci << 5) | (cd[c] << 14));
                    p++;
                }
            }
        }
        top += ch_total;
        int delta = (int)nc - (has_node ? 1 : 0);
        if (delta && (has_node || has_seed)) atomicAdd(&sm.live[slot], delta);
        __syncwarp();

        // ---- share work with idle warps near the end of the batch
        if ((iter & 31) == 31 && top - bot > DONATE_MIN) {
            int give = 0;
            if (lane == 0) {
                uint32_t h = vload(&ctl->spill_head);
                uint32_t R = min(vload(&ctl->spill_reserve), spill_cap);
                give = h >= R && vload64(&ctl->task_head) >= a.ntasks &&
                       (int)vload((const unsigned *)&ctl->busy) < a.total_warps;
            }
            if (__shfl_sync(FULL, give, 0)) spill_bottom(sm, a, bot, DONATE_N, s_read, s_info, lane, c_spills);
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
    v = c_rounds; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->rounds, v);
    v = c_seeds + c_nodes; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->lane_ops, v);
}

}  // namespace

// --------------------------------------------------------------------------
// Host launcher
// --------------------------------------------------------------------------

constexpr int P_SCAP = 256;
constexpr int P_WARPS = 8;

static int g_num_sms = 0, g_persist_blocks = 0;
static std::mutex g_grid_mu;

static int persistent_grid(int device, int &blocks_per_sm, size_t smem)
{
    std::lock_guard<std::mutex> lk(g_grid_mu);
    if (g_num_sms == 0) {
        MICA_CUDA_TRY(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, device));
        MICA_CUDA_TRY(cudaFuncSetAttribute(k_persistent<P_SCAP, P_WARPS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        MICA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &g_persist_blocks, k_persistent<P_SCAP, P_WARPS>, P_WARPS * 32, smem));
        if (g_persist_blocks < 1) g_persist_blocks = 1;
    }
    blocks_per_sm = g_persist_blocks;
    return 0;
}

int run_search(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd,
               const SearchConfig &cfg, cudaStream_t s)
{
    uint64_t n = rd.n;
    int rc;
    if ((rc = dev_reserve(w.ctl, sizeof(SearchCtl) + 64))) return rc;
    if ((rc = dev_reserve(w.iv_cnt, std::max<uint64_t>(n, 1) * 4))) return rc;
    if (w.iv_cap == 0) w.iv_cap = (uint32_t)std::min<uint64_t>(4 * n + 65536, 1ull << 30);
    if (w.spill_cap == 0) w.spill_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(n, 1u << 20), 1ull << 28);
    SearchCtl *d_ctl = (SearchCtl *)w.ctl.p;
    const size_t smem = sizeof(WarpSmem<P_SCAP>) * P_WARPS;
    for (int attempt = 0; attempt < 8; attempt++) {
        if ((rc = dev_reserve(w.iv, (size_t)w.iv_cap * sizeof(Interval)))) return rc;
        if ((rc = dev_reserve(w.spill, (size_t)w.spill_cap * sizeof(WorkItem)))) return rc;
        if (w.spill_dirty) {
            MICA_CUDA_TRY(cudaMemsetAsync(w.spill.p, 0, (size_t)w.spill_cap * sizeof(WorkItem), s));
            w.spill_dirty = false;
        }
        SearchCtl h{};
        h.ntasks = 2 * n;
        h.spill_cap = w.spill_cap;
        h.iv_cap = w.iv_cap;
        MICA_CUDA_TRY(cudaMemcpyAsync(d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, s));
        MICA_CUDA_TRY(cudaMemsetAsync(w.iv_cnt.p, 0, std::max<uint64_t>(n, 1) * 4, s));
        if (n > 0) {
            if (cfg.kernel == MICA_KERNEL_PERSISTENT) {
                int bps = 0;
                if ((rc = persistent_grid(idx->device, bps, smem))) return rc;
                PersistArgs pa;
                pa.ix = idx->view; pa.rd = rd; pa.read_list = nullptr; pa.ntasks = 2 * n;
                pa.ctl = d_ctl; pa.iv = (Interval *)w.iv.p; pa.iv_cnt = (uint32_t *)w.iv_cnt.p;
                pa.spill = (WorkItem *)w.spill.p;
                int grid = g_num_sms * bps;
                pa.total_warps = grid * P_WARPS;
                MICA_CUDA_TRY(cudaEventRecord(w.kev[0], s));
                k_persistent<P_SCAP, P_WARPS><<<grid, P_WARPS * 32, smem, s>>>(pa);
                MICA_CUDA_TRY(cudaGetLastError());
                MICA_CUDA_TRY(cudaEventRecord(w.kev[1], s));
                st.launches++;
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
                int blk = cfg.plain_block > 0 ? cfg.plain_block : 128;
                MICA_CUDA_TRY(cudaEventRecord(w.kev[0], s));
                k_plain<<<(unsigned)((pa.ntasks + blk - 1) / blk), blk, 0, s>>>(pa);
                MICA_CUDA_TRY(cudaGetLastError());
                MICA_CUDA_TRY(cudaEventRecord(w.kev[1], s));
                st.launches++;
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
                    MICA_CUDA_TRY(cudaEventRecord(w.kev[1], s));
                    st.launches++;
                }
            }
        }
        SearchCtl out;
        MICA_CUDA_TRY(cudaMemcpyAsync(&out, d_ctl, sizeof(out), cudaMemcpyDeviceToHost, s));
        MICA_CUDA_TRY(cudaStreamSynchronize(s));
        if (out.error & ERR_TIMEOUT) { w.spill_dirty = true; return MICA_ETIMEOUT; }
        if (out.error & (ERR_IV_OVERFLOW | ERR_SPILL_OVERFLOW)) {
            st.retries++;
            if (out.error & ERR_IV_OVERFLOW)
                w.iv_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(2ull * out.iv_count, 2ull * w.iv_cap), 0xfffffff0ull);
            if (out.error & ERR_SPILL_OVERFLOW)
                w.spill_cap = (uint32_t)std::min<uint64_t>(4ull * w.spill_cap, 1ull << 30);
            w.spill_dirty = true;
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
        return 0;
    }
    return MICA_EINTERNAL;
}

}  // namespace mica
