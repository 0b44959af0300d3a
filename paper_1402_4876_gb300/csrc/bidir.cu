// Bidirectional k-mismatch search (MICA, Section 2: reads are placed with few
// mismatches by searching a BWT index; SOAP3-dp, whose index MICA uses,
// descends from 2BWT, which keeps the index of the genome and of its
// reversal so that a pattern can grow at either end).
//
// A pattern P of m bases with budget k is cut into p = k + 1 pieces of
// m / p bases (piece i = P[bnd(i), bnd(i + 1)), bnd(i) = i m / p).  Any
// placement with at most k substitutions leaves some piece exact; scheme j
// finds exactly the placements whose leftmost exact piece is piece j:
//   1. piece j exact: its last min(q, |piece|) bases from the two q-mer tables
//      (the genome's for the forward interval, the reversed genome's for the
//      interval of the reversed string), then base by base to its start;
//   2. left through pieces j - 1, ..., 0, each of which must take at least one
//      substitution;
//   3. right through pieces j + 1, ..., p - 1, freely within the budget.
// The schemes partition the placements (each has one leftmost exact piece),
// and each placement's matched string is reached on one path, so the leaf
// intervals are those of the one-directional search, and so is the result.
// Reads shorter than k + 1 bases take one scheme from the full interval,
// leftwards with any substitutions.
//
// A node holds the matched substring P[a, b) as its interval [l, l + sz) in
// the genome's index and [lr, lr + sz) in the reversed genome's (both count
// its occurrences).  Extending to the left is a backward step on the genome's
// index; the other interval keeps its start shifted by the rows whose
// preceding base sorts below the new one (and the row of an occurrence at the
// genome's start, whose preceding symbol is $).  Extending to the right is the
// same step on the reversed genome's index.
//
// The kernel is a persistent warp pool like k_persistent: each warp holds up
// to 32 tasks, one per lane slot, and two node stacks in shared memory
// (multi-row and single-row nodes); every round extends up to 32 nodes of one
// kind, or seeds up to 32 schemes.  A full stack moves its oldest nodes to the
// warp's overflow stack in global memory.  A warp leaves when the task
// counter is spent and it holds no work; no warp ever waits for another.
//
// Most trees are narrow (after an exact piece most intervals hold one row),
// but a read in a tandem array or a young repeat family can grow a tree of
// 10^5 - 10^6 nodes, and a warp working through it alone would hold the whole
// launch up.  So a task that expands more nodes than its budget exports its
// pending nodes to a global frontier buffer, and the next launch of the same
// kernel takes those nodes as its tasks, spread over every warp; rounds repeat
// until no node is exported.  No work is lost or repeated.  A warp whose
// overflow stack is full also moves its oldest nodes to the frontier buffer.
// Only when the frontier buffer fills, or nodes are still exported after the
// last round, is a read given up (the paper's rule for repetitive reads,
// Section 2): its leaves are dropped and the persistent kernel searches it
// again after the rounds.
#include <algorithm>
#include <mutex>

#include "search_common.cuh"

namespace mica {
namespace {

constexpr unsigned BFULL = 0xffffffffu;
constexpr uint32_t BD_DEEP_MIN = 8192;      // entries of each per-warp overflow stack, at least
constexpr uint32_t SCHEME_FREE = 7;         // the single scheme of reads shorter than k + 1
constexpr uint32_t BD_BUDGET = 1u << 12;    // node expansions a task may take before it exports its nodes
constexpr uint32_t BD_VERIFY_MIN = 12;      // matched bases of a one-row node before it is checked against the text
constexpr uint32_t BD_VERIFY_LEFT = 8;      // ... when at least this many bases are left to match
constexpr int VCAP = 128;                   // rows waiting for that check (the round choice and the room
                                            // checks below keep it from overflowing)
constexpr uint32_t BD_SPLIT_MAX = 8;        // an interval of at most this many rows is checked row by row
constexpr uint32_t BD_CHAIN = 16;           // extension steps a lane may take on one multi-row node in a round
constexpr uint32_t NSLOT_MAX = 64;          // task slots per warp: 32 (one per lane) or 64 (two)
constexpr uint32_t BD_ADMIT_LOW = 96;       // admit new tasks while fewer items are pending ...
constexpr uint32_t BD_ADMIT_FREE = 16;      // ... and at least this many slots are free (or nothing is pending)

// node meta: slot (6 bits) | a (9) | b (9) | d (2) | d0 (2) | scheme (3)
__device__ __forceinline__ uint32_t bd_meta(uint32_t slot, uint32_t a, uint32_t b, uint32_t d, uint32_t d0,
                                            uint32_t j)
{
    return slot | (a << 6) | (b << 15) | (d << 24) | (d0 << 26) | (j << 28);
}
constexpr uint32_t BM_SLOT_MASK = 63u;
__device__ __forceinline__ uint32_t bm_slot(uint32_t x) { return x & BM_SLOT_MASK; }
__device__ __forceinline__ uint32_t bm_a(uint32_t x) { return (x >> 6) & 511u; }
__device__ __forceinline__ uint32_t bm_b(uint32_t x) { return (x >> 15) & 511u; }
__device__ __forceinline__ uint32_t bm_d(uint32_t x) { return (x >> 24) & 3u; }
__device__ __forceinline__ uint32_t bm_d0(uint32_t x) { return (x >> 26) & 3u; }
__device__ __forceinline__ uint32_t bm_j(uint32_t x) { return (x >> 28) & 7u; }

// piece boundaries of a pattern of m bases in p pieces
__device__ __forceinline__ uint32_t bnd(uint32_t i, uint32_t m, uint32_t p) { return i * m / p; }

// The boundaries bnd(0) .. bnd(4) of a task's pieces as 9-bit fields (fields
// past p hold 511), computed once per task so that a node's scheme check
// needs no division.
__device__ __forceinline__ unsigned long long pack_bounds(uint32_t m, uint32_t p)
{
    unsigned long long v = 0;
#pragma unroll
    for (uint32_t i = 0; i <= 4; i++) v |= (unsigned long long)(i <= p ? bnd(i, m, p) : 511u) << (9 * i);
    return v;
}
__device__ __forceinline__ uint32_t bound_at(unsigned long long v, uint32_t i) { return (uint32_t)(v >> (9 * i)) & 511u; }
// the piece holding position pos: the boundaries 1..3 at or below it
__device__ __forceinline__ uint32_t piece_at(unsigned long long v, uint32_t pos)
{
    return (pos >= bound_at(v, 1)) + (pos >= bound_at(v, 2)) + (pos >= bound_at(v, 3));
}

struct BidirArgs {
    IndexView ix;
    OccSide fwd, rev;
    ReadsView rd;
    uint64_t ntasks;
    SearchCtl *ctl;
    Interval *iv;
    uint32_t *iv_cnt;
    uint4 *deep_m;   // per warp: deep_cap multi-row nodes (l, lr, sz, meta)
    uint4 *deep_s;   // per warp: deep_cap single-row nodes (l, lr, meta, 0)
    uint32_t deep_cap;
    uint32_t *redo;  // one bit per read: given up here, to be searched by the persistent kernel
    uint32_t budget; // node expansions per task before it exports its nodes
    // frontier rounds: mode 0 takes (read, strand) tasks, mode 1 the nodes
    // exported by the previous round (task t = 2 read + strand, l, lr, sz; meta)
    uint32_t mode;
    const uint4 *fr_in;
    const uint32_t *fr_in_meta;
    uint4 *fr_out;
    uint32_t *fr_out_meta;
    uint32_t fr_cap;
    // one-row nodes with at least verify_min matched bases are checked
    // against the text (needs the whole suffix array); 0 = never
    uint32_t verify_min;
};

template <int SCAP, int NS>
struct BdSmem {
    uint32_t ml[SCAP], mlr[SCAP], msz[SCAP], mm[SCAP];   // multi-row nodes
    uint32_t sl[SCAP], slr[SCAP], sm[SCAP];              // single-row nodes
    uint32_t vl[VCAP], vm[VCAP];                         // rows to check against the text (row, meta)
    uint32_t pat[NS][MAX_WORDS + 1];                  // pattern of each task slot
    // task slot s: read id, info = m | k << 9 | minus << 11 | p << 12 | end of
    // its scheme range << 15, next scheme to seed
    uint32_t sread[NS], sinfo[NS], snext[NS];
    int live[NS];                                     // nodes of each slot on the stacks
    uint32_t work[NS];                                // node expansions of each slot's task
    unsigned long long bounds[NS];                    // piece boundaries of each slot's pattern
    unsigned long long stage_off[NS];                 // admission: word offset of each new slot's read,
    uint32_t stage_m[NS];                             //   its length | minus << 15,
    uint8_t rank_lane[NS];                            //   and the slot of the j-th new task
    uint8_t seed_list[32];                               // a seed round's slots
};

template <int SCAP, int NS>
__device__ __forceinline__ uint32_t slot_task(const BdSmem<SCAP, NS> &W, uint32_t slot)
{
    return 2 * W.sread[slot] + ((W.sinfo[slot] >> 11) & 1u);
}

// Occ(c, row) for one symbol c on one side, from a loaded block.
__device__ __forceinline__ uint32_t occ_single_side(const OccSide &ix, uint32_t b, uint32_t o, const uint4 &sup,
                                                    const OccBlock &k, uint32_t c)
{
    uint32_t xl = (c & 1u) ? 0u : 0xffffffffu;
    uint32_t xh = (c & 2u) ? 0u : 0xffffffffu;
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint32_t rem = min(max((int)o - 32 * j, 0), 32);
        n += __popc((k.lo[j] ^ xl) & (k.hi[j] ^ xh) & low_mask(rem));
    }
    uint32_t start = b * OCC_ROWS;
    if (c == 0 && ix.dollar_row >= start && ix.dollar_row < start + o) n -= 1;
    uint32_t rel = c == 0 ? (k.ac & 0xffffu) : c == 1 ? (k.ac >> 16) : c == 2 ? (k.gt & 0xffffu) : (k.gt >> 16);
    uint32_t base = c == 0 ? sup.x : c == 1 ? sup.y : c == 2 ? sup.z : sup.w;
    return base + rel + n;
}

__device__ __forceinline__ uint32_t side_C(const OccSide &s, uint32_t c)
{
    return c == 0 ? s.C[0] : c == 1 ? s.C[1] : c == 2 ? s.C[2] : s.C[3];
}

// Stage the packed words of `nnew` newly admitted slots into their pattern
// rows, four lanes per slot and eight slots per pass: lane g of a quad loads
// the 16-byte-aligned chunks g and g + 4 of the slot's read, so consecutive
// lanes read consecutive chunks.  The words of neighbouring reads a chunk
// covers are dropped; a chunk that would reach outside the batch's words
// array (its first or last read only) is read word by word.  Minus-strand
// rows are stored word-reversed; the slot's own lane then complements them.
template <int SCAP, int NS>
__device__ __forceinline__ void bd_stage_patterns(BdSmem<SCAP, NS> &W, const uint32_t *words, const uint32_t *words_end,
                                                  uint32_t nnew, int lane)
{
    const uint32_t quad = (uint32_t)lane >> 2, g = (uint32_t)lane & 3u;
    for (uint32_t base = 0; base < nnew; base += 8) {
        const uint32_t r = base + quad;
        if (r >= nnew) continue;
        const uint32_t src = W.rank_lane[r];
        const uint64_t off = W.stage_off[src];
        const uint32_t m = W.stage_m[src] & 511u, minus = W.stage_m[src] >> 15, Wn = (m + 15) >> 4;
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

__device__ __forceinline__ void bd_complement_row(uint32_t *row, uint32_t m)
{
    const uint32_t Wn = (m + 15) >> 4;
    for (uint32_t q = 0; q < Wn; q++) {
        uint32_t hi = row[q], lo = q + 1 < Wn ? row[q + 1] : 0u;
        row[q] = rc_word(hi, lo, m);
    }
}

// May a child that extends P[a, b) by base c at position pos (to the left
// when a > 0, else to the right) exist under scheme j?  Returns the child's
// d0 (mismatches before its current left piece) through d0n.
__device__ __forceinline__ bool bd_allowed(uint32_t j, uint32_t a, uint32_t pos, unsigned long long bounds,
                                           uint32_t k, uint32_t d, uint32_t d0, uint32_t cost, uint32_t &d0n)
{
    const uint32_t dn = d + cost;
    d0n = d0;
    if (dn > k) return false;
    if (j == SCHEME_FREE || a == 0) return true;              // free scheme, or the right phase
    const uint32_t i = piece_at(bounds, pos);
    if (i == j) return cost == 0;                             // the exact piece
    // a piece left of j: it needs a substitution, and so do pieces 0 .. i - 1
    d0n = (a == bound_at(bounds, i + 1)) ? d : d0;            // entering piece i
    const uint32_t dp = dn - d0n;
    if (pos == bound_at(bounds, i)) return dp >= 1 && dn + i <= k;   // piece i complete
    return dn + i + (dp == 0 ? 1u : 0u) <= k;
}

// The text check of a one-row node: its pattern `pat` (m bases in p pieces
// with boundaries `bnds`, scheme j, budget k) has P[A, B) matched at text
// position t = SA[l].  Below a one-row node the tree is a single path, the
// text around that occurrence (each row has one preceding and, in the
// reversed genome's index, one following symbol), so the node has a leaf iff
// the window G[t - A, t - A + m) lies inside G and meets the scheme: at most
// k mismatches in all, none in piece j, at least one in each piece left of j
// (the free scheme of short reads: the budget alone).  The window's mismatch
// count goes to d, the text words read to words and the 32-byte sectors
// they span to sectors.
__device__ __forceinline__ bool bd_check_window(const uint32_t *__restrict__ text, uint64_t n, const uint32_t *pat,
                                                uint32_t m, unsigned long long bnds, uint32_t j, uint32_t k,
                                                uint32_t t, uint32_t A, uint32_t &d, uint32_t &words,
                                                uint32_t &sectors)
{
    words = 0;
    sectors = 0;
    d = 0;
    if (t < A || (uint64_t)(t - A) + m > n) return false;
    const uint32_t s0 = t - A, w0 = s0 >> 4, sh = 2u * (s0 & 15u);
    const uint32_t Wn = (m + 15) >> 4;
    const int b1 = (int)bound_at(bnds, 1), b2 = (int)bound_at(bnds, 2), b3 = (int)bound_at(bnds, 3);
    uint32_t tot = 0, c1 = 0, c2 = 0, c3 = 0;   // mismatches in all and before boundaries 1, 2, 3
    uint32_t prev = __ldg(text + w0);
    for (uint32_t q0 = 0; q0 < Wn; q0 += 8) {
        uint32_t tw[8];
#pragma unroll
        for (int i = 0; i < 8; i++) tw[i] = (q0 + i < Wn) ? __ldg(text + w0 + q0 + i + 1) : 0u;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const uint32_t q = q0 + (uint32_t)i;
            if (q < Wn) {
                const uint32_t g = __funnelshift_r(prev, tw[i], sh);   // G[s0 + 16 q, s0 + 16 q + 16)
                prev = tw[i];
                uint32_t x = pat[q] ^ g;
                x = (x | (x >> 1)) & 0x55555555u;                     // bit 2i: base 16 q + i differs
                const int base = 16 * (int)q;
                x &= low_mask(2u * (uint32_t)min(max((int)m - base, 0), 16));
                tot += __popc(x);
                c1 += __popc(x & low_mask(2u * (uint32_t)min(max(b1 - base, 0), 16)));
                c2 += __popc(x & low_mask(2u * (uint32_t)min(max(b2 - base, 0), 16)));
                c3 += __popc(x & low_mask(2u * (uint32_t)min(max(b3 - base, 0), 16)));
            }
        }
    }
    words = Wn + 1;
    sectors = ((w0 & 7u) * 4u + 4u * words + 31u) / 32u;
    d = tot;
    if (tot > k) return false;
    if (j == SCHEME_FREE) return true;
    const uint32_t pc0 = c1, pc1 = c2 - c1, pc2 = c3 - c2, pc3 = tot - c3;
    const uint32_t pj = j == 0 ? pc0 : j == 1 ? pc1 : j == 2 ? pc2 : pc3;
    return pj == 0 && (j < 1 || pc0 > 0) && (j < 2 || pc1 > 0) && (j < 3 || pc2 > 0);
}

// Move the n oldest nodes of a stack to the warp's overflow stack (n fits).
template <int SCAP, int NS, bool SINGLE>
__device__ __forceinline__ void bd_deep_push(BdSmem<SCAP, NS> &W, uint4 *deep, uint32_t &dtop, uint32_t &bot, uint32_t n,
                                             int lane)
{
    for (uint32_t r0 = 0; r0 < n; r0 += 32) {
        uint32_t t = r0 + (uint32_t)lane;
        if (t < n) {
            uint32_t q = (bot + t) & (SCAP - 1);
            deep[dtop + t] = SINGLE ? make_uint4(W.sl[q], W.slr[q], W.sm[q], 0u)
                                    : make_uint4(W.ml[q], W.mlr[q], W.msz[q], W.mm[q]);
        }
    }
    dtop += n;
    bot += n;
    __syncwarp();
}

// Bring the n most recently moved nodes back under the stack's bottom.
template <int SCAP, int NS, bool SINGLE>
__device__ __forceinline__ void bd_deep_pop(BdSmem<SCAP, NS> &W, const uint4 *deep, uint32_t &dtop, uint32_t &bot,
                                            uint32_t n, int lane)
{
    for (uint32_t r0 = 0; r0 < n; r0 += 32) {
        uint32_t t = r0 + (uint32_t)lane;
        if (t < n) {
            uint32_t q = (bot - n + t) & (SCAP - 1);
            uint4 v = deep[dtop - n + t];
            if (SINGLE) { W.sl[q] = v.x; W.slr[q] = v.y; W.sm[q] = v.z; }
            else { W.ml[q] = v.x; W.mlr[q] = v.y; W.msz[q] = v.z; W.mm[q] = v.w; }
        }
    }
    dtop -= n;
    bot -= n;
    __syncwarp();
}

// Give up a read (the paper's rule for repetitive reads, Section 2): its bit
// in the redo set; the first to set it counts it.
__device__ __forceinline__ void bd_give_up(const BidirArgs &a, uint32_t rid)
{
    const uint32_t bit = 1u << (rid & 31);
    if (!(atomicOr(&a.redo[rid >> 5], bit) & bit)) atomicAdd(&a.ctl->redo_reads, 1u);
}

// Export one node to the frontier buffer slot q (past the end: give its read up).
__device__ __forceinline__ void bd_export_one(const BidirArgs &a, uint32_t q, uint32_t task, uint32_t l, uint32_t lr,
                                              uint32_t sz, uint32_t meta)
{
    if (q < a.fr_cap) {
        a.fr_out[q] = make_uint4(task, l, lr, sz);
        a.fr_out_meta[q] = meta & ~BM_SLOT_MASK;
    } else {
        bd_give_up(a, task >> 1);
    }
}

// Move the nodes of the slots in `expm` out of one stack (the shared-memory
// part [bot, top) or the overflow part deep[0, dtop)): exported nodes go to
// the frontier buffer, the others are compacted in their order.  Returns
// the nodes kept.
template <int SCAP, int NS, bool SINGLE, bool DEEP>
__device__ __forceinline__ uint32_t bd_export_stack(BdSmem<SCAP, NS> &W, const BidirArgs &a, uint4 *deep, uint32_t bot,
                                                    uint32_t top, unsigned long long expm, int lane)
{
    const unsigned lt = (1u << lane) - 1u;
    uint32_t kept = 0;
    for (uint32_t r0 = bot; r0 < top; r0 += 32) {
        const uint32_t e = r0 + (uint32_t)lane;
        const bool has = e < top;
        uint32_t l = 0, lr = 0, sz = 1, meta = 0;
        if (has) {
            if (DEEP) {
                const uint4 v = deep[e];
                l = v.x; lr = v.y;
                if (SINGLE) meta = v.z; else { sz = v.z; meta = v.w; }
            } else {
                const uint32_t q = e & (SCAP - 1);
                if (SINGLE) { l = W.sl[q]; lr = W.slr[q]; meta = W.sm[q]; }
                else { l = W.ml[q]; lr = W.mlr[q]; sz = W.msz[q]; meta = W.mm[q]; }
            }
        }
        const uint32_t slot = bm_slot(meta);
        const bool ex = has && ((expm >> slot) & 1ull);
        const uint32_t task = ex ? slot_task(W, slot) : 0u;
        const bool keep = has && !ex;
        const unsigned em = __ballot_sync(BFULL, ex), km = __ballot_sync(BFULL, keep);
        uint32_t base = 0;
        if (em) {
            if (lane == 0) base = atomicAdd(&a.ctl->fr_count, (unsigned)__popc(em));
            base = __shfl_sync(BFULL, base, 0);
        }
        __syncwarp();   // every lane has read its entry before any is overwritten below
        if (ex) bd_export_one(a, base + __popc(em & lt), task, l, lr, sz, meta);
        if (keep) {
            const uint32_t o = (DEEP ? 0u : bot) + kept + __popc(km & lt);
            if (DEEP) deep[o] = SINGLE ? make_uint4(l, lr, meta, 0u) : make_uint4(l, lr, sz, meta);
            else {
                const uint32_t q = o & (SCAP - 1);
                if (SINGLE) { W.sl[q] = l; W.slr[q] = lr; W.sm[q] = meta; }
                else { W.ml[q] = l; W.mlr[q] = lr; W.msz[q] = sz; W.mm[q] = meta; }
            }
        }
        kept += __popc(km);
        __syncwarp();
    }
    return kept;
}

// Room for `add` more nodes on a stack: its oldest nodes go to the warp's
// overflow stack, or, when that is full, to the frontier buffer as tasks of
// the next round.
template <int SCAP, int NS, bool SINGLE>
__device__ __forceinline__ void bd_make_room(BdSmem<SCAP, NS> &W, const BidirArgs &a, uint4 *deep, uint32_t &dtop,
                                             uint32_t &bot, uint32_t top, uint32_t add, int lane, uint32_t &c_deep)
{
    if ((top - bot) + add <= (uint32_t)SCAP) return;
    uint32_t nsp = (top - bot) + add - SCAP + SCAP / 4;
    nsp = min((nsp + 31) & ~31u, top - bot);
    if (dtop + nsp <= a.deep_cap) {
        bd_deep_push<SCAP, NS, SINGLE>(W, deep, dtop, bot, nsp, lane);
        c_deep += nsp;
        return;
    }
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t r0 = 0; r0 < nsp; r0 += 32) {
        const uint32_t t = r0 + (uint32_t)lane;
        const bool has = t < nsp;
        uint32_t l = 0, lr = 0, sz = 1, meta = 0;
        if (has) {
            const uint32_t q = (bot + t) & (SCAP - 1);
            if (SINGLE) { l = W.sl[q]; lr = W.slr[q]; meta = W.sm[q]; }
            else { l = W.ml[q]; lr = W.mlr[q]; sz = W.msz[q]; meta = W.mm[q]; }
        }
        const uint32_t slot = bm_slot(meta);
        const uint32_t task = has ? slot_task(W, slot) : 0u;
        const unsigned em = __ballot_sync(BFULL, has);
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&a.ctl->fr_count, (unsigned)__popc(em));
        base = __shfl_sync(BFULL, base, 0);
        if (has) {
            bd_export_one(a, base + __popc(em & lt), task, l, lr, sz, meta);
            atomicAdd(&W.live[slot], -1);
        }
    }
    bot += nsp;
    __syncwarp();
}

// Write the leaves of this round (at most four per lane) with one warp-wide atomic.
__device__ __forceinline__ void bd_emit(const BidirArgs &a, uint32_t nleaf, const uint32_t (&cl)[4],
                                        const uint32_t (&csz)[4], const uint32_t (&cd)[4], uint32_t leafmask,
                                        uint32_t rid, uint32_t minus, int lane)
{
    if (!__ballot_sync(BFULL, nleaf != 0)) return;
    uint32_t pre = nleaf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(BFULL, pre, o);
        if (lane >= o) pre += y;
    }
    uint32_t tot = __shfl_sync(BFULL, pre, 31);
    pre -= nleaf;
    uint32_t at0 = 0;
    if (lane == 0) at0 = atomicAdd(&a.ctl->iv_count, tot);
    at0 = __shfl_sync(BFULL, at0, 0);
    if (nleaf) {
        atomicAdd(&a.iv_cnt[rid], nleaf);
        uint32_t q = at0 + pre;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (leafmask >> c & 1u) {
                if (q < a.ctl->iv_cap) {
                    Interval x;
                    x.read = rid; x.meta = cd[c] | (minus << 2); x.l = cl[c]; x.r = cl[c] + csz[c];
                    a.iv[q] = x;
                } else {
                    atomicOr(&a.ctl->error, ERR_IV_OVERFLOW);
                }
                q++;
            }
        }
    }
}

// Rows for the text-check stack: each lane asks for `want` rows (0: none).
// Lanes are taken in lane order while their rows fit in the stack's room (the
// taken lanes form a prefix, so their rows lie contiguously from vtop); a
// lane gets its first position in pos.  vtop grows by the rows taken.
__device__ __forceinline__ bool bd_take_rows(uint32_t want, uint32_t &vtop, uint32_t &pos, int lane)
{
    uint32_t end = want;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(BFULL, end, o);
        if (lane >= o) end += y;
    }
    const bool ok = want > 0 && end <= (uint32_t)VCAP - vtop;
    pos = vtop + end - want;
    vtop += __reduce_max_sync(BFULL, ok ? end : 0u);
    return ok;
}

template <int SCAP, int WARPS, int MINB, int NS>
__global__ void __launch_bounds__(WARPS * 32, MINB) k_bidir(BidirArgs a)
{
    // a frontier round with nothing exported to it (most batches need none)
    const unsigned long long ntasks = *(volatile unsigned long long *)&a.ctl->ntasks;
    if (ntasks == 0) return;
    extern __shared__ uint4 bd_smem_raw[];
    BdSmem<SCAP, NS> *all = reinterpret_cast<BdSmem<SCAP, NS> *>(bd_smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    BdSmem<SCAP, NS> &W = all[warp];
    const IndexView &ix = a.ix;
    SearchCtl *ctl = a.ctl;
    const unsigned lt = (1u << lane) - 1u;
    const int wg = (int)blockIdx.x * WARPS + warp;
    uint4 *deep_m = a.deep_m + (size_t)wg * a.deep_cap;
    uint4 *deep_s = a.deep_s + (size_t)wg * a.deep_cap;
    const uint32_t *words_end = a.rd.words + a.rd.word_off[a.rd.n];

    // slot lane (and, with 64 slots, lane + 32) belong to this lane for the bookkeeping below
    constexpr bool TWO = NS == 64;
    constexpr uint32_t HS = TWO ? 2 : 1;
    for (uint32_t h = 0; h < HS; h++) {
        const uint32_t sl = (uint32_t)lane + 32 * h;
        W.live[sl] = 0;
        W.work[sl] = 0;
        W.sread[sl] = 0;
        W.sinfo[sl] = 0;
        W.snext[sl] = 0;
    }
    unsigned used_lo = 0, used_hi = 0;   // slots holding a task (warp-uniform)
    uint32_t mbot = 0, mtop = 0, sbot = 0, stop = 0, dmt = 0, dst = 0;
    uint32_t vtop = 0;   // nodes waiting for the text check: W.v*[0, vtop)
    bool tasks_left = true;
    // once the launch's task counter is spent, a task keeps an eighth of its
    // budget: a warp left holding heavy trees hands them to the next round,
    // where every warp takes part, instead of working through them alone
    uint32_t budget = a.budget;
    uint32_t c_seeds = 0, c_nodes = 0, c_blocks = 0, c_deep = 0, c_rounds = 0, c_verify = 0, c_vbytes = 0, c_vsect = 0;
    __syncwarp();

    for (uint32_t iter = 0;; iter++) {
        if ((iter & 15) == 0 && *(volatile unsigned *)&ctl->error != 0) break;
        // a slot frees once its nodes are gone and its schemes are seeded
        const uint32_t lane2 = TWO ? (uint32_t)lane + 32 : (uint32_t)lane;   // the lane's second slot
        bool u0 = (used_lo >> lane) & 1u, u1 = TWO && ((used_hi >> lane) & 1u);
        const uint32_t i0 = W.sinfo[lane], i1 = W.sinfo[lane2];
        const uint32_t n0 = W.snext[lane], n1 = W.snext[lane2];
        if (u0 && W.live[lane] == 0 && n0 >= ((i0 >> 15) & 7u)) u0 = false;
        if (u1 && W.live[lane2] == 0 && n1 >= ((i1 >> 15) & 7u)) u1 = false;
        used_lo = __ballot_sync(BFULL, u0);
        used_hi = __ballot_sync(BFULL, u1);
        uint32_t mc = mtop - mbot, sc = stop - sbot;
        if (mc < 32 && dmt > 0) {
            uint32_t n = min(dmt, 64u);
            bd_deep_pop<SCAP, NS, false>(W, deep_m, dmt, mbot, n, lane);
            mc += n;
        }
        if (sc < 32 && dst > 0) {
            uint32_t n = min(dst, 64u);
            bd_deep_pop<SCAP, NS, true>(W, deep_s, dst, sbot, n, lane);
            sc += n;
        }
        if ((iter & 63) == 63 && budget == a.budget) {
            int spent = 0;
            if (lane == 0) spent = *(volatile unsigned long long *)&ctl->task_head >= ntasks;
            if (__shfl_sync(BFULL, spent, 0)) budget = max(a.budget >> 3, min(a.budget, 32u));
        }
        // ---- slots over their node budget hand their nodes to the next
        // round (one pass over both stacks), and their schemes not yet seeded
        // as seed items (size 0, the scheme in the meta word)
        const bool over0 = u0 && W.work[lane] >= budget && (W.live[lane] > 0 || n0 < ((i0 >> 15) & 7u));
        const bool over1 = u1 && W.work[lane2] >= budget && (W.live[lane2] > 0 || n1 < ((i1 >> 15) & 7u));
        const unsigned ex_lo = __ballot_sync(BFULL, over0), ex_hi = __ballot_sync(BFULL, over1);
        if (ex_lo | ex_hi) {
            const unsigned long long expm = (unsigned long long)ex_lo | ((unsigned long long)ex_hi << 32);
            const uint32_t ns0 = over0 ? ((i0 >> 15) & 7u) - n0 : 0u, ns1 = over1 ? ((i1 >> 15) & 7u) - n1 : 0u;
            uint32_t pre = ns0 + ns1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(BFULL, pre, o);
                if (lane >= o) pre += y;
            }
            const uint32_t tot = __shfl_sync(BFULL, pre, 31);
            pre -= ns0 + ns1;
            if (tot) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&ctl->fr_count, tot);
                base = __shfl_sync(BFULL, base, 0);
                for (uint32_t i = 0; i < ns0; i++)
                    bd_export_one(a, base + pre + i, slot_task(W, lane), 0, 0, 0, bd_meta(0, 0, 0, 0, 0, n0 + i));
                for (uint32_t i = 0; i < ns1; i++)
                    bd_export_one(a, base + pre + ns0 + i, slot_task(W, lane2), 0, 0, 0,
                                  bd_meta(0, 0, 0, 0, 0, n1 + i));
            }
            if (over0) W.snext[lane] = (i0 >> 15) & 7u;
            if (over1) W.snext[lane2] = (i1 >> 15) & 7u;
            mtop = mbot + bd_export_stack<SCAP, NS, false, false>(W, a, nullptr, mbot, mtop, expm, lane);
            stop = sbot + bd_export_stack<SCAP, NS, true, false>(W, a, nullptr, sbot, stop, expm, lane);
            if (dmt) dmt = bd_export_stack<SCAP, NS, false, true>(W, a, deep_m, 0, dmt, expm, lane);
            if (dst) dst = bd_export_stack<SCAP, NS, true, true>(W, a, deep_s, 0, dst, expm, lane);
            if (over0) W.live[lane] = 0;   // their nodes are gone: the slots free above ...
            if (over1) W.live[lane2] = 0;
            __syncwarp();
            // ... once the rows they have waiting for the text check are done: those stay here (a row
            // split from an interval has no row of the reversed genome to travel with)
            for (uint32_t e = (uint32_t)lane; e < vtop; e += 32) {
                const uint32_t sl = bm_slot(W.vm[e]);
                if ((expm >> sl) & 1ull) atomicAdd(&W.live[sl], 1);
            }
            if (over0) W.work[lane] = 0;   // (so that this pass does not repeat while they wait)
            if (over1) W.work[lane2] = 0;
            __syncwarp();
            continue;
        }
        const bool av0 = u0 && n0 < ((i0 >> 15) & 7u), av1 = u1 && n1 < ((i1 >> 15) & 7u);
        const unsigned avail_lo = __ballot_sync(BFULL, av0), avail_hi = __ballot_sync(BFULL, av1);
        const uint32_t seeds_total = __popc(avail_lo) + __popc(avail_hi);
        const uint32_t cnt = mc + sc + vtop;

        // ---- admission of fresh tasks (or of the last round's exported nodes) into free slots
        const unsigned free_lo = ~used_lo, free_hi = TWO ? ~used_hi : 0u;
        const uint32_t nfree = __popc(free_lo) + __popc(free_hi);
        // the nodes of a frontier round's tasks go onto the stacks at once: room for them
        const uint32_t room = a.mode == 1 ? (uint32_t)SCAP - max(mc, sc) : nfree;
        if (tasks_left && nfree != 0 && dmt + dst == 0 && cnt + seeds_total < BD_ADMIT_LOW &&
            (cnt + seeds_total == 0 || nfree >= BD_ADMIT_FREE) && room > 0) {
            uint32_t want = min(nfree, room), got = 0;
            unsigned long long t0 = 0;
            if (lane == 0) {
                if (*(volatile unsigned long long *)&ctl->task_head < ntasks) {
                    t0 = atomicAdd(&ctl->task_head, (unsigned long long)want);
                    if (t0 < ntasks) got = (uint32_t)min((unsigned long long)want, ntasks - t0);
                }
            }
            got = __shfl_sync(BFULL, got, 0);
            t0 = __shfl_sync(BFULL, t0, 0);
            if (got == 0) {
                tasks_left = false;
            } else {
                const uint32_t nlo = __popc(free_lo);
                uint4 it[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
                uint32_t imeta[2] = {0, 0};
                bool push[2] = {false, false};
                uint32_t minus_new = 0;
#pragma unroll
                for (uint32_t h = 0; h < HS; h++) {
                    const uint32_t sl = (uint32_t)lane + 32 * h;
                    const bool fr = h == 0 ? ((free_lo >> lane) & 1u) : ((free_hi >> lane) & 1u);
                    const uint32_t jr = h == 0 ? __popc(free_lo & lt) : nlo + __popc(free_hi & lt);
                    if (!fr || jr >= got) continue;
                    unsigned long long t = t0 + jr;
                    uint32_t seed_j = 8;                   // 8: not a seed item
                    if (a.mode == 1) {                     // a node (or a scheme to seed) exported by the last round
                        it[h] = a.fr_in[t];
                        imeta[h] = a.fr_in_meta[t];
                        if (it[h].w == 0) seed_j = bm_j(imeta[h]);
                        t = it[h].x;
                    }
                    const uint32_t rid = (uint32_t)(t >> 1), minus = (uint32_t)(t & 1);
                    const uint32_t m = a.rd.len[rid], k = a.rd.k[rid];
                    const uint32_t p = m >= k + 1 ? k + 1 : 1u;
                    const uint32_t nsch = m >= k + 1 ? p : 1u;
                    const bool given_up = a.mode == 1 && ((a.redo[rid >> 5] >> (rid & 31)) & 1u);
                    // a seed item seeds its one scheme: the slot's scheme range is [j, j + 1)
                    const uint32_t send = seed_j < 8 ? seed_j + 1 : nsch;
                    W.sread[sl] = rid;
                    W.sinfo[sl] = m | (k << 9) | (minus << 11) | (p << 12) | (send << 15);
                    W.snext[sl] = a.mode == 0 ? 0 : (seed_j < 8 && !given_up ? seed_j : send);
                    // the node of a read already given up is not continued
                    push[h] = a.mode == 1 && seed_j == 8 && !given_up;
                    W.live[sl] = push[h] ? 1 : 0;
                    W.work[sl] = 0;
                    W.bounds[sl] = pack_bounds(m, p);
                    W.rank_lane[jr] = (uint8_t)sl;
                    W.stage_off[sl] = a.rd.word_off[rid];
                    W.stage_m[sl] = m | (minus << 15);
                    if (minus) minus_new |= 1u << h;
                    if (h == 0) u0 = true; else u1 = true;
                }
                used_lo = __ballot_sync(BFULL, u0);
                used_hi = __ballot_sync(BFULL, u1);
                __syncwarp();
                bd_stage_patterns<SCAP, NS>(W, a.rd.words, words_end, got, lane);
                __syncwarp();
                for (uint32_t h = 0; h < HS; h++)
                    if ((minus_new >> h) & 1u) {
                        const uint32_t sl = (uint32_t)lane + 32 * h;
                        bd_complement_row(W.pat[sl], W.sinfo[sl] & 511u);
                    }
                if (a.mode == 1) {
                    // the admitted nodes onto the stacks
#pragma unroll
                    for (uint32_t h = 0; h < HS; h++) {
                        const uint32_t sl = (uint32_t)lane + 32 * h;
                        const bool single = it[h].w == 1;
                        const unsigned bm = __ballot_sync(BFULL, push[h] && !single),
                                       bs = __ballot_sync(BFULL, push[h] && single);
                        if (push[h] && !single) {
                            uint32_t q = (mtop + __popc(bm & lt)) & (SCAP - 1);
                            W.ml[q] = it[h].y; W.mlr[q] = it[h].z; W.msz[q] = it[h].w; W.mm[q] = imeta[h] | sl;
                        }
                        if (push[h] && single) {
                            uint32_t q = (stop + __popc(bs & lt)) & (SCAP - 1);
                            W.sl[q] = it[h].y; W.slr[q] = it[h].z; W.sm[q] = imeta[h] | sl;
                        }
                        mtop += __popc(bm);
                        stop += __popc(bs);
                    }
                }
                __syncwarp();
                continue;
            }
        }
        if (cnt + seeds_total == 0) {
            if (!tasks_left && (used_lo | used_hi) == 0) break;   // nothing held, nothing left
            if (!tasks_left) {
                // slots held but no work: cannot happen while the counts are right
                if (lane == 0) atomicOr(&ctl->error, ERR_TIMEOUT);
                break;
            }
            continue;
        }
        c_rounds++;

        // (rounds other than the text check's run only while fewer than 32
        // rows wait for it; they add rows only while those fit)
        int kind;
        const bool seed_room = mc + 32 <= (uint32_t)SCAP && sc + 32 <= (uint32_t)SCAP;
        if (vtop >= 32) kind = 3;
        else if (mc >= 32) kind = 0;
        else if (sc >= 32) kind = 1;
        else if (seeds_total > 0 && seed_room && (seeds_total >= 32 || seeds_total >= max(max(mc, sc), vtop)))
            kind = 2;
        else if (mc && mc >= sc && mc >= vtop) kind = 0;
        else if (sc && sc >= vtop) kind = 1;
        else if (vtop) kind = 3;
        else kind = 2;

        if (kind == 2) {
            // ---- one scheme's seed for each of up to 32 slots with schemes left:
            // piece j's last bases from both tables
            const uint32_t r0 = __popc(avail_lo & lt), r1 = __popc(avail_lo) + __popc(avail_hi & lt);
            if (av0 && r0 < 32) W.seed_list[r0] = (uint8_t)lane;
            if (av1 && r1 < 32) W.seed_list[r1] = (uint8_t)lane2;
            __syncwarp();
            const bool avail = (uint32_t)lane < min(seeds_total, 32u);
            const uint32_t slot = avail ? W.seed_list[lane] : 0u;
            const uint32_t info = W.sinfo[slot];
            bool push = false, leaf = false;
            uint32_t l = 0, lr = 0, sz = 0, meta = 0;
            if (avail) {
                const uint32_t m = info & 511u, k = (info >> 9) & 3u, p = (info >> 12) & 7u;
                const uint32_t nsch = (info >> 15) & 7u;
                const uint32_t j = W.snext[slot]++;
                const uint32_t *pat = W.pat[slot];
                if (nsch == 1 && p == 1 && k > 0) {
                    // a read shorter than k + 1 bases: the whole tree from the full interval
                    l = 0; lr = 0; sz = ix.rows;
                    meta = bd_meta(slot, m, m, 0, 0, SCHEME_FREE);
                    push = true;
                } else {
                    // from the longer seed tables when the index has them
                    const bool longer = ix.lfwd.table != nullptr;
                    const uint32_t tq = longer ? ix.lfwd.q : ix.q;
                    const uint32_t bj = bound_at(W.bounds[slot], j + 1), aj = bound_at(W.bounds[slot], j);
                    const uint32_t qe = min(tq, bj - aj);
                    // the codes of P[bj - qe, bj) (forward: P[bj - qe] first) and of its reversal
                    // (P[bj - 1] first).  The 64-slot shape reads them straight off the packed
                    // pattern: the bases least significant first are the reversal's code, the same
                    // groups in reverse order the forward one; the 32-slot shape builds them base by
                    // base, which measured faster there (7.7 against 8.2 ms on a 512 Mbp genome,
                    // while the word form took 64 Mbp from 2.33 to 2.24 ms)
                    uint32_t code = 0, rcode = 0;
                    if (TWO) {
                        const uint32_t s0 = bj - qe, wi = s0 >> 4;
                        rcode = __funnelshift_r(pat[wi], pat[wi + 1], 2 * (s0 & 15)) & ((1u << (2 * qe)) - 1u);
                        code = rev_groups(rcode) >> (2 * (16 - qe));
                    } else {
                        for (uint32_t t = 0; t < qe; t++) {
                            code = (code << 2) | pat_base(pat, bj - qe + t);
                            rcode = (rcode << 2) | pat_base(pat, bj - 1 - t);
                        }
                    }
                    uint32_t fl, fr, rl, rr;
                    if (longer) {
                        seed_interval_in(ix.lfwd.table, tq, ix.lfwd.nshort, ix.lfwd.short_pad, ix.lfwd.short_len,
                                         ix.lfwd.short_bloom, code, qe, fl, fr);
                        seed_interval_in(ix.lrev.table, tq, ix.lrev.nshort, ix.lrev.short_pad, ix.lrev.short_len,
                                         ix.lrev.short_bloom, rcode, qe, rl, rr);
                    } else {
                        seed_interval_in(ix.table, ix.q, ix.nshort, ix.short_pad, ix.short_len, ix.short_bloom, code,
                                         qe, fl, fr);
                        seed_interval_in(ix.rev.table, ix.q, ix.rev.nshort, ix.rev.short_pad, ix.rev.short_len,
                                         ix.rev.short_bloom, rcode, qe, rl, rr);
                    }
                    c_seeds++;
                    if (fl < fr) {
                        l = fl; lr = rl; sz = fr - fl;
                        const uint32_t a0 = bj - qe;
                        if (a0 == 0 && bj == m) leaf = true;
                        else { meta = bd_meta(slot, a0, bj, 0, 0, j); push = true; }
                    }
                }
            }
            const uint32_t minus = (info >> 11) & 1u;
            uint32_t cl[4] = {l, 0, 0, 0}, cs[4] = {sz, 0, 0, 0}, cd[4] = {0, 0, 0, 0};
            bd_emit(a, leaf ? 1u : 0u, cl, cs, cd, leaf ? 1u : 0u, W.sread[slot], minus, lane);
            const bool single = sz == 1;
            // a seed of a few rows, far enough in, goes straight to the text check row by row
            const uint32_t matched = bm_b(meta) - bm_a(meta);
            const bool checkable = push && a.verify_min && sz <= BD_SPLIT_MAX && matched >= a.verify_min &&
                                   (info & 511u) - matched >= BD_VERIFY_LEFT;
            uint32_t vpos = 0;
            const bool to_v = bd_take_rows(checkable ? sz : 0u, vtop, vpos, lane);
            if (to_v)
                for (uint32_t i = 0; i < sz; i++) { W.vl[vpos + i] = l + i; W.vm[vpos + i] = meta; }
            const unsigned bm = __ballot_sync(BFULL, push && !single && !to_v),
                           bs = __ballot_sync(BFULL, push && single && !to_v);
            if (push && !single && !to_v) {
                uint32_t q = (mtop + __popc(bm & lt)) & (SCAP - 1);
                W.ml[q] = l; W.mlr[q] = lr; W.msz[q] = sz; W.mm[q] = meta;
            }
            if (push && single && !to_v) {
                uint32_t q = (stop + __popc(bs & lt)) & (SCAP - 1);
                W.sl[q] = l; W.slr[q] = lr; W.sm[q] = meta;
            }
            mtop += __popc(bm);
            stop += __popc(bs);
            if (push) atomicAdd(&W.live[slot], to_v ? (int)sz : 1);
        } else if (kind == 1) {
            // ---- single-row nodes: the one possible child is the row's symbol
            const uint32_t npop = min(sc, 32u);
            const bool has = (uint32_t)lane < npop;
            uint32_t l = 0, lr = 0, meta = 0;
            if (has) {
                uint32_t q = (stop - 1 - lane) & (SCAP - 1);
                l = W.sl[q]; lr = W.slr[q]; meta = W.sm[q];
            }
            stop -= npop;
            __syncwarp();
            const uint32_t slot = bm_slot(meta);
            const uint32_t info = W.sinfo[slot];
            const uint32_t rid = W.sread[slot];
            bool child = false, leaf = false;
            uint32_t nl = l, nlr = lr, nmeta = 0, dn = 0;
            // a node far enough in (and far enough from the end) goes to the text check
            const uint32_t matched = bm_b(meta) - bm_a(meta);
            const bool checkable = has && a.verify_min && matched >= a.verify_min &&
                                   (info & 511u) - matched >= BD_VERIFY_LEFT;
            uint32_t vpos = 0;
            const bool to_v = bd_take_rows(checkable ? 1u : 0u, vtop, vpos, lane);
            if (to_v) { W.vl[vpos] = l; W.vm[vpos] = meta; }
            const bool live_node = has && !to_v;
            if (live_node) atomicAdd(&W.work[slot], 1u);
            if (live_node) {
                const uint32_t m = info & 511u, k = (info >> 9) & 3u;
                const uint32_t A = bm_a(meta), B = bm_b(meta), d = bm_d(meta), d0 = bm_d0(meta), j = bm_j(meta);
                const bool left = A > 0;
                const OccSide &sd = left ? a.fwd : a.rev;
                const uint32_t row = left ? l : lr;
                c_nodes++;
                if (row != sd.dollar_row) {
                    const uint32_t bk = row / OCC_ROWS, o = row - bk * OCC_ROWS;
                    uint4 sup = ld_nc(sd.super + bk / SB_BLOCKS);
                    OccBlock blk;
                    load_block(sd, bk, o + 1, blk);
                    c_blocks++;
                    const uint32_t c = block_symbol(blk, o);
                    const uint32_t pos = left ? A - 1 : B;
                    const uint32_t cost = c != pat_base(W.pat[slot], pos) ? 1u : 0u;
                    uint32_t d0n;
                    if (bd_allowed(j, A, pos, W.bounds[slot], k, d, d0, cost, d0n)) {
                        const uint32_t nr = side_C(sd, c) + occ_single_side(sd, bk, o, sup, blk, c);
                        if (left) nl = nr; else nlr = nr;
                        dn = d + cost;
                        const uint32_t nA = left ? pos : 0, nB = left ? B : pos + 1;
                        if (nA == 0 && nB == m) leaf = true;
                        else { child = true; nmeta = bd_meta(slot, nA, nB, dn, d0n, j); }
                    }
                }
            }
            uint32_t cl[4] = {nl, 0, 0, 0}, cs[4] = {1, 0, 0, 0}, cd[4] = {dn, 0, 0, 0};
            bd_emit(a, leaf ? 1u : 0u, cl, cs, cd, leaf ? 1u : 0u, rid, (info >> 11) & 1u, lane);
            const unsigned bsm = __ballot_sync(BFULL, child);
            if (child) {
                uint32_t q = (stop + __popc(bsm & lt)) & (SCAP - 1);
                W.sl[q] = nl; W.slr[q] = nlr; W.sm[q] = nmeta;
            }
            stop += __popc(bsm);
            if (live_node && !child) atomicAdd(&W.live[slot], -1);
        } else if (kind == 3) {
            // ---- one-row nodes checked against the text: SA gives where the
            // matched part lies, the text window decides the leaf, ISA its row
            const uint32_t npop = min(vtop, 32u);
            const bool has = (uint32_t)lane < npop;
            uint32_t l = 0, meta = 0;
            if (has) {
                const uint32_t q = vtop - 1 - lane;
                l = W.vl[q]; meta = W.vm[q];
            }
            vtop -= npop;
            __syncwarp();
            const uint32_t slot = bm_slot(meta);
            const uint32_t info = W.sinfo[slot];
            const uint32_t rid = W.sread[slot];
            bool leaf = false;
            uint32_t row = 0, dn = 0;
            if (has) {
                atomicAdd(&W.work[slot], 1u);
                const uint32_t m = info & 511u, k = (info >> 9) & 3u;
                const uint32_t t = __ldg(ix.sa_full + l);
                uint32_t words = 0, sectors = 0;
                leaf = bd_check_window(ix.text, ix.n, W.pat[slot], m, W.bounds[slot], bm_j(meta), k, t, bm_a(meta),
                                       dn, words, sectors);
                if (leaf) row = __ldg(ix.isa + (t - bm_a(meta)));
                c_verify++;
                c_vbytes += 4u + 4u * words + (leaf ? 4u : 0u);
                c_vsect += 1u + sectors + (leaf ? 1u : 0u);
            }
            uint32_t cl[4] = {row, 0, 0, 0}, cs[4] = {1, 0, 0, 0}, cd[4] = {dn, 0, 0, 0};
            bd_emit(a, leaf ? 1u : 0u, cl, cs, cd, leaf ? 1u : 0u, rid, (info >> 11) & 1u, lane);
            if (has) atomicAdd(&W.live[slot], -1);
        } else {
            // ---- multi-row nodes: counts of all four symbols at both ends
            // A node whose one child left to push has several rows (a chain
            // through a repeat: the read's base continues, the few rows that
            // differ go to the text check) is extended again in the same
            // round, up to CHAIN steps, instead of a push and a pop per step;
            // only while the next multi-row round would have idle lanes anyway,
            // and only in the 64-slot shape (an HBM-resident index: heavier
            // trees, fuller rounds, and a step that waits longer on memory).
            constexpr uint32_t CHAIN = TWO ? BD_CHAIN : 1u;
            const uint32_t npop = min(mc, 32u);
            bool has = (uint32_t)lane < npop;
            uint32_t l = 0, lr = 0, sz = 0, meta = 0;
            if (has) {
                uint32_t q = (mtop - 1 - lane) & (SCAP - 1);
                l = W.ml[q]; lr = W.mlr[q]; sz = W.msz[q]; meta = W.mm[q];
            }
            mtop -= npop;
            __syncwarp();
            for (uint32_t step = 0; step < CHAIN; step++) {
                const uint32_t slot = bm_slot(meta);
                const uint32_t info = W.sinfo[slot];
                const uint32_t rid = W.sread[slot];
                uint32_t cl[4] = {0, 0, 0, 0}, clr[4] = {0, 0, 0, 0}, cs[4] = {0, 0, 0, 0}, cd[4] = {0, 0, 0, 0};
                uint32_t cmeta[4] = {0, 0, 0, 0};
                uint32_t leafmask = 0, nodemask = 0;
                uint32_t cmatched = 0, cleft = 0;                // the children's matched bases and bases to go
                const bool live_node = has;
                if (has) atomicAdd(&W.work[slot], 1u);
                if (live_node) {
                    const uint32_t m = info & 511u, k = (info >> 9) & 3u;
                    const uint32_t A = bm_a(meta), B = bm_b(meta), d = bm_d(meta), d0 = bm_d0(meta), j = bm_j(meta);
                    const bool left = A > 0;
                    cmatched = B - A + 1;
                    cleft = m - cmatched;
                    const OccSide &sd = left ? a.fwd : a.rev;
                    const uint32_t pl = left ? l : lr;          // interval on the side being extended
                    uint32_t ol[4], orr[4];
                    c_blocks += occ_pair(sd, pl, pl + sz, ol, orr);
                    c_nodes++;
                    const uint32_t pos = left ? A - 1 : B;
                    const uint32_t base = pat_base(W.pat[slot], pos);
                    const uint32_t nA = left ? pos : 0, nB = left ? B : pos + 1;
                    // the other side's interval start: rows of lower symbols (and a $) come first
                    uint32_t acc = (left ? lr : l) + ((sd.dollar_row >= pl && sd.dollar_row < pl + sz) ? 1u : 0u);
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const uint32_t n_c = orr[c] - ol[c];
                        const uint32_t cost = (uint32_t)c != base ? 1u : 0u;
                        uint32_t d0n;
                        if (n_c > 0 && bd_allowed(j, A, pos, W.bounds[slot], k, d, d0, cost, d0n)) {
                            const uint32_t start = side_C(sd, c) + ol[c];
                            cl[c] = left ? start : acc;
                            clr[c] = left ? acc : start;
                            cs[c] = n_c;
                            cd[c] = d + cost;
                            if (nA == 0 && nB == m) leafmask |= 1u << c;
                            else { nodemask |= 1u << c; cmeta[c] = bd_meta(slot, nA, nB, d + cost, d0n, j); }
                        }
                        acc += n_c;
                    }
                }
                bd_emit(a, (uint32_t)__popc(leafmask), cl, cs, cd, leafmask, rid, (info >> 11) & 1u, lane);
                // children of a few rows, far enough in, go to the text check row by row
                uint32_t smask = 0, want = 0;
                if (a.verify_min && cmatched >= a.verify_min && cleft >= BD_VERIFY_LEFT) {
#pragma unroll
                    for (int c = 0; c < 4; c++)
                        if ((nodemask >> c & 1u) && cs[c] <= BD_SPLIT_MAX) { smask |= 1u << c; want += cs[c]; }
                }
                uint32_t vpos = 0;
                if (!bd_take_rows(want, vtop, vpos, lane)) { smask = 0; want = 0; }
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if (smask >> c & 1u)
                        for (uint32_t i = 0; i < cs[c]; i++) { W.vl[vpos] = cl[c] + i; W.vm[vpos] = cmeta[c]; vpos++; }
                nodemask &= ~smask;
                bool cont = false;
                uint32_t nl = 0, nlr = 0, nsz = 0, nmeta = 0;
                if (step + 1 < CHAIN) {
#pragma unroll
                    for (int c = 0; c < 4; c++)
                        if (nodemask == (1u << c) && cs[c] > 1) {
                            cont = true; nl = cl[c]; nlr = clr[c]; nsz = cs[c]; nmeta = cmeta[c];
                        }
                    cont = cont && W.work[slot] < budget;
                    // only while the next multi-row round would have idle lanes anyway
                    if ((mtop - mbot) + dmt + __popc(__ballot_sync(BFULL, cont)) > 32u) cont = false;
                    if (cont) nodemask = 0;
                }
                uint32_t nm = 0, ns = 0;
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if (nodemask >> c & 1u) { if (cs[c] == 1) ns++; else nm++; }
                uint32_t packed = nm | (ns << 8), pre = packed;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(BFULL, pre, o);
                    if (lane >= o) pre += y;
                }
                const uint32_t tot = __shfl_sync(BFULL, pre, 31);
                pre -= packed;
                const uint32_t tm = tot & 0xffu, ts = tot >> 8;
                if (tm | ts) {
                    if (tm) bd_make_room<SCAP, NS, false>(W, a, deep_m, dmt, mbot, mtop, tm, lane, c_deep);
                    if (ts) bd_make_room<SCAP, NS, true>(W, a, deep_s, dst, sbot, stop, ts, lane, c_deep);
                }
                if (nm | ns) {
                    uint32_t pm = mtop + (pre & 0xffu), ps = stop + (pre >> 8);
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        if (nodemask >> c & 1u) {
                            if (cs[c] == 1) {
                                uint32_t q = ps++ & (SCAP - 1);
                                W.sl[q] = cl[c]; W.slr[q] = clr[c]; W.sm[q] = cmeta[c];
                            } else {
                                uint32_t q = pm++ & (SCAP - 1);
                                W.ml[q] = cl[c]; W.mlr[q] = clr[c]; W.msz[q] = cs[c]; W.mm[q] = cmeta[c];
                            }
                        }
                    }
                }
                mtop += tm;
                stop += ts;
                const int delta = (int)(nm + ns + want) - (cont ? 0 : 1);
                if (has && delta) atomicAdd(&W.live[slot], delta);
                if (CHAIN == 1) break;
                __syncwarp();                                   // this step's pushes before the next one's
                if (!__any_sync(BFULL, cont)) break;
                has = cont; l = nl; lr = nlr; sz = nsz; meta = nmeta;
            }
        }
        __syncwarp();
    }

    // counters
    unsigned long long v;
    v = c_seeds;  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(BFULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->seeds, v);
    v = c_nodes;  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(BFULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->nodes, v);
    v = c_blocks; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(BFULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->rank_blocks, v);
    v = (unsigned long long)c_seeds + c_nodes; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(BFULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->lane_ops, v);
    v = c_verify; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(BFULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->verified, v);
    v = c_vbytes; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(BFULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->verify_bytes, v);
    v = c_vsect; for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(BFULL, v, o);
    if (lane == 0 && v) atomicAdd(&ctl->verify_sectors, v);
    if (lane == 0) {
        atomicAdd(&ctl->rounds, (unsigned long long)c_rounds);
        if (c_deep) atomicAdd(&ctl->deep_moves, (unsigned long long)c_deep);
    }
}

// The reads whose bit is set: into list[0, *n_list), with their leaf counts
// set to 0 (their leaves are purged and found again by the persistent kernel).
__global__ void k_redo_collect(const uint32_t *__restrict__ bits, uint64_t n_reads, uint32_t *__restrict__ list,
                               unsigned int *__restrict__ n_list, uint32_t *__restrict__ iv_cnt)
{
    const uint64_t words = (n_reads + 31) / 32;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t b = bits[w];
        while (b) {
            const uint32_t r = (uint32_t)(w * 32) + (uint32_t)(__ffs(b) - 1);
            b &= b - 1;
            list[atomicAdd(n_list, 1u)] = r;
            iv_cnt[r] = 0;
        }
    }
}

// Mark the leaves of given-up reads as purged (the interval scatter skips them).
__global__ void k_iv_purge(Interval *__restrict__ iv, const unsigned int *__restrict__ count_p, uint32_t cap,
                           const uint32_t *__restrict__ bits)
{
    const uint32_t count = min(*count_p, cap);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const uint32_t r = iv[e].read;
        if (r != IV_PURGED && (bits[r >> 5] >> (r & 31) & 1u)) iv[e].read = IV_PURGED;
    }
}

// Between frontier rounds: the nodes the last round exported become the
// next round's tasks.
__global__ void k_bd_round(SearchCtl *ctl, uint32_t fr_cap)
{
    const uint32_t n = min(ctl->fr_count, fr_cap);
    ctl->spills += ctl->fr_count;
    ctl->ntasks = n;
    ctl->task_head = 0;
    ctl->fr_count = 0;
}

// After the last round: the reads of nodes still in the frontier are given up.
__global__ void k_bd_give_up_frontier(SearchCtl *ctl, const uint4 *__restrict__ fr, uint32_t fr_cap,
                                      uint32_t *__restrict__ redo)
{
    const uint32_t n = min(ctl->fr_count, fr_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t rid = fr[i].x >> 1, bit = 1u << (rid & 31);
        if (!(atomicOr(&redo[rid >> 5], bit) & bit)) atomicAdd(&ctl->redo_reads, 1u);
    }
}

struct BidirShape {
    void (*fn)(BidirArgs);
    int scap, warps, minb, slots;
    size_t smem;
    int blocks_per_sm;
};

// 0: 64 task slots per warp, 6 warps per CTA (fuller rounds when each task is
// short: an index whose occurrence blocks stay in L2); 1: 32 slots, 8 warps
// (more warps to hide HBM latency for the deep trees of a human-scale index)
#define MICA_BD_SHAPE(S, W, B, N) {k_bidir<S, W, B, N>, S, W, B, N, sizeof(BdSmem<S, N>) * W, 0}
BidirShape g_bd_shapes[] = {
    MICA_BD_SHAPE(128, 6, 3, 64),
    MICA_BD_SHAPE(128, 8, 3, 32),
};
#undef MICA_BD_SHAPE

std::mutex g_bd_mu;
int g_bd_sms = 0;

int bidir_grid(int device, BidirShape &sh, int &grid)
{
    std::lock_guard<std::mutex> lk(g_bd_mu);
    if (g_bd_sms == 0) MICA_CUDA_TRY(cudaDeviceGetAttribute(&g_bd_sms, cudaDevAttrMultiProcessorCount, device));
    if (sh.blocks_per_sm == 0) {
        MICA_CUDA_TRY(cudaFuncSetAttribute(sh.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
        MICA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh.blocks_per_sm, sh.fn, sh.warps * 32, sh.smem));
        if (sh.blocks_per_sm < 1) sh.blocks_per_sm = 1;
    }
    grid = g_bd_sms * sh.blocks_per_sm;
    return 0;
}

}  // namespace

// The compiled shape a call uses: the tuning's choice, else 64 slots per
// warp when the genome's occurrence blocks stay in L2 (96 MiB or less) and
// 32 when they live in HBM.
int bidir_shape_index(const mica_index *idx)
{
    if (idx->tuning.bidir_shape >= 0) return idx->tuning.bidir_shape;
    return idx->n_occ_blocks * 32 > (96ull << 20) ? 1 : 0;
}

int bidir_shape_count() { return (int)(sizeof(g_bd_shapes) / sizeof(g_bd_shapes[0])); }

bool bidir_available(const mica_index *idx)
{
    return idx->has_rev && idx->view.rev.table != nullptr;
}

// Entries of each warp's overflow stacks: their 32 bytes per entry and warp
// take a sixteenth of the device memory free at the workspace's first
// bidirectional call, at most 8 GiB and at least BD_DEEP_MIN entries.  The
// stacks of a warp whose tasks sit in long repeats (a read inside a tandem
// array matches thousands of rows and branches at every substitution) hold
// the frontier of its depth-first walk; when one fills, its oldest nodes go
// to the next round.
static uint32_t bidir_deep_cap(Workspace &w, uint64_t warps)
{
    if (w.bd_deep_cap == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = 0; }
        uint64_t budget = std::min<uint64_t>(fr / 16, 8ull << 30);
        uint64_t cap = budget / (warps * 32);
        w.bd_deep_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(cap, BD_DEEP_MIN), 1u << 20);
    }
    return w.bd_deep_cap;
}

static uint64_t redo_bits_bytes(uint64_t n) { return ((n + 31) / 32 * 4 + 15) & ~15ull; }
// Items per frontier buffer: 2n, at least 2^20, at most 2^28, and a multiple
// of 4 so that the second buffer and both meta arrays (20 B per item in all)
// start on a 16-byte boundary, as the kernel's 16-byte item loads and stores
// require (an odd batch above 2^19 reads would otherwise put the second
// buffer 8 bytes off).
static uint32_t frontier_cap(uint64_t n)
{
    return (uint32_t)((std::min<uint64_t>(std::max<uint64_t>(2 * n, 1u << 20), 1u << 28) + 3) & ~3ull);
}
constexpr int BD_GRAPH_ROUNDS = 8;   // frontier rounds a captured batch runs (more: the regular path)
constexpr int BD_MAX_ROUNDS = 64;
static uint64_t redo_bytes(uint64_t n) { return redo_bits_bytes(n) + std::max<uint64_t>(n, 1) * 4 + 16; }

// Reserve the bidirectional search's buffers for n reads; fills the control
// block template and the grid.
int prepare_bidir(const mica_index *idx, Workspace &w, uint64_t n, SearchCtl &tmpl, int &grid)
{
    int rc;
    BidirShape &sh = g_bd_shapes[bidir_shape_index(idx)];
    if ((rc = bidir_grid(idx->device, sh, grid))) return rc;
    if ((rc = dev_reserve(w.ctl, sizeof(SearchCtl) + 64))) return rc;
    if ((rc = dev_reserve(w.iv_cnt, std::max<uint64_t>(n, 1) * 4))) return rc;
    w.iv_cap = (uint32_t)std::max<uint64_t>(w.iv_cap, std::min<uint64_t>(4 * n + 65536, 1ull << 30));
    if ((rc = dev_reserve(w.iv, (size_t)w.iv_cap * sizeof(Interval)))) return rc;
    const uint64_t warps = (uint64_t)grid * sh.warps;
    if ((rc = dev_reserve(w.deep, (size_t)warps * bidir_deep_cap(w, warps) * 32))) return rc;
    // given-up reads: a bit per read, then a list of them and its length
    if ((rc = dev_reserve(w.redo, redo_bytes(n)))) return rc;
    // exported nodes: two rounds' buffers of (task, l, lr, sz) and meta
    if ((rc = dev_reserve(w.frontier, 2 * frontier_cap(n) * 20))) return rc;
    tmpl = SearchCtl{};
    tmpl.ntasks = 2 * n;
    tmpl.iv_cap = w.iv_cap;
    return 0;
}

static void bidir_args(const mica_index *idx, Workspace &w, const ReadsView &rd, int grid, BidirArgs &ba)
{
    const BidirShape &sh = g_bd_shapes[bidir_shape_index(idx)];
    ba.ix = idx->view;
    ba.fwd.occ = idx->view.occ;
    ba.fwd.super = idx->view.super;
    ba.fwd.dollar_row = idx->view.dollar_row;
    ba.rev.occ = idx->view.rev.occ;
    ba.rev.super = idx->view.rev.super;
    ba.rev.dollar_row = idx->view.rev.dollar_row;
    for (int c = 0; c < 5; c++) {
        ba.fwd.C[c] = idx->view.C[c];
        ba.rev.C[c] = idx->view.rev.C[c];
    }
    ba.rd = rd;
    ba.ctl = (SearchCtl *)w.ctl.p;
    ba.iv = (Interval *)w.iv.p;
    ba.iv_cnt = (uint32_t *)w.iv_cnt.p;
    ba.deep_cap = w.bd_deep_cap;
    ba.deep_m = (uint4 *)w.deep.p;
    ba.deep_s = (uint4 *)((char *)w.deep.p + (size_t)grid * sh.warps * w.bd_deep_cap * 16);
    ba.redo = (uint32_t *)w.redo.p;
    ba.budget = idx->tuning.bidir_budget ? idx->tuning.bidir_budget : BD_BUDGET;
    ba.fr_cap = frontier_cap(rd.n);
    const uint32_t vmin = idx->tuning.bidir_verify ? idx->tuning.bidir_verify : BD_VERIFY_MIN;
    ba.verify_min = (idx->view.sa_full && vmin < 256) ? vmin : 0u;
}

// Frontier buffer b (0 or 1): items, then meta words.
static uint4 *frontier_items(Workspace &w, uint64_t n, int b)
{
    return (uint4 *)((char *)w.frontier.p + (size_t)b * frontier_cap(n) * 20);
}
static uint32_t *frontier_meta(Workspace &w, uint64_t n, int b)
{
    return (uint32_t *)(frontier_items(w, n, b) + frontier_cap(n));
}

// The kernel moves frontier items and overflow-stack entries as 16-byte
// vectors: refuse a launch whose buffers are not on 16-byte boundaries.
static int check_vector_alignment(const BidirArgs &ba)
{
    const void *ps[] = {ba.deep_m, ba.deep_s, ba.fr_in, ba.fr_out};
    for (const void *p : ps)
        if ((uintptr_t)p & 15) {
            set_last_cuda_error(cudaErrorMisalignedAddress, "bidirectional search buffer alignment", __FILE__,
                                __LINE__);
            return MICA_ECUDA;
        }
    return 0;
}

// Launch frontier round r >= 1 (its tasks: the nodes round r - 1 exported).
static int launch_round(const mica_index *idx, Workspace &w, const ReadsView &rd, int grid, int r, cudaStream_t s,
                        uint64_t &launches)
{
    const BidirShape &sh = g_bd_shapes[bidir_shape_index(idx)];
    BidirArgs ba;
    bidir_args(idx, w, rd, grid, ba);
    ba.mode = 1;
    ba.fr_in = frontier_items(w, rd.n, (r + 1) & 1);
    ba.fr_in_meta = frontier_meta(w, rd.n, (r + 1) & 1);
    ba.fr_out = frontier_items(w, rd.n, r & 1);
    ba.fr_out_meta = frontier_meta(w, rd.n, r & 1);
    if (int rc = check_vector_alignment(ba)) return rc;
    k_bd_round<<<1, 1, 0, s>>>(ba.ctl, ba.fr_cap);
    sh.fn<<<grid, sh.warps * 32, sh.smem, s>>>(ba);
    launches += 2;
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

// Enqueue one bidirectional search (control block from `tmpl_src`, which is
// pinned host memory when captured; zeroed per-read counters and give-up
// bits), then `rounds` frontier rounds, between the timing events.  No host
// reads, so it can be captured.
int enqueue_bidir(const mica_index *idx, Workspace &w, const ReadsView &rd, int grid, const SearchCtl *tmpl_src,
                  cudaStream_t s, uint64_t &launches, int rounds)
{
    const BidirShape &sh = g_bd_shapes[bidir_shape_index(idx)];
    SearchCtl *d_ctl = (SearchCtl *)w.ctl.p;
    MICA_CUDA_TRY(cudaMemcpyAsync(d_ctl, tmpl_src, sizeof(SearchCtl), cudaMemcpyHostToDevice, s));
    MICA_CUDA_TRY(cudaMemsetAsync(w.iv_cnt.p, 0, std::max<uint64_t>(rd.n, 1) * 4, s));
    MICA_CUDA_TRY(cudaMemsetAsync(w.redo.p, 0, redo_bits_bytes(rd.n), s));
    MICA_CUDA_TRY(record_event(w.kev[0], s));
    if (rd.n) {
        BidirArgs ba;
        bidir_args(idx, w, rd, grid, ba);
        ba.mode = 0;
        ba.fr_in = nullptr;
        ba.fr_in_meta = nullptr;
        ba.fr_out = frontier_items(w, rd.n, 0);
        ba.fr_out_meta = frontier_meta(w, rd.n, 0);
        if (int rc = check_vector_alignment(ba)) return rc;
        sh.fn<<<grid, sh.warps * 32, sh.smem, s>>>(ba);
        launches++;
        MICA_CUDA_TRY(cudaGetLastError());
        for (int r = 1; r <= rounds; r++)
            if (int rc = launch_round(idx, w, rd, grid, r, s, launches)) return rc;
    }
    MICA_CUDA_TRY(record_event(w.kev[1], s));
    return 0;
}

int enqueue_bidir_graph(const mica_index *idx, Workspace &w, const ReadsView &rd, int grid, const SearchCtl *tmpl_src,
                        cudaStream_t s, uint64_t &launches)
{
    return enqueue_bidir(idx, w, rd, grid, tmpl_src, s, launches, BD_GRAPH_ROUNDS);
}

// The reads the kernel gave up on: purge their leaves and search them again
// with the persistent kernel, appending to the interval buffer.
int redo_given_up(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd, const SearchCtl &out,
                  cudaStream_t s)
{
    const uint64_t n = rd.n;
    const uint32_t *bits = (const uint32_t *)w.redo.p;
    uint32_t *list = (uint32_t *)((char *)w.redo.p + redo_bits_bytes(n));
    unsigned int *n_list = (unsigned int *)(list + std::max<uint64_t>(n, 1));
    MICA_CUDA_TRY(cudaMemsetAsync(n_list, 0, 4, s));
    const uint64_t words = (n + 31) / 32;
    unsigned g = (unsigned)std::min<uint64_t>((words + 255) / 256, 152ull * 8);
    k_redo_collect<<<std::max(g, 1u), 256, 0, s>>>(bits, n, list, n_list, (uint32_t *)w.iv_cnt.p);
    SearchCtl *d_ctl = (SearchCtl *)w.ctl.p;
    unsigned gi = (unsigned)std::min<uint64_t>((std::max<uint64_t>(out.iv_count, 1) + 255) / 256, 152ull * 32);
    k_iv_purge<<<gi, 256, 0, s>>>((Interval *)w.iv.p, &d_ctl->iv_count, w.iv_cap, bits);
    st.launches += 2;
    MICA_CUDA_TRY(cudaGetLastError());
    uint32_t nl = 0;
    MICA_CUDA_TRY(cudaMemcpyAsync(&nl, n_list, 4, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    st.fallback_reads = nl;
    return run_search_list(idx, w, st, rd, list, nl, out.iv_count, idx->has_rev, s);
}

// The bidirectional search of a batch, growing the interval buffer when it
// overflows, then the reads it gave up on.  Returns BIDIR_FALLBACK when the
// persistent search of those reads overflows a buffer (the caller then runs
// the persistent search over the whole batch).
int run_search_bidir(const mica_index *idx, Workspace &w, mica_stats &st, const ReadsView &rd, cudaStream_t s)
{
    const uint64_t n = rd.n;
    for (int attempt = 0; attempt < 8; attempt++) {
        SearchCtl h{};
        int grid = 0;
        if (int rc = prepare_bidir(idx, w, n, h, grid)) return rc;
        if (int rc = enqueue_bidir(idx, w, rd, grid, &h, s, st.launches, 0)) return rc;
        SearchCtl out;
        MICA_CUDA_TRY(cudaMemcpyAsync(&out, w.ctl.p, sizeof(out), cudaMemcpyDeviceToHost, s));
        MICA_CUDA_TRY(cudaStreamSynchronize(s));
        // frontier rounds while the last one exported nodes (and nothing failed)
        int r = 1;
        // four rounds per host read of the control block (a round with
        // nothing exported to it returns at once)
        while (r <= BD_MAX_ROUNDS && out.fr_count && !out.error) {
            for (int q = 0; q < 4 && r <= BD_MAX_ROUNDS; q++, r++)
                if (int rc = launch_round(idx, w, rd, grid, r, s, st.launches)) return rc;
            MICA_CUDA_TRY(cudaMemcpyAsync(&out, w.ctl.p, sizeof(out), cudaMemcpyDeviceToHost, s));
            MICA_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (out.fr_count && !out.error) {
            // still exporting after the last round: those reads are given up
            k_bd_give_up_frontier<<<152, 256, 0, s>>>((SearchCtl *)w.ctl.p, frontier_items(w, n, (r - 1) & 1),
                                                      frontier_cap(n), (uint32_t *)w.redo.p);
            st.launches++;
            MICA_CUDA_TRY(cudaMemcpyAsync(&out, w.ctl.p, sizeof(out), cudaMemcpyDeviceToHost, s));
            MICA_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (out.error & ERR_TIMEOUT) return MICA_ETIMEOUT;
        if (out.error & ERR_IV_OVERFLOW) {
            st.retries++;
            w.iv_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(2ull * out.iv_count, 2ull * w.iv_cap),
                                                    0xfffffff0ull);
            continue;
        }
        if (out.error) return BIDIR_FALLBACK;
        st.tasks = 2 * n;
        st.seeds = out.seeds;
        st.nodes = out.nodes;
        st.rank_blocks = out.rank_blocks;
        st.intervals = out.iv_count;
        st.warp_rounds = out.rounds;
        st.lane_ops = out.lane_ops;
        st.overflow_moves = out.deep_moves;
        st.verified = out.verified;
        st.verify_bytes = out.verify_bytes;
        st.verify_sectors = out.verify_sectors;
        st.spills = out.spills + out.fr_count;   // nodes exported to later rounds
        st.grid_ctas = (uint64_t)grid;
        w.bd_redo_seen = out.redo_reads > 0 || r > BD_GRAPH_ROUNDS;
        if (out.redo_reads) {
            int rc = redo_given_up(idx, w, st, rd, out, s);
            if (rc) return rc;
        }
        MICA_CUDA_TRY(record_event(w.kev[1], s));   // the kernel time covers the re-search too
        return 0;
    }
    set_last_internal("bidirectional search: interval buffer growth did not converge");
    return MICA_EINTERNAL;
}

}  // namespace mica
