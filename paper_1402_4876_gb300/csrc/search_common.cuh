// Device helpers shared by the search and locate kernels: occurrence counts
// from one 32-byte block, interval extension, read patterns and seed lookups.
#pragma once

#include "mica_internal.cuh"

namespace mica {

// V(q', k): ways to substitute at most k of q' bases (each by one of 3).
__device__ __forceinline__ uint32_t n_variants(uint32_t q, uint32_t k)
{
    uint32_t v = 1;
    if (k >= 1) v += 3 * q;
    if (k >= 2) v += 9 * (q * (q - 1) / 2);
    if (k >= 3) v += 27 * (q * (q - 1) * (q - 2) / 6);
    return v;
}

__device__ __forceinline__ uint4 ld_nc(const uint4 *p) { return __ldg(p); }

// Low `rem` bits set, rem in [0, 32].
__device__ __forceinline__ uint32_t low_mask(uint32_t rem)
{
    return ~__funnelshift_lc(0u, 0xffffffffu, rem);
}

// One occurrence block in registers: relative counts and the bit planes.
struct OccBlock {
    uint32_t ac, gt;          // relative counts A | C << 16, G | T << 16
    uint32_t lo[3], hi[3];    // rows 0-31, 32-63, 64-95
};

// Load block b; rows at offsets >= 32 are only fetched when `need` > 32.
__device__ __forceinline__ void load_block(const IndexView &ix, uint32_t b, uint32_t need, OccBlock &k)
{
    const uint4 *p = ix.occ + (size_t)b * 2;
    uint4 q0 = ld_nc(p);
    uint4 q1 = make_uint4(0, 0, 0, 0);
    if (need > 32) q1 = ld_nc(p + 1);
    k.ac = q0.x; k.gt = q0.y;
    k.lo[0] = q0.z; k.hi[0] = q0.w;
    k.lo[1] = q1.x; k.hi[1] = q1.y;
    k.lo[2] = q1.z; k.hi[2] = q1.w;
}

// Occ(A..T, b * 96 + o) from a loaded block and its superblock entry.
__device__ __forceinline__ void occ_from(const IndexView &ix, uint32_t b, uint32_t o, const uint4 &sup,
                                         const OccBlock &k, uint32_t (&occ)[4])
{
    uint32_t sl = 0, sh = 0, st = 0;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint32_t rem = min(max((int)o - 32 * j, 0), 32);
        uint32_t m = low_mask(rem);
        uint32_t L = k.lo[j] & m, H = k.hi[j] & m;
        st += __popc(L & H);
        sl += __popc(L);
        sh += __popc(H);
    }
    uint32_t nt = st, nc = sl - st, ng = sh - st;
    uint32_t na = o - nc - ng - nt;
    uint32_t start = b * OCC_ROWS;
    if (ix.dollar_row >= start && ix.dollar_row < start + o) na -= 1;   // $ is stored as A
    occ[0] = sup.x + (k.ac & 0xffffu) + na;
    occ[1] = sup.y + (k.ac >> 16) + nc;
    occ[2] = sup.z + (k.gt & 0xffffu) + ng;
    occ[3] = sup.w + (k.gt >> 16) + nt;
}

// Occ(c, b * 96 + o) for one symbol c.
__device__ __forceinline__ uint32_t occ_single(const IndexView &ix, uint32_t b, uint32_t o, const uint4 &sup,
                                               const OccBlock &k, uint32_t c)
{
    uint32_t xl = (c & 1u) ? 0u : 0xffffffffu;   // select rows whose low bit equals c's
    uint32_t xh = (c & 2u) ? 0u : 0xffffffffu;
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint32_t rem = min(max((int)o - 32 * j, 0), 32);
        n += __popc((k.lo[j] ^ xl) & (k.hi[j] ^ xh) & low_mask(rem));
    }
    uint32_t start = b * OCC_ROWS;
    if (c == 0 && ix.dollar_row >= start && ix.dollar_row < start + o) n -= 1;   // $ is stored as A
    uint32_t rel = c == 0 ? (k.ac & 0xffffu) : c == 1 ? (k.ac >> 16) : c == 2 ? (k.gt & 0xffffu) : (k.gt >> 16);
    uint32_t base = c == 0 ? sup.x : c == 1 ? sup.y : c == 2 ? sup.z : sup.w;
    return base + rel + n;
}

__device__ __forceinline__ uint32_t C_of(const IndexView &ix, uint32_t c)
{
    return c == 0 ? ix.C[0] : c == 1 ? ix.C[1] : c == 2 ? ix.C[2] : ix.C[3];
}

// Symbol code at offset o of a loaded block.
__device__ __forceinline__ uint32_t block_symbol(const OccBlock &k, uint32_t o)
{
    uint32_t j = o >> 5, bit = o & 31;
    uint32_t lo = j == 0 ? k.lo[0] : j == 1 ? k.lo[1] : k.lo[2];
    uint32_t hi = j == 0 ? k.hi[0] : j == 1 ? k.hi[1] : k.hi[2];
    return ((lo >> bit) & 1u) | (((hi >> bit) & 1u) << 1);
}

// Occ(c, l) and Occ(c, r) for all c; one block read when l and r share it.
// Returns the number of 32-byte blocks touched (1 or 2).
__device__ __forceinline__ int occ_pair(const IndexView &ix, uint32_t l, uint32_t r,
                                        uint32_t (&ol)[4], uint32_t (&orr)[4])
{
    uint32_t bl = l / OCC_ROWS, xl = l - bl * OCC_ROWS;
    uint32_t br = r / OCC_ROWS, xr = r - br * OCC_ROWS;
    uint4 sl = ld_nc(ix.super + bl / SB_BLOCKS);
    OccBlock a;
    if (bl == br) {
        load_block(ix, bl, xr, a);
        occ_from(ix, bl, xl, sl, a, ol);
        occ_from(ix, br, xr, sl, a, orr);
        return 1;
    }
    uint4 sr = ld_nc(ix.super + br / SB_BLOCKS);
    OccBlock c;
    load_block(ix, bl, xl, a);
    load_block(ix, br, xr, c);
    occ_from(ix, bl, xl, sl, a, ol);
    occ_from(ix, br, xr, sr, c, orr);
    return 2;
}

// One of the two indices of a bidirectional search (the genome's, or the
// reversed genome's): its occurrence blocks, superblocks, $ row and C[].
struct OccSide {
    const uint4 *occ;
    const uint4 *super;
    uint32_t dollar_row;
    uint32_t C[5];
};

__device__ __forceinline__ void load_block(const OccSide &ix, uint32_t b, uint32_t need, OccBlock &k)
{
    const uint4 *p = ix.occ + (size_t)b * 2;
    uint4 q0 = ld_nc(p);
    uint4 q1 = make_uint4(0, 0, 0, 0);
    if (need > 32) q1 = ld_nc(p + 1);
    k.ac = q0.x; k.gt = q0.y;
    k.lo[0] = q0.z; k.hi[0] = q0.w;
    k.lo[1] = q1.x; k.hi[1] = q1.y;
    k.lo[2] = q1.z; k.hi[2] = q1.w;
}

// Occ(A..T, b * 96 + o) on one side ($ excluded from A).
__device__ __forceinline__ void occ_from(const OccSide &ix, uint32_t b, uint32_t o, const uint4 &sup,
                                         const OccBlock &k, uint32_t (&occ)[4])
{
    uint32_t sl = 0, sh = 0, st = 0;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint32_t rem = min(max((int)o - 32 * j, 0), 32);
        uint32_t m = low_mask(rem);
        uint32_t L = k.lo[j] & m, H = k.hi[j] & m;
        st += __popc(L & H);
        sl += __popc(L);
        sh += __popc(H);
    }
    uint32_t nt = st, nc = sl - st, ng = sh - st;
    uint32_t na = o - nc - ng - nt;
    uint32_t start = b * OCC_ROWS;
    if (ix.dollar_row >= start && ix.dollar_row < start + o) na -= 1;
    occ[0] = sup.x + (k.ac & 0xffffu) + na;
    occ[1] = sup.y + (k.ac >> 16) + nc;
    occ[2] = sup.z + (k.gt & 0xffffu) + ng;
    occ[3] = sup.w + (k.gt >> 16) + nt;
}

// Occ(c, l) and Occ(c, r) for all c on one side; returns the blocks read.
__device__ __forceinline__ int occ_pair(const OccSide &ix, uint32_t l, uint32_t r, uint32_t (&ol)[4],
                                        uint32_t (&orr)[4])
{
    uint32_t bl = l / OCC_ROWS, xl = l - bl * OCC_ROWS;
    uint32_t br = r / OCC_ROWS, xr = r - br * OCC_ROWS;
    uint4 sl = ld_nc(ix.super + bl / SB_BLOCKS);
    OccBlock a;
    if (bl == br) {
        load_block(ix, bl, xr, a);
        occ_from(ix, bl, xl, sl, a, ol);
        occ_from(ix, br, xr, sl, a, orr);
        return 1;
    }
    uint4 sr = ld_nc(ix.super + br / SB_BLOCKS);
    OccBlock c;
    load_block(ix, bl, xl, a);
    load_block(ix, br, xr, c);
    occ_from(ix, bl, xl, sl, a, ol);
    occ_from(ix, br, xr, sr, c, orr);
    return 2;
}

// Base t of a packed pattern.
__device__ __forceinline__ uint32_t pat_base(const uint32_t *pat, uint32_t t)
{
    return (pat[t >> 4] >> (2 * (t & 15))) & 3u;
}

// Reverse the order of the 16 two-bit groups of a word.
__device__ __forceinline__ uint32_t rev_groups(uint32_t x)
{
    x = __brev(x);
    return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}

// Word j of the reverse complement of a read of m bases held in W words,
// given raw words hi = raw[W-1-j] and lo = raw[W-2-j] (0 when out of range).
__device__ __forceinline__ uint32_t rc_word(uint32_t hi, uint32_t lo, uint32_t m)
{
    uint32_t W = (m + 15) >> 4;
    uint32_t sh = 2 * (16 * W - m);          // pad bits above the read in the last word
    uint32_t a = ~rev_groups(hi), b = ~rev_groups(lo);
    return sh ? (a >> sh) | (b << (32 - sh)) : a;
}

// q-mer code of pattern bases [m - qe, m), first base most significant.
__device__ __forceinline__ uint32_t window_code(const uint32_t *pat, uint32_t m, uint32_t qe)
{
    uint32_t code = 0;
    for (uint32_t t = m - qe; t < m; t++) code = (code << 2) | pat_base(pat, t);
    return code;
}

// SA interval of a (qe)-mer code x from a q-mer table (the genome's or the
// reversed genome's) with its short-suffix corrections.
__device__ __forceinline__ void seed_interval_in(const uint32_t *table, uint32_t q, uint32_t nshort,
                                                 const uint32_t *short_pad, const uint32_t *short_len,
                                                 unsigned long long bloom, uint32_t code, uint32_t qe,
                                                 uint32_t &l, uint32_t &r)
{
    uint32_t sh = 2 * (q - qe);
    uint32_t start = code << sh, end = (code + 1) << sh;
    l = __ldg(table + (size_t)start);
    r = __ldg(table + (size_t)end);
    if (((bloom >> (start & 63)) | (bloom >> (end & 63))) & 1ull) {
        for (uint32_t t = 0; t < nshort; t++) {
            l -= (short_pad[t] == start && short_len[t] >= qe);
            r -= (short_pad[t] == end);
        }
    }
}

// SA interval of a (qe)-mer code x from the q-mer table, whose entry at a
// q-mer y is the number of suffixes smaller than y:
//   l = bound[x * 4^(q-qe)]     - #{short u$ padded to that start, |u| >= qe},
//   r = bound[(x+1) * 4^(q-qe)] - #{short u$ padded to that end}.
__device__ __forceinline__ void seed_interval(const IndexView &ix, uint32_t code, uint32_t qe,
                                              uint32_t &l, uint32_t &r)
{
    uint32_t sh = 2 * (ix.q - qe);
    uint32_t start = code << sh, end = (code + 1) << sh;
    l = __ldg(ix.table + (size_t)start);
    r = __ldg(ix.table + (size_t)end);
    if (((ix.short_bloom >> (start & 63)) | (ix.short_bloom >> (end & 63))) & 1ull) {
        for (uint32_t t = 0; t < ix.nshort; t++) {
            l -= (ix.short_pad[t] == start && ix.short_len[t] >= qe);
            r -= (ix.short_pad[t] == end);
        }
    }
}

}  // namespace mica
