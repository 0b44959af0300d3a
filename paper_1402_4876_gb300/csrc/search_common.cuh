// Device helpers shared by the search and locate kernels: occurrence counts
// from one 64-byte block, interval extension, read patterns and seed lookups.
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

// Counts of C, G, T among the first `o` symbols (o <= 192) of the 12 BWT
// words a[0..11].  Words beyond the prefix may hold anything: they are masked.
// Two words share one popcount: the even-bit masks of word 2p and (shifted
// left by one) of word 2p+1 never overlap.
__device__ __forceinline__ void prefix_counts(const uint32_t (&a)[12], uint32_t o,
                                              uint32_t &nc, uint32_t &ng, uint32_t &nt)
{
    uint32_t sc = 0, sg = 0, st = 0;
#pragma unroll
    for (int p = 0; p < 6; p++) {
        int rem0 = (int)o - 32 * p, rem1 = rem0 - 16;
        uint32_t m0 = rem0 >= 16 ? 0x55555555u : (rem0 <= 0 ? 0u : (0x55555555u >> (32 - 2 * rem0)));
        uint32_t m1 = rem1 >= 16 ? 0x55555555u : (rem1 <= 0 ? 0u : (0x55555555u >> (32 - 2 * rem1)));
        uint32_t x0 = a[2 * p], x1 = a[2 * p + 1];
        uint32_t lo0 = x0 & m0, hi0 = (x0 >> 1) & m0;
        uint32_t lo1 = x1 & m1, hi1 = (x1 >> 1) & m1;
        uint32_t lo = lo0 | (lo1 << 1), hi = hi0 | (hi1 << 1);
        uint32_t both = (lo0 & hi0) | ((lo1 & hi1) << 1);
        st += __popc(both);
        sc += __popc(lo);
        sg += __popc(hi);
    }
    nt = st;
    nc = sc - st;   // code 1 = low bit only
    ng = sg - st;   // code 2 = high bit only
}

// Load the words of block `blk` needed for the first `need` symbols.
__device__ __forceinline__ void load_block_words(const uint4 *blk, uint32_t need, uint32_t (&a)[12])
{
    uint4 w0 = make_uint4(0, 0, 0, 0), w1 = w0, w2 = w0;
    if (need > 0) w0 = ld_nc(blk + 1);
    if (need > 64) w1 = ld_nc(blk + 2);
    if (need > 128) w2 = ld_nc(blk + 3);
    a[0] = w0.x; a[1] = w0.y; a[2] = w0.z; a[3] = w0.w;
    a[4] = w1.x; a[5] = w1.y; a[6] = w1.z; a[7] = w1.w;
    a[8] = w2.x; a[9] = w2.y; a[10] = w2.z; a[11] = w2.w;
}

// Occ(A..T, i) into occ[0..3] from a header and already-loaded words.
__device__ __forceinline__ void occ_from(const IndexView &ix, uint32_t b, uint32_t o, const uint4 &h,
                                         const uint32_t (&a)[12], uint32_t (&occ)[4])
{
    uint32_t nc, ng, nt;
    prefix_counts(a, o, nc, ng, nt);
    uint32_t na = o - nc - ng - nt;
    uint32_t start = b * OCC_ROWS;
    if (ix.dollar_row >= start && ix.dollar_row < start + o) na -= 1;   // $ is stored as A
    occ[0] = h.x + na;
    occ[1] = h.y + nc;
    occ[2] = h.z + ng;
    occ[3] = h.w + nt;
}

// Occ(c, l) and Occ(c, r) for all c; one block read when l and r share it.
// Returns the number of 64-byte blocks touched (1 or 2).
__device__ __forceinline__ int occ_pair(const IndexView &ix, uint32_t l, uint32_t r,
                                        uint32_t (&ol)[4], uint32_t (&orr)[4])
{
    uint32_t bl = l / OCC_ROWS, xl = l - bl * OCC_ROWS;
    uint32_t br = r / OCC_ROWS, xr = r - br * OCC_ROWS;
    const uint4 *pl = ix.occ + (size_t)bl * 4;
    uint32_t a[12];
    if (bl == br) {
        uint4 h = ld_nc(pl);
        load_block_words(pl, xr, a);
        occ_from(ix, bl, xl, h, a, ol);
        occ_from(ix, br, xr, h, a, orr);
        return 1;
    }
    const uint4 *pr = ix.occ + (size_t)br * 4;
    uint4 hl = ld_nc(pl), hr = ld_nc(pr);
    uint32_t b2[12];
    load_block_words(pl, xl, a);
    load_block_words(pr, xr, b2);
    occ_from(ix, bl, xl, hl, a, ol);
    occ_from(ix, br, xr, hr, b2, orr);
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
    for (uint32_t t = 0; t < ix.nshort; t++) {
        l -= (ix.short_pad[t] == start && ix.short_len[t] >= qe);
        r -= (ix.short_pad[t] == end);
    }
}

}  // namespace mica
