// From leaf SA intervals to per-read hit lists:
//   1. group the intervals by read (prefix sum of per-read counts + scatter);
//   2. per read: order the intervals by (d, strand, first row), total = sum of
//      interval sizes (exact), keep = min(total, cap) rows in that order;
//   3. prefix sum of keep -> CSR offsets; expand the kept rows;
//   4. resolve each row to a text position by LF walks to the nearest marked
//      row (SA[j] % s == 0), whose SA value is stored:
//          SA[j] = SA[LF^t(j)] + t,   LF(j) = C[BWT[j]] + Occ(BWT[j], j);
//   5. sort each read's hits by (position, strand).
#include <algorithm>
#include <vector>

#include "search_common.cuh"

namespace mica {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr uint32_t SMALL_SORT = 32;
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t SMEM_SORT = 4096;
constexpr uint32_t WARP_SORT = 256;            // reads up to this many hits: one warp sorts each ...
constexpr uint32_t WARP_SORT_WARPS = 8;        // ... 8 warps per block (2 KB of shared memory each);
constexpr uint32_t BLOCK_SORT_THREADS = 128;   // larger ones (up to SMEM_SORT): a block of 128 threads each

// ---- exclusive scan (n values -> n + 1 offsets) ----

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const T *__restrict__ in, uint64_t n,
                                                             uint64_t *__restrict__ out,
                                                             uint64_t *__restrict__ tile_sums)
{
    __shared__ uint64_t warp_sums[SCAN_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    uint64_t v[SCAN_ITEMS];
    uint64_t sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        v[j] = (base + j < n) ? (uint64_t)in[base + j] : 0ull;
        sum += v[j];
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    uint64_t woff = 0, total = 0;
    for (int w = 0; w < SCAN_THREADS / 32; w++) {
        if (w < warp) woff += warp_sums[w];
        total += warp_sums[w];
    }
    uint64_t run = woff + incl - sum;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// one block: exclusive scan of the tile sums, grand total at [ntiles]
__global__ void __launch_bounds__(1024) k_scan_sums(uint64_t *__restrict__ s, uint64_t ntiles)
{
    __shared__ uint64_t warp_sums[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t b0 = 0; b0 < ntiles; b0 += 1024) {
        uint64_t i = b0 + threadIdx.x;
        uint64_t x = i < ntiles ? s[i] : 0;
        uint64_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        uint64_t woff = 0, tot = 0;
        for (int w = 0; w < 32; w++) {
            if (w < warp) woff += warp_sums[w];
            tot += warp_sums[w];
        }
        uint64_t c = carry;
        if (i < ntiles) s[i] = c + woff + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) s[ntiles] = carry;
}

__global__ void k_scan_add(uint64_t *__restrict__ out, uint64_t n, const uint64_t *__restrict__ tile_sums)
{
    uint64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] += tile_sums[i / SCAN_TILE];
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_sums[ntiles];
}

template <typename T>
int exclusive_scan(DevBuf &tmp, const T *in, uint64_t n, uint64_t *out, cudaStream_t s, uint64_t &launches)
{
    uint64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (int rc = dev_reserve(tmp, (ntiles + 1) * 8)) return rc;
    uint64_t *ts = (uint64_t *)tmp.p;
    if (ntiles) { k_scan_tiles<T><<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(in, n, out, ts); launches++; }
    k_scan_sums<<<1, 1024, 0, s>>>(ts, ntiles);
    unsigned g = (unsigned)std::min<uint64_t>(std::max<uint64_t>((n + 255) / 256, 1), 152 * 32);
    k_scan_add<<<g, 256, 0, s>>>(out, n, ts);
    launches += 2;
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

// ---- intervals grouped by read ----

// Every post kernel that indexes by the search's per-read counts first reads
// the search's error word: after an overflow the counts exceed what was
// stored, so these kernels do nothing and the caller recomputes the batch.
//
// count: the search's interval counter on the device, read here (capped at
// the buffer's capacity) so the launch needs no host round trip
__global__ void k_iv_scatter(const Interval *__restrict__ iv, const unsigned int *__restrict__ count_p,
                             uint32_t cap, const uint64_t *__restrict__ iv_off, uint32_t *__restrict__ cursor,
                             Interval *__restrict__ out, const unsigned int *__restrict__ err)
{
    if (*err) return;
    uint32_t count = min(*count_p, cap);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        Interval x = iv[e];
        if (x.read == IV_PURGED) continue;   // a leaf of a read that was searched again
        uint32_t at = atomicSub(&cursor[x.read], 1u) - 1u;
        out[iv_off[x.read] + at] = x;
    }
}

__device__ __forceinline__ uint64_t iv_key(const Interval &x)
{
    return ((uint64_t)(x.meta & 3u) << 33) | ((uint64_t)((x.meta >> 2) & 1u) << 32) | x.l;
}

// Best-stratum reporting: a read keeps only its intervals with the smallest
// d; the others become empty (r = l) and so count and list nothing.
__global__ void k_stratum(Interval *__restrict__ ivs, const uint64_t *__restrict__ iv_off, uint64_t n,
                          const unsigned int *__restrict__ err)
{
    if (*err) return;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t b = iv_off[r], e = iv_off[r + 1];
        uint32_t dmin = 3;
        for (uint64_t i = b; i < e; i++) dmin = min(dmin, ivs[i].meta & 3u);
        for (uint64_t i = b; i < e; i++)
            if ((ivs[i].meta & 3u) > dmin) ivs[i].r = ivs[i].l;
    }
}

// Per read: total = the sum of its interval sizes (exact) and keep = the
// rows it lists, min(total, cap).  When total > cap the listed rows are the
// first cap in the order (d, strand, SA row); k_expand takes rows from the
// front of the read's interval list until it has `keep`, so that list must
// start with the kept rows.  A read with at most SUMMARY_SMALL intervals is
// done here by one thread (insertion sort into key order when over the cap);
// a longer list goes to `many` for k_summarize_many.
constexpr uint32_t SUMMARY_SMALL = 32;

__global__ void k_summarize(Interval *__restrict__ ivs, const uint64_t *__restrict__ iv_off, uint64_t n,
                            uint32_t cap, uint64_t *__restrict__ total, uint64_t *__restrict__ keep,
                            uint32_t *__restrict__ many, unsigned int *__restrict__ n_many,
                            const unsigned int *__restrict__ err)
{
    if (*err) return;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t b = iv_off[r], e = iv_off[r + 1];
        if (e - b > SUMMARY_SMALL) {
            many[atomicAdd(n_many, 1u)] = (uint32_t)r;
            continue;
        }
        uint64_t t = 0;
        for (uint64_t i = b; i < e; i++) t += ivs[i].r - ivs[i].l;
        if (cap && t > cap) {
            for (uint64_t i = b + 1; i < e; i++) {
                Interval x = ivs[i];
                uint64_t kx = iv_key(x);
                uint64_t j = i;
                while (j > b && iv_key(ivs[j - 1]) > kx) { ivs[j] = ivs[j - 1]; j--; }
                ivs[j] = x;
            }
        }
        total[r] = t;
        keep[r] = (cap && t > cap) ? cap : t;
    }
}

// Block-wide sum of one value per thread (blockDim.x = MANY_THREADS).
constexpr int MANY_THREADS = 256;

__device__ __forceinline__ uint64_t block_sum(uint64_t v, uint64_t *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    __syncthreads();                       // red[] free from the previous use
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    uint64_t s = 0;
    for (int w = 0; w < MANY_THREADS / 32; w++) s += red[w];
    return s;
}

// One block per read with more than SUMMARY_SMALL intervals.  The rows a
// capped read lists are found without sorting: interval keys (d, strand, l)
// are distinct, so a bitwise search from the top key bit finds the key K at
// which the running row count in key order first reaches cap (35 passes,
// each a block-wide sum of the sizes below the candidate prefix).  Intervals
// with key < K are kept whole, K's interval keeps its first cap - before
// rows, and the kept ones are compacted to the front of the read's list in
// chunks of the block size (each chunk read before any of it is overwritten;
// writes never pass the chunk being read).
__global__ void __launch_bounds__(MANY_THREADS) k_summarize_many(Interval *__restrict__ ivs,
                                                                 const uint64_t *__restrict__ iv_off,
                                                                 uint32_t cap, uint64_t *__restrict__ total,
                                                                 uint64_t *__restrict__ keep,
                                                                 const uint32_t *__restrict__ many,
                                                                 const unsigned int *__restrict__ n_many_p,
                                                                 const unsigned int *__restrict__ err)
{
    if (*err) return;
    __shared__ uint64_t red[MANY_THREADS / 32];
    __shared__ uint32_t wsum[MANY_THREADS / 32];
    const unsigned n_many = *n_many_p;
    for (unsigned mi = blockIdx.x; mi < n_many; mi += gridDim.x) {
        const uint32_t r = many[mi];
        const uint64_t b = iv_off[r], e = iv_off[r + 1];
        uint64_t part = 0;
        for (uint64_t i = b + threadIdx.x; i < e; i += MANY_THREADS) part += ivs[i].r - ivs[i].l;
        const uint64_t t = block_sum(part, red);
        if (threadIdx.x == 0) {
            total[r] = t;
            keep[r] = (cap && t > cap) ? cap : t;
        }
        if (!(cap && t > cap)) continue;
        // bitwise search for K over the 35-bit keys
        uint64_t prefix = 0, before = 0;
        for (int bit = 34; bit >= 0; bit--) {
            const uint64_t hi = prefix >> (bit + 1);
            uint64_t z = 0;
            for (uint64_t i = b + threadIdx.x; i < e; i += MANY_THREADS) {
                Interval x = ivs[i];
                uint64_t k = iv_key(x);
                if ((k >> (bit + 1)) == hi && !((k >> bit) & 1u)) z += x.r - x.l;
            }
            z = block_sum(z, red);
            if (before + z < cap) { before += z; prefix |= 1ull << bit; }
        }
        const uint64_t K = prefix;
        const uint32_t take = (uint32_t)(cap - before);   // rows of K's interval, 1 .. its size
        // compact the kept intervals to the front
        uint64_t out = b;
        for (uint64_t c0 = b; c0 < e; c0 += MANY_THREADS) {
            uint64_t i = c0 + threadIdx.x;
            Interval x{};
            bool kept = false;
            if (i < e) {
                x = ivs[i];
                uint64_t k = iv_key(x);
                kept = k <= K;
                if (k == K) x.r = x.l + take;
            }
            unsigned bal = __ballot_sync(FULL, kept);
            __syncthreads();                 // every read of this chunk is done
            if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(bal);
            __syncthreads();
            uint32_t pre = 0, all = 0;
            for (int w = 0; w < MANY_THREADS / 32; w++) {
                if (w < (int)(threadIdx.x >> 5)) pre += wsum[w];
                all += wsum[w];
            }
            pre += __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
            if (kept) ivs[out + pre] = x;
            out += all;
            __syncthreads();                 // writes done before the next chunk is read
        }
    }
}

__global__ void k_expand(const Interval *__restrict__ ivs, const uint64_t *__restrict__ iv_off,
                         const uint64_t *__restrict__ hit_off, uint64_t n, Hit *__restrict__ hits,
                         uint64_t capacity, const unsigned int *__restrict__ err)
{
    if (*err) return;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t q = hit_off[r], qe = min(hit_off[r + 1], capacity);
        for (uint64_t i = iv_off[r]; i < iv_off[r + 1] && q < qe; i++) {
            Interval x = ivs[i];
            for (uint32_t row = x.l; row < x.r && q < qe; row++, q++) {
                Hit h;
                h.pos = row;   // resolved to a position by k_locate
                h.strand = (uint8_t)((x.meta >> 2) & 1u);
                h.mm = (uint8_t)(x.meta & 3u);
                h.pad = 0;
                hits[q] = h;
            }
        }
    }
}

}  // namespace

// ---- locate: SA[j] by LF walks to a marked row ----

__device__ __forceinline__ uint32_t locate_row(const IndexView &ix, uint32_t j, uint32_t &steps)
{
    uint32_t t = 0;
    for (;;) {
        uint32_t mb = j / MARK_ROWS, mo = j - mb * MARK_ROWS;
        const uint4 *mp = ix.marks + (size_t)mb * 4;
        uint4 q0 = __ldg(mp), q1 = __ldg(mp + 1), q2 = __ldg(mp + 2), q3 = __ldg(mp + 3);
        uint32_t w[16] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                          q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
        uint32_t wi = mo >> 5, bi = mo & 31;
        uint32_t word = 0, before = 0;
#pragma unroll
        for (int x = 0; x < 15; x++) {
            if ((uint32_t)x < wi) before += __popc(w[1 + x]);
            if ((uint32_t)x == wi) word = w[1 + x];
        }
        if ((word >> bi) & 1u) {
            uint32_t rank = w[0] + before + __popc(word & ((1u << bi) - 1u));
            steps += t;
            return __ldg(ix.samples + rank) + t;
        }
        // LF step: c = BWT[j] (never $: the $ row has SA = 0, which is marked)
        uint32_t b = j / OCC_ROWS, o = j - b * OCC_ROWS;
        uint4 sup = __ldg(ix.super + b / SB_BLOCKS);
        OccBlock k;
        load_block(ix, b, o + 1, k);
        uint32_t c = block_symbol(k, o);
        uint32_t occ[4];
        occ_from(ix, b, o, sup, k, occ);
        uint32_t oc = c == 0 ? occ[0] : c == 1 ? occ[1] : c == 2 ? occ[2] : occ[3];
        uint32_t Cc = c == 0 ? ix.C[0] : c == 1 ? ix.C[1] : c == 2 ? ix.C[2] : ix.C[3];
        j = Cc + oc;
        t++;
    }
}

namespace {

__global__ void k_locate(const IndexView ix, Hit *__restrict__ hits, const uint64_t *__restrict__ nh_p,
                         uint64_t capacity, unsigned long long *__restrict__ steps_out,
                         const unsigned int *__restrict__ err)
{
    if (*err) return;   // hits not expanded: rows would be stale
    uint64_t nh = min(*nh_p, capacity);
    uint32_t steps = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nh;
         i += (uint64_t)gridDim.x * blockDim.x) {
        hits[i].pos = ix.sa_full ? __ldg(ix.sa_full + hits[i].pos) : locate_row(ix, hits[i].pos, steps);
    }
    unsigned mask = __activemask();
    unsigned s = __reduce_add_sync(mask, steps);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1) && s) atomicAdd(steps_out, (unsigned long long)s);
}

__device__ __forceinline__ uint64_t hit_key(uint64_t raw)
{
    return ((raw & 0xffffffffull) << 1) | ((raw >> 32) & 1ull);   // (pos, strand)
}

// per read: sort <= SMALL_SORT hits in place; list larger reads for the
// block sort (from the front of `lists`) or the global sort (from the back)
__global__ void k_sort_small(uint64_t *__restrict__ hits, const uint64_t *__restrict__ hit_off, uint64_t n,
                             uint64_t capacity, uint32_t *__restrict__ lists, unsigned int *__restrict__ counts)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t b = hit_off[r], e = hit_off[r + 1];
        if (e - b <= 1 || e > capacity) continue;
        if (e - b > SMEM_SORT) {
            lists[n - 1 - atomicAdd(&counts[1], 1u)] = (uint32_t)r;
            continue;
        }
        if (e - b > SMALL_SORT) {
            lists[atomicAdd(&counts[0], 1u)] = (uint32_t)r;
            continue;
        }
        for (uint64_t i = b + 1; i < e; i++) {
            uint64_t x = hits[i], kx = hit_key(x);
            uint64_t j = i;
            while (j > b && hit_key(hits[j - 1]) > kx) { hits[j] = hits[j - 1]; j--; }
            hits[j] = x;
        }
    }
}

// Bitonic sort of the packed hits sh[0, P) (P a power of two, padding ~0 last)
// by (pos, strand), by the `nt` threads numbered `tid` of a warp (BLOCK false)
// or a block (true), which meet at a barrier between phases: log2(P) (log2(P)
// + 1) / 2 phases, each thread taking every nt-th compare-exchange pair
// (i, i ^ jj) with i's jj bit clear (the pairs of a phase are disjoint); a
// thread loads up to four pairs before it compares and stores any of them.
template <bool BLOCK>
__device__ __forceinline__ void bitonic_hits(uint64_t *sh, uint32_t P, uint32_t tid, uint32_t nt)
{
    for (uint32_t kk = 2; kk <= P; kk <<= 1)
        for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
            for (uint32_t t0 = tid; t0 < P / 2; t0 += 4 * nt) {
                uint32_t ii[4];
                uint64_t xs[4], ys[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t t = t0 + (uint32_t)u * nt;
                    ii[u] = ((t & ~(jj - 1)) << 1) | (t & (jj - 1));
                    if (t < P / 2) { xs[u] = sh[ii[u]]; ys[u] = sh[ii[u] ^ jj]; }
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t t = t0 + (uint32_t)u * nt;
                    if (t < P / 2) {
                        const uint64_t kx = xs[u] == ~0ull ? ~0ull : hit_key(xs[u]);
                        const uint64_t ky = ys[u] == ~0ull ? ~0ull : hit_key(ys[u]);
                        if ((kx > ky) == ((ii[u] & kk) == 0)) { sh[ii[u]] = ys[u]; sh[ii[u] ^ jj] = xs[u]; }
                    }
                }
            }
            if (BLOCK) __syncthreads(); else __syncwarp();
        }
}

// Reads with SMALL_SORT < hits <= WARP_SORT: one warp each, taken from the
// listed reads by a counter (reads differ a lot in size: a fixed stride left
// one warp with the largest); larger listed reads are left to k_sort_block.
__global__ void __launch_bounds__(WARP_SORT_WARPS * 32) k_sort_warp(uint64_t *__restrict__ hits,
                                                                    const uint64_t *__restrict__ hit_off,
                                                                    const uint32_t *__restrict__ big,
                                                                    const unsigned int *__restrict__ nbig_p,
                                                                    unsigned int *__restrict__ next)
{
    __shared__ uint64_t shw[WARP_SORT_WARPS][WARP_SORT];
    const unsigned lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    uint64_t *sh = shw[wi];
    const unsigned nbig = *nbig_p;
    for (;;) {
        unsigned bi = 0;
        if (lane == 0) bi = atomicAdd(next, 1u);
        bi = __shfl_sync(0xffffffffu, bi, 0);
        if (bi >= nbig) break;
        const uint32_t r = big[bi];
        const uint64_t b = hit_off[r], cnt = hit_off[r + 1] - b;
        if (cnt > WARP_SORT) continue;
        uint32_t P = 1;
        while (P < cnt) P <<= 1;
        // the packed hits themselves (below 2^48), padded with ~0, ordered by (pos, strand)
        for (uint32_t i = lane; i < P; i += 32) sh[i] = i < cnt ? hits[b + i] : ~0ull;
        __syncwarp();
        bitonic_hits<false>(sh, P, lane, 32);
        for (uint32_t i = lane; i < cnt; i += 32) hits[b + i] = sh[i];
        __syncwarp();
    }
}

// Reads with WARP_SORT < hits <= SMEM_SORT: one block of 128 threads each,
// taken by a counter.
__global__ void __launch_bounds__(BLOCK_SORT_THREADS) k_sort_block(uint64_t *__restrict__ hits,
                                                                   const uint64_t *__restrict__ hit_off,
                                                                   const uint32_t *__restrict__ big,
                                                                   const unsigned int *__restrict__ nbig_p,
                                                                   unsigned int *__restrict__ next)
{
    __shared__ uint64_t sh[SMEM_SORT];
    __shared__ unsigned bi_s;
    const unsigned nbig = *nbig_p;
    for (;;) {
        if (threadIdx.x == 0) bi_s = atomicAdd(next, 1u);
        __syncthreads();
        const unsigned bi = bi_s;
        __syncthreads();
        if (bi >= nbig) break;
        const uint32_t r = big[bi];
        const uint64_t b = hit_off[r], cnt = hit_off[r + 1] - b;
        if (cnt <= WARP_SORT) continue;
        uint32_t P = 1;
        while (P < cnt) P <<= 1;
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < cnt ? hits[b + i] : ~0ull;
        __syncthreads();
        bitonic_hits<true>(sh, P, threadIdx.x, blockDim.x);
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) hits[b + i] = sh[i];
        __syncthreads();
    }
}

// one read with more than SMEM_SORT hits: bitonic network over a global scratch
__global__ void __launch_bounds__(1024) k_sort_global(uint64_t *__restrict__ hits, uint64_t cnt,
                                                      uint64_t *__restrict__ scratch, uint64_t P)
{
    for (uint64_t i = threadIdx.x; i < P; i += blockDim.x) scratch[i] = i < cnt ? hits[i] : ~0ull;
    __syncthreads();
    for (uint64_t kk = 2; kk <= P; kk <<= 1)
        for (uint64_t jj = kk >> 1; jj > 0; jj >>= 1) {
            for (uint64_t i = threadIdx.x; i < P; i += blockDim.x) {
                uint64_t p = i ^ jj;
                if (p > i) {
                    uint64_t x = scratch[i], y = scratch[p];
                    bool up = (i & kk) == 0;
                    uint64_t kx = x == ~0ull ? ~0ull : hit_key(x), ky = y == ~0ull ? ~0ull : hit_key(y);
                    if ((kx > ky) == up) { scratch[i] = y; scratch[p] = x; }
                }
            }
            __syncthreads();
        }
    for (uint64_t i = threadIdx.x; i < cnt; i += blockDim.x) hits[i] = scratch[i];
}

__global__ void k_debug_occ(const IndexView ix, const uint64_t *__restrict__ rows, uint64_t n,
                            uint32_t *__restrict__ out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t j = (uint32_t)rows[i];
        uint32_t ol[4], orr[4];
        occ_pair(ix, j, j, ol, orr);
        for (int c = 0; c < 4; c++) out[4 * i + c] = ol[c];
    }
}

__global__ void k_debug_locate(const IndexView ix, const uint64_t *__restrict__ rows, uint64_t n,
                               uint32_t *__restrict__ out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t steps = 0;
        out[i] = locate_row(ix, (uint32_t)rows[i], steps);
    }
}

__global__ void k_debug_seed(const IndexView ix, const uint32_t *__restrict__ codes, uint32_t len, uint64_t n,
                             uint32_t *__restrict__ out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t l, r;
        seed_interval(ix, codes[i], len, l, r);
        out[2 * i] = l;
        out[2 * i + 1] = r < l ? l : r;
    }
}

unsigned grid1(uint64_t n, int block = 256)
{
    return (unsigned)std::min<uint64_t>(std::max<uint64_t>((n + block - 1) / block, 1), 152ull * 64);
}

}  // namespace

// Exclusive scan of n uint64 counts into n + 1 offsets with caller-provided
// tile scratch of at least n / 2048 + 2 entries (no allocation).
int exclusive_scan_u64_scratch(const uint64_t *in, uint64_t n, uint64_t *out, unsigned long long *scratch,
                               cudaStream_t s)
{
    uint64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint64_t *ts = (uint64_t *)scratch;
    if (ntiles) k_scan_tiles<uint64_t><<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(in, n, out, ts);
    k_scan_sums<<<1, 1024, 0, s>>>(ts, ntiles);
    unsigned g = (unsigned)std::min<uint64_t>(std::max<uint64_t>((n + 255) / 256, 1), 152 * 32);
    k_scan_add<<<g, 256, 0, s>>>(out, n, ts);
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

static uint64_t big_list_bytes(uint64_t n)
{
    return (std::max<uint64_t>(n, 1) * 4 + 15) & ~15ull;
}

// w.big holds: the sort lists (n u32), 64 bytes of counters (locate steps
// u64, sort-list counts u32[2], many-interval count u32, the two sort
// kernels' next-read counters u32[2]), then the list of reads with many
// intervals (n u32).
struct PostLists {
    uint32_t *sort_lists;
    unsigned long long *steps;
    unsigned int *nbig;       // [0] reads for the shared-memory sorts, [1] above them
    unsigned int *n_many;
    unsigned int *sort_next;  // [0] k_sort_warp's next listed read, [1] k_sort_block's
    uint32_t *many;
};

static uint64_t post_list_bytes(uint64_t n) { return 2 * big_list_bytes(n) + 64; }

static PostLists post_lists(Workspace &w, uint64_t n)
{
    PostLists p;
    char *base = (char *)w.big.p;
    p.sort_lists = (uint32_t *)base;
    p.steps = (unsigned long long *)(base + big_list_bytes(n));
    p.nbig = (unsigned int *)(p.steps + 1);
    p.n_many = p.nbig + 2;
    p.sort_next = p.nbig + 3;
    p.many = (uint32_t *)(base + big_list_bytes(n) + 64);
    return p;
}

// The whole post-search pipeline for one batch, enqueued with every count
// read on the device (fixed grids, capacity-guarded writes) so it can be
// captured in a CUDA graph.  Buffers must already hold `hit_capacity` hits.
// Ends with a copy of the status (search control block, hit total, locate
// steps and sort-list counts) into pinned host memory `status`.
int enqueue_post_device(const mica_index *idx, Workspace &w, const ReadsView &rd, uint32_t hit_cap,
                        uint32_t report, uint64_t hit_capacity, cudaStream_t s, void *status, uint64_t &L)
{
    uint64_t n = rd.n;
    uint64_t *iv_off = (uint64_t *)w.iv_off.p, *hit_off = (uint64_t *)w.hit_off.p;
    PostLists pl = post_lists(w, n);
    unsigned long long *steps = pl.steps;
    unsigned int *nbig = pl.nbig;
    SearchCtl *ctl = (SearchCtl *)w.ctl.p;
    const unsigned G = 152 * 16;
    int rc;
    MICA_CUDA_TRY(cudaMemsetAsync(steps, 0, 64, s));
    if ((rc = exclusive_scan<uint32_t>(w.scan_tmp, (const uint32_t *)w.iv_cnt.p, n, iv_off, s, L))) return rc;
    k_iv_scatter<<<G, 256, 0, s>>>((const Interval *)w.iv.p, &ctl->iv_count, w.iv_cap, iv_off,
                                   (uint32_t *)w.iv_cnt.p, (Interval *)w.iv_sorted.p, &ctl->error);
    if (report == MICA_REPORT_BEST_STRATUM) {
        k_stratum<<<grid1(n, 128), 128, 0, s>>>((Interval *)w.iv_sorted.p, iv_off, n, &ctl->error);
        L++;
    }
    k_summarize<<<grid1(n, 128), 128, 0, s>>>((Interval *)w.iv_sorted.p, iv_off, n, hit_cap, (uint64_t *)w.total.p,
                                              (uint64_t *)w.keep.p, pl.many, pl.n_many, &ctl->error);
    k_summarize_many<<<152 * 2, MANY_THREADS, 0, s>>>((Interval *)w.iv_sorted.p, iv_off, hit_cap,
                                                      (uint64_t *)w.total.p, (uint64_t *)w.keep.p, pl.many,
                                                      pl.n_many, &ctl->error);
    L += 3;
    if ((rc = exclusive_scan<uint64_t>(w.scan_tmp, (const uint64_t *)w.keep.p, n, hit_off, s, L))) return rc;
    k_expand<<<grid1(n, 128), 128, 0, s>>>((const Interval *)w.iv_sorted.p, iv_off, hit_off, n, (Hit *)w.hits.p,
                                           hit_capacity, &ctl->error);
    k_locate<<<G, 256, 0, s>>>(idx->view, (Hit *)w.hits.p, hit_off + n, hit_capacity, steps, &ctl->error);
    k_sort_small<<<grid1(n, 128), 128, 0, s>>>((uint64_t *)w.hits.p, hit_off, n, hit_capacity, (uint32_t *)w.big.p,
                                               nbig);
    k_sort_warp<<<152 * 4, WARP_SORT_WARPS * 32, 0, s>>>((uint64_t *)w.hits.p, hit_off, (const uint32_t *)w.big.p,
                                                        nbig, pl.sort_next);
    k_sort_block<<<152 * 8, BLOCK_SORT_THREADS, 0, s>>>((uint64_t *)w.hits.p, hit_off, (const uint32_t *)w.big.p,
                                                        nbig, pl.sort_next + 1);
    L += 5;
    char *st = (char *)status;
    MICA_CUDA_TRY(cudaMemcpyAsync(st, ctl, sizeof(SearchCtl), cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaMemcpyAsync(st + sizeof(SearchCtl), hit_off + n, 8, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaMemcpyAsync(st + sizeof(SearchCtl) + 8, steps, 16, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

// Reserve every post-search buffer for n reads and hit_capacity hits.
// Device bytes reserve_post takes for n reads (the sizes below).
uint64_t post_workspace_bytes(uint64_t n, uint64_t iv_cap, uint64_t hit_capacity)
{
    uint64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return std::max<uint64_t>(iv_cap, 1) * sizeof(Interval) + 2 * (n + 1) * 8 + 2 * std::max<uint64_t>(n, 1) * 8 +
           post_list_bytes(n) + (ntiles + 1) * 8 + std::max<uint64_t>(hit_capacity, 1) * sizeof(Hit) + 64;
}

int reserve_post(Workspace &w, uint64_t n, uint32_t iv_cap, uint64_t hit_capacity)
{
    int rc;
    uint64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if ((rc = dev_reserve(w.iv_sorted, std::max<uint64_t>(iv_cap, 1) * sizeof(Interval))) ||
        (rc = dev_reserve(w.iv_off, (n + 1) * 8)) || (rc = dev_reserve(w.total, std::max<uint64_t>(n, 1) * 8)) ||
        (rc = dev_reserve(w.keep, std::max<uint64_t>(n, 1) * 8)) || (rc = dev_reserve(w.hit_off, (n + 1) * 8)) ||
        (rc = dev_reserve(w.big, post_list_bytes(n))) || (rc = dev_reserve(w.scan_tmp, (ntiles + 1) * 8)) ||
        (rc = dev_reserve(w.hits, std::max<uint64_t>(hit_capacity, 1) * sizeof(Hit) + 64)))
        return rc;
    return 0;
}

int run_post(const mica_index *idx, Workspace &w, mica_stats &stt, const ReadsView &rd, uint32_t hit_cap,
             uint32_t report, cudaStream_t s, uint64_t *n_hits_out)
{
    uint64_t n = rd.n;
    uint32_t niv = (uint32_t)stt.intervals;
    int rc;
    if ((rc = dev_reserve(w.iv_sorted, std::max<uint64_t>(niv, 1) * sizeof(Interval))) ||
        (rc = dev_reserve(w.iv_off, (n + 1) * 8)) || (rc = dev_reserve(w.total, std::max<uint64_t>(n, 1) * 8)) ||
        (rc = dev_reserve(w.keep, std::max<uint64_t>(n, 1) * 8)) || (rc = dev_reserve(w.hit_off, (n + 1) * 8)) ||
        (rc = dev_reserve(w.big, post_list_bytes(n))))
        return rc;
    uint64_t *iv_off = (uint64_t *)w.iv_off.p, *hit_off = (uint64_t *)w.hit_off.p;
    uint64_t &L = stt.launches;
    PostLists pl = post_lists(w, n);
    unsigned long long *steps = pl.steps;
    unsigned int *nbig = pl.nbig;
    MICA_CUDA_TRY(cudaMemsetAsync(steps, 0, 64, s));
    if ((rc = exclusive_scan<uint32_t>(w.scan_tmp, (const uint32_t *)w.iv_cnt.p, n, iv_off, s, L))) return rc;
    const unsigned int *err = &((SearchCtl *)w.ctl.p)->error;
    if (niv) { k_iv_scatter<<<grid1(niv), 256, 0, s>>>((const Interval *)w.iv.p, &((SearchCtl *)w.ctl.p)->iv_count,
                                                       w.iv_cap, iv_off, (uint32_t *)w.iv_cnt.p,
                                                       (Interval *)w.iv_sorted.p, err); L++; }
    if (n && report == MICA_REPORT_BEST_STRATUM) {
        k_stratum<<<grid1(n, 128), 128, 0, s>>>((Interval *)w.iv_sorted.p, iv_off, n, err);
        L++;
    }
    if (n) {
        k_summarize<<<grid1(n, 128), 128, 0, s>>>((Interval *)w.iv_sorted.p, iv_off, n, hit_cap,
                                                  (uint64_t *)w.total.p, (uint64_t *)w.keep.p, pl.many, pl.n_many,
                                                  err);
        k_summarize_many<<<152 * 2, MANY_THREADS, 0, s>>>((Interval *)w.iv_sorted.p, iv_off, hit_cap,
                                                          (uint64_t *)w.total.p, (uint64_t *)w.keep.p, pl.many,
                                                          pl.n_many, err);
        L += 2;
    }
    if ((rc = exclusive_scan<uint64_t>(w.scan_tmp, (const uint64_t *)w.keep.p, n, hit_off, s, L))) return rc;
    uint64_t nh = 0;
    MICA_CUDA_TRY(cudaMemcpyAsync(&nh, hit_off + n, 8, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    if ((rc = dev_reserve(w.hits, std::max<uint64_t>(nh, 1) * sizeof(Hit) + 64))) return rc;
    if (n) { k_expand<<<grid1(n, 128), 128, 0, s>>>((const Interval *)w.iv_sorted.p, iv_off, hit_off, n,
                                                   (Hit *)w.hits.p, nh, err); L++; }
    if (nh) { k_locate<<<grid1(nh), 256, 0, s>>>(idx->view, (Hit *)w.hits.p, hit_off + n, nh, steps, err); L++; }
    if (n) { k_sort_small<<<grid1(n, 128), 128, 0, s>>>((uint64_t *)w.hits.p, hit_off, n, nh, (uint32_t *)w.big.p,
                                                       nbig); L++; }
    unsigned int hb[2] = {0, 0};
    unsigned long long st = 0;
    MICA_CUDA_TRY(cudaMemcpyAsync(&st, steps, 8, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaMemcpyAsync(hb, nbig, 8, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    if (hb[0]) {
        k_sort_warp<<<std::min((hb[0] + WARP_SORT_WARPS - 1) / WARP_SORT_WARPS, 152u * 4), WARP_SORT_WARPS * 32, 0,
                      s>>>((uint64_t *)w.hits.p, hit_off, (const uint32_t *)w.big.p, nbig, pl.sort_next);
        k_sort_block<<<std::min(hb[0], 152u * 8), BLOCK_SORT_THREADS, 0, s>>>(
            (uint64_t *)w.hits.p, hit_off, (const uint32_t *)w.big.p, nbig, pl.sort_next + 1);
        L += 2;
    }
    if (hb[1]) {
        // reads above the shared-memory size (only without a cap or with a cap above it)
        std::vector<uint32_t> huge(hb[1]);
        MICA_CUDA_TRY(cudaMemcpyAsync(huge.data(), (const uint32_t *)w.big.p + (n - hb[1]), 4ull * hb[1],
                                      cudaMemcpyDeviceToHost, s));
        MICA_CUDA_TRY(cudaStreamSynchronize(s));
        for (uint32_t r : huge) {
            uint64_t ob[2];
            MICA_CUDA_TRY(cudaMemcpy(ob, hit_off + r, 16, cudaMemcpyDeviceToHost));
            uint64_t cnt = ob[1] - ob[0];
            uint64_t P = 1;
            while (P < cnt) P <<= 1;
            DevBuf scratch;
            if ((rc = dev_reserve(scratch, P * 8))) return rc;
            k_sort_global<<<1, 1024, 0, s>>>((uint64_t *)w.hits.p + ob[0], cnt, (uint64_t *)scratch.p, P);
            L++;
            MICA_CUDA_TRY(cudaStreamSynchronize(s));
            dev_release(scratch);
        }
    }
    MICA_CUDA_TRY(cudaGetLastError());
    stt.located = nh;
    stt.lf_steps = st;
    *n_hits_out = nh;
    return 0;
}

int debug_occ(const mica_index *idx, const uint64_t *d_rows, uint64_t n, uint32_t *d_out, cudaStream_t s)
{
    if (n) k_debug_occ<<<grid1(n), 256, 0, s>>>(idx->view, d_rows, n, d_out);
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

int debug_seed(const mica_index *idx, const uint32_t *d_codes, uint32_t len, uint64_t n, uint32_t *d_out,
               cudaStream_t s)
{
    if (n) k_debug_seed<<<grid1(n), 256, 0, s>>>(idx->view, d_codes, len, n, d_out);
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

int debug_locate(const mica_index *idx, const uint64_t *d_rows, uint64_t n, uint32_t *d_out, cudaStream_t s)
{
    if (n) k_debug_locate<<<grid1(n), 256, 0, s>>>(idx->view, d_rows, n, d_out);
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace mica
