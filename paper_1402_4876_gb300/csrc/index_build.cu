// GPU construction of the resident FM index (MICA, Section 2: a BWT index of
// the reference genome in the accelerator's global memory, organised to cut
// memory transactions per query).
//
//   1. suffix array of T = G$ by prefix doubling: sort positions by their
//      first 21 symbols (3 bits each), then repeatedly by (rank[i], rank[i+h])
//      with h doubling, until all ranks are distinct;
//   2. BWT[j] = T[SA[j]-1] as two bit planes in 32-byte blocks of 96 rows
//      that start with Occ(A..T, block start) relative to a superblock of
//      682 blocks, whose absolute counts sit in a small separate table;
//   3. mark bits for rows with SA[j] % s == 0 (64-byte blocks of 480 rows that
//      start with the number of marked rows before them) and the sampled SA
//      values in row order;
//   4. the q-mer table: bound[x] = number of suffixes of T smaller than the
//      q-mer x.  The SA interval of x is [bound[x], bound[x+1]) less the
//      suffixes u$ (|u| < q, at most q of them, at the end of G) whose
//      A-padded code is x+1: they sort after every suffix starting with x
//      (and, for shorter seeds, see seed_interval).
//
// The sorts and scans of this one-time build use CUB; the search path uses
// only this library's own kernels.
#include <cub/cub.cuh>

#include <algorithm>
#include <vector>

#include "mica_internal.cuh"

namespace mica {

namespace {

constexpr int KEY_SYMS = 21;   // symbols in the initial 63-bit key

__global__ void k_init_keys(const uint8_t *__restrict__ codes, uint64_t n,
                            uint64_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    uint64_t rows = n + 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < rows;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t key = 0;
#pragma unroll
        for (int j = 0; j < KEY_SYMS; j++) {
            uint64_t p = i + j;
            uint64_t s = p < n ? (uint64_t)codes[p] + 1 : 0;   // $ and beyond: 0
            key = (key << 3) | s;
        }
        keys[i] = key;
        vals[i] = (uint32_t)i;
    }
}

// head flag -> group head index (inclusive max-scan input); flags "not done"
__global__ void k_heads(const uint64_t *__restrict__ keys, uint64_t rows,
                        uint32_t *__restrict__ hv, int *__restrict__ not_done)
{
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < rows;
         p += (uint64_t)gridDim.x * blockDim.x) {
        bool head = (p == 0) || keys[p] != keys[p - 1];
        hv[p] = head ? (uint32_t)p : 0u;
        if (!head) *not_done = 1;
    }
}

__global__ void k_scatter_rank(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ grp,
                               uint64_t rows, uint32_t *__restrict__ rank)
{
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < rows;
         p += (uint64_t)gridDim.x * blockDim.x)
        rank[sa[p]] = grp[p];
}

__global__ void k_pair_keys(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ rank,
                            uint64_t n, uint64_t h, int bits, uint64_t *__restrict__ keys)
{
    uint64_t rows = n + 1;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < rows;
         p += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t i = sa[p];
        uint64_t r1 = rank[i];
        uint64_t r2 = (i + h <= n) ? (uint64_t)rank[i + h] + 1 : 0;
        keys[p] = (r1 << bits) | r2;
    }
}

struct MaxOp {
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a > b ? a : b; }
};

struct Sum4 {
    __device__ __forceinline__ uint4 operator()(const uint4 &a, const uint4 &b) const
    {
        return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
};

int grid_for(uint64_t n, int block = 256)
{
    uint64_t g = (n + block - 1) / block;
    return (int)std::min<uint64_t>(std::max<uint64_t>(g, 1), 152ull * 64);
}

template <typename NumT>
int sort_pairs(DevBuf &tmp, cub::DoubleBuffer<uint64_t> &keys, cub::DoubleBuffer<uint32_t> &vals,
               NumT rows, int end_bit, cudaStream_t s)
{
    size_t need = 0;
    MICA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, need, keys, vals, rows, 0, end_bit, s));
    if (int rc = dev_reserve(tmp, need)) return rc;
    MICA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, need, keys, vals, rows, 0, end_bit, s));
    return 0;
}

template <typename NumT>
int max_scan(DevBuf &tmp, const uint32_t *in, uint32_t *out, NumT rows, cudaStream_t s)
{
    size_t need = 0;
    MICA_CUDA_TRY(cub::DeviceScan::InclusiveScan(nullptr, need, in, out, MaxOp(), rows, s));
    if (int rc = dev_reserve(tmp, need)) return rc;
    MICA_CUDA_TRY(cub::DeviceScan::InclusiveScan(tmp.p, need, in, out, MaxOp(), rows, s));
    return 0;
}

template <typename NumT>
int doubling(const uint8_t *d_codes, uint64_t n, uint32_t *d_sa, cudaStream_t s)
{
    uint64_t rows = n + 1;
    DevBuf k0, k1, v1, rank, tmp, flag;
    int rc = 0;
    auto cleanup = [&]() { dev_release(k0); dev_release(k1); dev_release(v1); dev_release(rank);
                           dev_release(tmp); dev_release(flag); };
    if ((rc = dev_reserve(k0, rows * 8)) || (rc = dev_reserve(k1, rows * 8)) ||
        (rc = dev_reserve(v1, rows * 4)) || (rc = dev_reserve(rank, rows * 4)) ||
        (rc = dev_reserve(flag, 16))) { cleanup(); return rc; }
    cub::DoubleBuffer<uint64_t> keys((uint64_t *)k0.p, (uint64_t *)k1.p);
    cub::DoubleBuffer<uint32_t> vals(d_sa, (uint32_t *)v1.p);
    int bits = 1;
    while ((1ull << bits) < rows + 1) bits++;          // rank + 1 <= rows fits in `bits`
    int g = grid_for(rows);
    k_init_keys<<<g, 256, 0, s>>>(d_codes, n, keys.Current(), vals.Current());
    if ((rc = sort_pairs<NumT>(tmp, keys, vals, (NumT)rows, 3 * KEY_SYMS, s))) { cleanup(); return rc; }
    uint64_t h = KEY_SYMS;
    for (int iter = 0; iter < 64; iter++) {
        uint32_t *hv = (uint32_t *)keys.Alternate();            // free after the sort
        uint32_t *grp = hv + rows;
        int *nd = (int *)flag.p;
        cudaMemsetAsync(nd, 0, sizeof(int), s);
        k_heads<<<g, 256, 0, s>>>(keys.Current(), rows, hv, nd);
        int not_done = 0;
        MICA_CUDA_TRY(cudaMemcpyAsync(&not_done, nd, sizeof(int), cudaMemcpyDeviceToHost, s));
        MICA_CUDA_TRY(cudaStreamSynchronize(s));
        if (!not_done) break;
        if ((rc = max_scan<NumT>(tmp, hv, grp, (NumT)rows, s))) { cleanup(); return rc; }
        k_scatter_rank<<<g, 256, 0, s>>>(vals.Current(), grp, rows, (uint32_t *)rank.p);
        k_pair_keys<<<g, 256, 0, s>>>(vals.Current(), (const uint32_t *)rank.p, n, h, bits,
                                      keys.Current());
        if ((rc = sort_pairs<NumT>(tmp, keys, vals, (NumT)rows, 2 * bits, s))) { cleanup(); return rc; }
        h *= 2;
    }
    if (vals.Current() != d_sa)
        MICA_CUDA_TRY(cudaMemcpyAsync(d_sa, vals.Current(), rows * 4, cudaMemcpyDeviceToDevice, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    MICA_CUDA_TRY(cudaGetLastError());
    cleanup();
    return 0;
}

// ---- BWT / occurrence blocks ----

__global__ void k_occ_counts(const uint32_t *__restrict__ sa, const uint8_t *__restrict__ codes,
                             uint64_t rows, uint64_t nblocks, uint4 *__restrict__ cnt,
                             uint32_t *__restrict__ dollar_row)
{
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c4[4] = {0, 0, 0, 0};
        uint64_t j0 = b * OCC_ROWS, j1 = min(rows, j0 + OCC_ROWS);
        for (uint64_t j = j0; j < j1; j++) {
            uint32_t i = sa[j];
            if (i == 0) { *dollar_row = (uint32_t)j; continue; }
            c4[codes[i - 1]]++;
        }
        cnt[b] = make_uint4(c4[0], c4[1], c4[2], c4[3]);
    }
}

__global__ void k_occ_super(const uint4 *__restrict__ base, uint64_t nblocks, uint64_t nsuper,
                            uint4 *__restrict__ super)
{
    for (uint64_t sb = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; sb < nsuper;
         sb += (uint64_t)gridDim.x * blockDim.x)
        super[sb] = base[sb * SB_BLOCKS];
}

__global__ void k_occ_blocks(const uint32_t *__restrict__ sa, const uint8_t *__restrict__ codes,
                             uint64_t rows, uint64_t nblocks, const uint4 *__restrict__ base,
                             const uint4 *__restrict__ super, uint32_t *__restrict__ occ)
{
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t *blk = occ + b * OCC_WORDS;
        uint4 c = base[b], sp = super[b / SB_BLOCKS];
        blk[0] = (c.x - sp.x) | ((c.y - sp.y) << 16);
        blk[1] = (c.z - sp.z) | ((c.w - sp.w) << 16);
        uint64_t j0 = b * OCC_ROWS;
        for (int w = 0; w < 3; w++) {
            uint32_t lo = 0, hi = 0;
            for (int t = 0; t < 32; t++) {
                uint64_t j = j0 + w * 32 + t;
                uint32_t sym = 0;
                if (j < rows) {
                    uint32_t i = sa[j];
                    sym = i == 0 ? 0u : codes[i - 1];     // $ stored as A
                }
                lo |= (sym & 1u) << t;
                hi |= (sym >> 1) << t;
            }
            blk[2 + 2 * w] = lo;
            blk[3 + 2 * w] = hi;
        }
    }
}

// ---- marks and SA samples ----

__global__ void k_mark_counts(const uint32_t *__restrict__ sa, uint64_t rows, uint64_t nblocks,
                              uint32_t s, uint32_t *__restrict__ cnt)
{
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c = 0;
        uint64_t j0 = b * MARK_ROWS, j1 = min(rows, j0 + MARK_ROWS);
        for (uint64_t j = j0; j < j1; j++) c += (sa[j] % s) == 0;
        cnt[b] = c;
    }
}

__global__ void k_mark_blocks(const uint32_t *__restrict__ sa, uint64_t rows, uint64_t nblocks,
                              uint32_t s, const uint32_t *__restrict__ base,
                              uint32_t *__restrict__ marks, uint32_t *__restrict__ samples)
{
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t *blk = marks + b * 16;
        uint32_t r = base[b];
        blk[0] = r;
        uint64_t j0 = b * MARK_ROWS;
        for (int w = 0; w < 15; w++) {
            uint32_t word = 0;
            for (int t = 0; t < 32; t++) {
                uint64_t j = j0 + w * 32 + t;
                if (j < rows && sa[j] % s == 0) {
                    word |= 1u << t;
                    samples[r++] = sa[j];
                }
            }
            blk[1 + w] = word;
        }
    }
}

// ---- q-mer table ----

__global__ void k_qmer_hist(const uint8_t *__restrict__ codes, uint64_t n, uint32_t q,
                            uint32_t *__restrict__ cnt)
{
    if (n < q) return;
    uint64_t last = n - q;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= last;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t code = 0;
        for (uint32_t t = 0; t < q; t++) code = (code << 2) | codes[i + t];
        atomicAdd(&cnt[code], 1u);
    }
}

// Suffixes shorter than q + 1 symbols (w$ with |w| < q) count as smaller
// than x exactly when w padded with A up to q symbols is <= x: add them to
// the exclusive scan's input (for x > pad) and, after the scan, to x = pad.
__global__ void k_qmer_short(const uint8_t *__restrict__ codes, uint64_t n, uint32_t q,
                             uint32_t *__restrict__ cnt, int after_scan)
{
    uint64_t first = n >= q ? n - q + 1 : 0;
    for (uint64_t i = first + threadIdx.x; i <= n; i += blockDim.x) {
        uint32_t code = 0;
        for (uint32_t t = 0; t < q; t++) {
            uint64_t p = i + t;
            code = (code << 2) | (p < n ? codes[p] : 0u);
        }
        atomicAdd(&cnt[code], 1u);
        (void)after_scan;
    }
}

int exclusive_sum_u32(DevBuf &tmp, const uint32_t *in, uint32_t *out, uint64_t n, cudaStream_t s)
{
    size_t need = 0;
    MICA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, need, in, out, (int64_t)n, s));
    if (int rc = dev_reserve(tmp, need)) return rc;
    MICA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp.p, need, in, out, (int64_t)n, s));
    return 0;
}

}  // namespace

int build_suffix_array(const uint8_t *d_codes, uint64_t n, uint32_t *d_sa, cudaStream_t s)
{
    if (n + 1 >= (1ull << 32)) return MICA_EINVAL;
    if (n + 1 < (1ull << 31)) return doubling<int>(d_codes, n, d_sa, s);
    return doubling<int64_t>(d_codes, n, d_sa, s);
}

// ---- seed variants ----

static uint32_t binom(uint32_t n, uint32_t k)
{
    if (k > n) return 0;
    uint64_t r = 1;
    for (uint32_t i = 0; i < k; i++) r = r * (n - i) / (i + 1);
    return (uint32_t)r;
}

uint32_t variant_count(uint32_t q, uint32_t k)
{
    uint32_t v = 0, p3 = 1;
    for (uint32_t d = 0; d <= k; d++) { v += binom(q, d) * p3; p3 *= 3; }
    return v;
}

void host_variant_table(uint32_t *out)
{
    for (uint32_t k = 0; k <= 3; k++) {
        struct E { int maxpos; uint32_t word; };
        std::vector<E> list;
        // every subset of the 12 window positions with at most k members
        for (uint32_t set = 0; set < (1u << MAX_Q); set++) {
            uint32_t d = __builtin_popcount(set);
            if (d > k) continue;
            uint32_t pos[3];
            uint32_t np = 0;
            for (uint32_t u = 0; u < MAX_Q; u++) if (set >> u & 1) pos[np++] = u;
            uint32_t combos = 1;
            for (uint32_t t = 0; t < d; t++) combos *= 3;
            for (uint32_t c = 0; c < combos; c++) {
                uint32_t mask = 0, cc = c;
                for (uint32_t t = 0; t < d; t++) { mask |= ((cc % 3) + 1) << (2 * pos[t]); cc /= 3; }
                list.push_back({d ? (int)pos[d - 1] : -1, mask | (d << 24)});
            }
        }
        std::stable_sort(list.begin(), list.end(), [](const E &a, const E &b) { return a.maxpos < b.maxpos; });
        for (size_t i = 0; i < list.size(); i++) out[VAR_OFF[k] + i] = list[i].word;
    }
}

int upload_variants(mica_index *idx)
{
    std::vector<uint32_t> v(N_VARIANTS);
    host_variant_table(v.data());
    if (int rc = dev_reserve(idx->variants, N_VARIANTS * 4)) return rc;
    MICA_CUDA_TRY(cudaMemcpy(idx->variants.p, v.data(), N_VARIANTS * 4, cudaMemcpyHostToDevice));
    idx->view.variants = (const uint32_t *)idx->variants.p;
    return 0;
}

// Occurrence blocks and superblocks of T = text$ from its suffix array: the
// block layout of the search (counts relative to the superblock, two bit
// planes), the $ row and C[].  Used for the genome and for its reversal.
static int build_occ(const uint8_t *d_codes, uint64_t n, const uint32_t *d_sa, DevBuf &occ, DevBuf &super,
                     uint32_t &dollar, uint32_t (&C)[5], cudaStream_t s)
{
    uint64_t rows = n + 1;
    uint64_t nb = rows / OCC_ROWS + 1;
    uint64_t nsb = (nb + SB_BLOCKS - 1) / SB_BLOCKS;
    DevBuf tmp, cnt, base, dr;
    auto cleanup = [&]() { dev_release(tmp); dev_release(cnt); dev_release(base); dev_release(dr); };
    int rc;
    if ((rc = dev_reserve(cnt, nb * 16)) || (rc = dev_reserve(base, nb * 16)) ||
        (rc = dev_reserve(dr, 16)) || (rc = dev_reserve(occ, nb * 32)) ||
        (rc = dev_reserve(super, nsb * 16))) { cleanup(); return rc; }
    int g = grid_for(nb);
    k_occ_counts<<<g, 256, 0, s>>>(d_sa, d_codes, rows, nb, (uint4 *)cnt.p, (uint32_t *)dr.p);
    {
        size_t need = 0;
        cudaError_t e = cub::DeviceScan::ExclusiveScan(nullptr, need, (const uint4 *)cnt.p, (uint4 *)base.p,
                                                       Sum4(), make_uint4(0, 0, 0, 0), (int64_t)nb, s);
        if (e == cudaSuccess && (rc = dev_reserve(tmp, need))) { cleanup(); return rc; }
        if (e == cudaSuccess)
            e = cub::DeviceScan::ExclusiveScan(tmp.p, need, (const uint4 *)cnt.p, (uint4 *)base.p, Sum4(),
                                               make_uint4(0, 0, 0, 0), (int64_t)nb, s);
        if (e != cudaSuccess) { cleanup(); set_last_cuda_error(e, "occ scan", __FILE__, __LINE__); return MICA_ECUDA; }
    }
    k_occ_super<<<grid_for(nsb), 256, 0, s>>>((const uint4 *)base.p, nb, nsb, (uint4 *)super.p);
    k_occ_blocks<<<g, 256, 0, s>>>(d_sa, d_codes, rows, nb, (const uint4 *)base.p, (const uint4 *)super.p,
                                   (uint32_t *)occ.p);
    // totals for C[]: the last block's base plus the rows inside it
    uint4 tot{}, last{};
    cudaError_t e = cudaMemcpyAsync(&dollar, dr.p, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, (const uint4 *)base.p + (nb - 1), 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last, (const uint4 *)cnt.p + (nb - 1), 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) { set_last_cuda_error(e, "occ totals", __FILE__, __LINE__); return MICA_ECUDA; }
    uint64_t cA = (uint64_t)tot.x + last.x, cC = (uint64_t)tot.y + last.y,
             cG = (uint64_t)tot.z + last.z, cT = (uint64_t)tot.w + last.w;
    C[0] = 1;
    C[1] = (uint32_t)(1 + cA);
    C[2] = (uint32_t)(1 + cA + cC);
    C[3] = (uint32_t)(1 + cA + cC + cG);
    C[4] = (uint32_t)(1 + cA + cC + cG + cT);
    return 0;
}

__global__ void k_reverse_codes(const uint8_t *__restrict__ in, uint64_t n, uint8_t *__restrict__ out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[n - 1 - i] = in[i];
}

// The q-mer table of a text T = codes$ (bound[x] = suffixes of T smaller than
// the q-mer x) and the A-padded codes of its suffixes shorter than q + 1
// symbols, which seed lookups correct for.
int build_qmer_table(const uint8_t *d_codes, uint64_t n, uint32_t q, DevBuf &table, QmerShort &sh, DevBuf &tmp,
                     cudaStream_t s)
{
    uint64_t tl = (1ull << (2 * q)) + 1;
    uint64_t first = n >= q ? n - q + 1 : 0;
    std::vector<uint8_t> tail(n - first);
    if (!tail.empty()) MICA_CUDA_TRY(cudaMemcpy(tail.data(), d_codes + first, tail.size(), cudaMemcpyDeviceToHost));
    sh = QmerShort{};
    for (uint64_t i = first; i <= n; i++) {
        uint32_t code = 0;
        for (uint32_t t = 0; t < q; t++) code = (code << 2) | (i + t < n ? tail[i + t - first] : 0u);
        sh.len[sh.nshort] = (uint32_t)(n - i);
        sh.pad[sh.nshort++] = code;
        sh.bloom |= 1ull << (code & 63);
    }
    DevBuf tcnt;
    int rc;
    if ((rc = dev_reserve(tcnt, tl * 4)) || (rc = dev_reserve(table, tl * 4))) { dev_release(tcnt); return rc; }
    MICA_CUDA_TRY(cudaMemsetAsync(tcnt.p, 0, tl * 4, s));
    k_qmer_hist<<<grid_for(n + 1), 256, 0, s>>>(d_codes, n, q, (uint32_t *)tcnt.p);
    k_qmer_short<<<1, 32, 0, s>>>(d_codes, n, q, (uint32_t *)tcnt.p, 0);
    if ((rc = exclusive_sum_u32(tmp, (const uint32_t *)tcnt.p, (uint32_t *)table.p, tl, s))) {
        dev_release(tcnt);
        return rc;
    }
    k_qmer_short<<<1, 32, 0, s>>>(d_codes, n, q, (uint32_t *)table.p, 1);
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    MICA_CUDA_TRY(cudaGetLastError());
    dev_release(tcnt);
    return 0;
}

void set_rev_short(IndexView &v, const QmerShort &sh)
{
    v.rev.nshort = sh.nshort;
    v.rev.short_bloom = sh.bloom;
    for (uint32_t t = 0; t < MAX_Q; t++) {
        v.rev.short_pad[t] = sh.pad[t];
        v.rev.short_len[t] = sh.len[t];
    }
}

int build_index_from_codes(const uint8_t *d_codes, uint64_t n, const mica_index_params &p,
                           mica_index *idx, cudaStream_t s)
{
    uint64_t rows = n + 1;
    DevBuf sa, tmp;
    auto cleanup = [&]() { dev_release(sa); dev_release(tmp); };
    int rc;
    if ((rc = dev_reserve(sa, rows * 4))) return rc;
    if ((rc = build_suffix_array(d_codes, n, (uint32_t *)sa.p, s))) { cleanup(); return rc; }
    const uint32_t *d_sa = (const uint32_t *)sa.p;

    // occurrence blocks and superblocks
    uint64_t nb = rows / OCC_ROWS + 1;
    uint64_t nsb = (nb + SB_BLOCKS - 1) / SB_BLOCKS;
    uint32_t dollar = 0, Cf[5];
    if ((rc = build_occ(d_codes, n, d_sa, idx->occ, idx->super, dollar, Cf, s))) { cleanup(); return rc; }

    // marks and samples
    uint32_t sr = p.sa_sample;
    uint64_t nm = rows / MARK_ROWS + 1;
    DevBuf mcnt, mbase;
    if ((rc = dev_reserve(mcnt, nm * 4)) || (rc = dev_reserve(mbase, nm * 4)) ||
        (rc = dev_reserve(idx->marks, nm * 64))) { cleanup(); dev_release(mcnt); dev_release(mbase); return rc; }
    int gm = grid_for(nm);
    k_mark_counts<<<gm, 256, 0, s>>>(d_sa, rows, nm, sr, (uint32_t *)mcnt.p);
    if ((rc = exclusive_sum_u32(tmp, (const uint32_t *)mcnt.p, (uint32_t *)mbase.p, nm, s))) {
        cleanup(); dev_release(mcnt); dev_release(mbase); return rc;
    }
    uint32_t mb_last = 0, mc_last = 0;
    MICA_CUDA_TRY(cudaMemcpyAsync(&mb_last, (const uint32_t *)mbase.p + nm - 1, 4, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaMemcpyAsync(&mc_last, (const uint32_t *)mcnt.p + nm - 1, 4, cudaMemcpyDeviceToHost, s));
    MICA_CUDA_TRY(cudaStreamSynchronize(s));
    uint64_t nsamp = (uint64_t)mb_last + mc_last;
    if ((rc = dev_reserve(idx->samples, std::max<uint64_t>(nsamp, 1) * 4))) {
        cleanup(); dev_release(mcnt); dev_release(mbase); return rc;
    }
    k_mark_blocks<<<gm, 256, 0, s>>>(d_sa, rows, nm, sr, (const uint32_t *)mbase.p,
                                     (uint32_t *)idx->marks.p, (uint32_t *)idx->samples.p);
    dev_release(mcnt);
    dev_release(mbase);

    // the whole suffix array (this one), its inverse and the 2-bit text
    if (p.full_sa && (rc = build_full_sa(idx, sa, d_codes, n, s))) { cleanup(); return rc; }

    // q-mer table
    uint64_t tl = (1ull << (2 * p.kmer_q)) + 1;
    {
        QmerShort sh;
        if ((rc = build_qmer_table(d_codes, n, p.kmer_q, idx->table, sh, tmp, s))) { cleanup(); return rc; }
        idx->view.nshort = sh.nshort;
        idx->view.short_bloom = sh.bloom;
        for (uint32_t t = 0; t < MAX_Q; t++) {
            idx->view.short_pad[t] = sh.pad[t];
            idx->view.short_len[t] = sh.len[t];
        }
    }

    // the reversed genome's occurrence blocks, for mismatch lower bounds
    uint32_t rdollar = 0, rC[5] = {0, 0, 0, 0, 0};
    if (p.lower_bounds) {
        DevBuf rcodes;
        if ((rc = dev_reserve(rcodes, std::max<uint64_t>(n, 1)))) { cleanup(); return rc; }
        if (n) k_reverse_codes<<<grid_for(n), 256, 0, s>>>(d_codes, n, (uint8_t *)rcodes.p);
        rc = dev_reserve(sa, rows * 4);   // (empty when the forward suffix array was kept)
        if (!rc) rc = build_suffix_array((const uint8_t *)rcodes.p, n, (uint32_t *)sa.p, s);
        if (!rc) rc = build_occ((const uint8_t *)rcodes.p, n, (const uint32_t *)sa.p, idx->rocc, idx->rsuper,
                                rdollar, rC, s);
        // and its q-mer table: the seed of a bidirectional search needs the
        // interval of the reversed q-mer too
        QmerShort rsh;
        if (!rc) rc = build_qmer_table((const uint8_t *)rcodes.p, n, p.kmer_q, idx->rtable, rsh, tmp, s);
        dev_release(rcodes);
        if (rc) { cleanup(); return rc; }
        set_rev_short(idx->view, rsh);
    }
    idx->has_rev = p.lower_bounds != 0;
    cleanup();

    idx->n = n;
    idx->params = p;
    idx->n_occ_blocks = nb;
    idx->n_super = nsb;
    idx->n_mark_blocks = nm;
    idx->n_samples = nsamp;
    idx->table_len = tl;
    IndexView &v = idx->view;
    v.occ = (const uint4 *)idx->occ.p;
    v.super = (const uint4 *)idx->super.p;
    v.marks = (const uint4 *)idx->marks.p;
    v.samples = (const uint32_t *)idx->samples.p;
    v.table = (const uint32_t *)idx->table.p;
    v.n = n;
    v.rows = (uint32_t)rows;
    v.dollar_row = dollar;
    for (int c = 0; c < 5; c++) v.C[c] = Cf[c];
    v.rev.occ = idx->has_rev ? (const uint4 *)idx->rocc.p : nullptr;
    v.rev.super = idx->has_rev ? (const uint4 *)idx->rsuper.p : nullptr;
    v.rev.dollar_row = rdollar;
    for (int c = 0; c < 5; c++) v.rev.C[c] = rC[c];
    v.rev.table = idx->has_rev ? (const uint32_t *)idx->rtable.p : nullptr;
    v.q = p.kmer_q;
    v.sa_sample = p.sa_sample;
    set_full_sa_view(idx);
    if (int rc2 = build_long_tables(idx, d_codes, s)) return rc2;
    return upload_variants(idx);
}

}  // namespace mica
