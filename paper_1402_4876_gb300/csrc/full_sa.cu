// The whole suffix array, its inverse and the 2-bit text, kept on the device
// when an index is built with full_sa (GB300's HBM holds them beside the
// index: 8 (N + 1) + N / 4 bytes, 25 GB for a 3.1 Gbp genome).
//
// With them the bidirectional search checks an interval of one row against
// the text: the row's suffix starts where the matched substring of the
// pattern lies in G, so one read of SA and one of the text window decide the
// rest of that node's subtree, which is a single path (each of its rows has
// one preceding and one following symbol), and ISA gives the leaf's row.
// Locating a row becomes one read of SA instead of an LF walk.
//
// At build time the suffix array is the one the index was built from.  An
// index file does not store them: loading rebuilds them from the sampled
// suffix array by inverting the BWT (Burrows and Wheeler; the LF mapping
// LF(j) = C[c] + Occ(c, j) with c = BWT[j] = G[SA[j] - 1] gives
// SA[LF(j)] = SA[j] - 1): from each row whose SA value is a multiple of s,
// LF steps recover the s - 1 positions below it, their rows and the symbols.
//
// The text also gives the bidirectional seeds longer q-mer tables (of G$ and
// of G~$, q about log4 N + 1, at most 15): a seed of that length is mostly a
// single occurrence already, so the search goes from the table lookup to the
// text check without the interval extensions in between.
#include <algorithm>

#include "search_common.cuh"

namespace mica {
namespace {

unsigned grid_of(uint64_t n, unsigned block = 256)
{
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + block - 1) / block, 152ull * 64));
}

__global__ void k_isa_scatter(const uint32_t *__restrict__ sa, uint64_t rows, uint32_t *__restrict__ isa)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < rows; j += (uint64_t)gridDim.x * blockDim.x)
        isa[sa[j]] = (uint32_t)j;
}

__global__ void k_pack_text(const uint8_t *__restrict__ codes, uint64_t n, uint64_t words, uint32_t *__restrict__ text)
{
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        const uint64_t p0 = w * 16;
#pragma unroll
        for (int i = 0; i < 16; i++)
            if (p0 + i < n) v |= (uint32_t)(codes[p0 + i] & 3u) << (2 * i);
        text[w] = v;
    }
}

// LF walk from row j with SA[j] = p down to the next multiple of s below p:
// SA and ISA of every row passed, and the symbols G[p' .. p - 1] OR-ed into
// the text words (zeroed before), one atomic per word touched.  The arrays
// come from a file: a row or position out of range sets *err and ends the walk.
__device__ void invert_from(const IndexView &ix, uint32_t j, uint32_t p, uint32_t s, uint32_t *__restrict__ sa,
                            uint32_t *__restrict__ isa, uint32_t *__restrict__ text, unsigned *err)
{
    if (j >= ix.rows || p > ix.n) { atomicOr(err, 1u); return; }
    sa[j] = p;
    isa[p] = j;
    uint32_t cur_w = 0xffffffffu, acc = 0;
    while (p > 0) {
        // c = BWT[j] = G[p - 1] (j is not the $ row: that row's SA value is 0)
        const uint32_t b = j / OCC_ROWS, o = j - b * OCC_ROWS;
        const uint4 sup = __ldg(ix.super + b / SB_BLOCKS);
        OccBlock k;
        load_block(ix, b, o + 1, k);
        const uint32_t c = block_symbol(k, o);
        const uint32_t q = p - 1, w = q >> 4;
        if (w != cur_w) {
            if (cur_w != 0xffffffffu) atomicOr(text + cur_w, acc);
            cur_w = w;
            acc = 0;
        }
        acc |= c << (2 * (q & 15u));
        j = ix.C[c] + occ_single(ix, b, o, sup, k, c);
        p = q;
        if (p % s == 0) break;   // a sampled position: its own walk covers what lies below
        if (j >= ix.rows) { atomicOr(err, 1u); break; }
        sa[j] = p;
        isa[p] = j;
    }
    if (cur_w != 0xffffffffu) atomicOr(text + cur_w, acc);
}

// One thread per mark block: a walk from each of its marked rows, and from
// row 0 (SA = N, the suffix $) when N is not a multiple of s.
__global__ void k_invert_bwt(const IndexView ix, uint64_t n_mark_blocks, uint64_t n_samples,
                             uint32_t *__restrict__ sa, uint32_t *__restrict__ isa, uint32_t *__restrict__ text,
                             unsigned *err)
{
    const uint32_t s = ix.sa_sample;
    for (uint64_t mb = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; mb < n_mark_blocks;
         mb += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t *blk = (const uint32_t *)(ix.marks + mb * 4);
        uint32_t rank = __ldg(blk);
        for (int wi = 0; wi < 15; wi++) {
            uint32_t word = __ldg(blk + 1 + wi);
            while (word) {
                const uint32_t bit = (uint32_t)__ffs(word) - 1;
                word &= word - 1;
                const uint32_t j = (uint32_t)(mb * MARK_ROWS) + 32u * wi + bit;
                if (rank >= n_samples) { atomicOr(err, 1u); break; }
                invert_from(ix, j, __ldg(ix.samples + rank), s, sa, isa, text, err);
                rank++;
            }
        }
        if (mb == 0 && ix.n % s != 0) invert_from(ix, 0, (uint32_t)ix.n, s, sa, isa, text, err);
    }
}

__global__ void k_unpack_text(const uint32_t *__restrict__ text, uint64_t n, int reverse, uint8_t *__restrict__ codes)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = reverse ? n - 1 - i : i;
        codes[i] = (uint8_t)((text[p >> 4] >> (2 * (p & 15))) & 3u);
    }
}

__global__ void k_reverse_bytes(const uint8_t *__restrict__ in, uint64_t n, uint8_t *__restrict__ out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = in[n - 1 - i];
}

void set_qmer_view(QmerView &v, const DevBuf &table, uint32_t q, const QmerShort &sh)
{
    v = QmerView{};
    v.table = (const uint32_t *)table.p;
    v.q = q;
    v.nshort = sh.nshort;
    v.short_bloom = sh.bloom;
    for (uint32_t t = 0; t < MAX_LQ; t++) {
        v.short_pad[t] = sh.pad[t];
        v.short_len[t] = sh.len[t];
    }
}

__global__ void k_table_interval(const QmerView t, const uint32_t *__restrict__ codes, uint32_t len, uint64_t n,
                                 uint32_t *__restrict__ out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t l, r;
        seed_interval_in(t.table, t.q, t.nshort, t.short_pad, t.short_len, t.short_bloom, codes[i], len, l, r);
        out[2 * i] = l;
        out[2 * i + 1] = r;
    }
}

}  // namespace

uint32_t long_seed_q(uint64_t n, uint32_t q)
{
    uint32_t l = 0;
    while (l < 16 && (1ull << (2 * l)) < n + 1) l++;   // ceil(log4(n + 1))
    return std::min(MAX_LQ, std::max(q, l + 1));
}

int build_long_tables(mica_index *idx, const uint8_t *d_codes, cudaStream_t s)
{
    idx->view.lfwd = QmerView{};
    idx->view.lrev = QmerView{};
    const uint64_t n = idx->n;
    const uint32_t lq = long_seed_q(n, idx->params.kmer_q);
    if (!idx->has_full_sa || !idx->has_rev || lq <= idx->params.kmer_q || n == 0) return 0;
    DevBuf own, rcodes, tmp;
    auto cleanup = [&]() { dev_release(own); dev_release(rcodes); dev_release(tmp); };
    int rc;
    if (!d_codes) {
        if ((rc = dev_reserve(own, n))) return rc;
        k_unpack_text<<<grid_of(n), 256, 0, s>>>((const uint32_t *)idx->text.p, n, 0, (uint8_t *)own.p);
        d_codes = (const uint8_t *)own.p;
    }
    QmerShort fsh, rsh;
    if ((rc = build_qmer_table(d_codes, n, lq, idx->ltable, fsh, tmp, s))) { cleanup(); return rc; }
    if ((rc = dev_reserve(rcodes, n))) { cleanup(); return rc; }
    k_reverse_bytes<<<grid_of(n), 256, 0, s>>>(d_codes, n, (uint8_t *)rcodes.p);
    if ((rc = build_qmer_table((const uint8_t *)rcodes.p, n, lq, idx->lrtable, rsh, tmp, s))) { cleanup(); return rc; }
    cleanup();
    set_qmer_view(idx->view.lfwd, idx->ltable, lq, fsh);
    set_qmer_view(idx->view.lrev, idx->lrtable, lq, rsh);
    return 0;
}

uint64_t full_sa_text_words(uint64_t n) { return ((n + 15) / 16 + 4 + 3) & ~3ull; }

uint64_t full_sa_bytes(uint64_t n) { return 8 * (n + 1) + 4 * full_sa_text_words(n); }

void set_full_sa_view(mica_index *idx)
{
    idx->view.sa_full = idx->has_full_sa ? (const uint32_t *)idx->sa_full.p : nullptr;
    idx->view.isa = idx->has_full_sa ? (const uint32_t *)idx->isa.p : nullptr;
    idx->view.text = idx->has_full_sa ? (const uint32_t *)idx->text.p : nullptr;
}

// At build time: takes the suffix array `sa` (rows entries) as the index's
// own, scatters its inverse and packs the text from the 2-bit codes.
int build_full_sa(mica_index *idx, DevBuf &sa, const uint8_t *d_codes, uint64_t n, cudaStream_t s)
{
    const uint64_t rows = n + 1, words = full_sa_text_words(n);
    std::swap(idx->sa_full, sa);
    int rc;
    if ((rc = dev_reserve(idx->isa, rows * 4)) || (rc = dev_reserve(idx->text, words * 4))) return rc;
    k_isa_scatter<<<grid_of(rows), 256, 0, s>>>((const uint32_t *)idx->sa_full.p, rows, (uint32_t *)idx->isa.p);
    k_pack_text<<<grid_of(words), 256, 0, s>>>(d_codes, n, words, (uint32_t *)idx->text.p);
    MICA_CUDA_TRY(cudaGetLastError());
    idx->has_full_sa = true;
    return 0;
}

// At load time: rebuilds all three from the occurrence blocks, the marks and
// the sampled suffix array (the index view must be complete).  MICA_EIO when
// those name a row, position or sample out of range.
int rebuild_full_sa(mica_index *idx, cudaStream_t s)
{
    const uint64_t n = idx->n, rows = n + 1, words = full_sa_text_words(n);
    int rc;
    DevBuf err;
    if ((rc = dev_reserve(idx->sa_full, rows * 4)) || (rc = dev_reserve(idx->isa, rows * 4)) ||
        (rc = dev_reserve(idx->text, words * 4)) || (rc = dev_reserve(err, 4)))
        return rc;
    unsigned herr = 0;
    cudaError_t e = cudaMemsetAsync(idx->text.p, 0, words * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err.p, 0, 4, s);
    if (e == cudaSuccess) {
        k_invert_bwt<<<grid_of(idx->n_mark_blocks, 128), 128, 0, s>>>(
            idx->view, idx->n_mark_blocks, idx->n_samples, (uint32_t *)idx->sa_full.p, (uint32_t *)idx->isa.p,
            (uint32_t *)idx->text.p, (unsigned *)err.p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_release(err);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "full suffix array rebuild", __FILE__, __LINE__);
        return MICA_ECUDA;
    }
    if (herr) return MICA_EIO;
    idx->has_full_sa = true;
    return 0;
}

}  // namespace mica

using namespace mica;

extern "C" int mica_debug_table_interval(const mica_index *idx, uint32_t which, const uint32_t *codes, uint32_t len,
                                         uint64_t n, uint32_t *lr_out)
{
    if (!idx || which > 3 || (n && (!codes || !lr_out))) return MICA_EINVAL;
    QmerView t{};
    const IndexView &v = idx->view;
    if (which < 2) {
        t.table = which == 0 ? v.table : v.rev.table;
        t.q = v.q;
        t.nshort = which == 0 ? v.nshort : v.rev.nshort;
        t.short_bloom = which == 0 ? v.short_bloom : v.rev.short_bloom;
        for (uint32_t i = 0; i < MAX_Q; i++) {
            t.short_pad[i] = which == 0 ? v.short_pad[i] : v.rev.short_pad[i];
            t.short_len[i] = which == 0 ? v.short_len[i] : v.rev.short_len[i];
        }
    } else {
        t = which == 2 ? v.lfwd : v.lrev;
    }
    if (!t.table || len < 1 || len > t.q) return MICA_EINVAL;
    for (uint64_t i = 0; i < n; i++)
        if ((uint64_t)codes[i] >= (1ull << (2 * len))) return MICA_EINVAL;
    if (n == 0) return 0;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    DevBuf dc, dout;
    int rc = dev_reserve(dc, n * 4);
    if (!rc) rc = dev_reserve(dout, n * 8);
    if (!rc && cudaMemcpy(dc.p, codes, n * 4, cudaMemcpyHostToDevice) != cudaSuccess) rc = MICA_ECUDA;
    if (!rc) {
        k_table_interval<<<grid_of(n), 256>>>(t, (const uint32_t *)dc.p, len, n, (uint32_t *)dout.p);
        if (cudaGetLastError() != cudaSuccess) rc = MICA_ECUDA;
    }
    if (!rc && cudaMemcpy(lr_out, dout.p, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MICA_ECUDA;
    dev_release(dc);
    dev_release(dout);
    return rc;
}

extern "C" int mica_debug_full_sa(const mica_index *idx, uint32_t which, uint64_t first, uint64_t n, uint32_t *out)
{
    if (!idx || which > 2 || (n && !out) || !idx->has_full_sa) return MICA_EINVAL;
    const uint64_t len = which == 2 ? full_sa_text_words(idx->n) : idx->n + 1;
    if (first > len || n > len - first) return MICA_EINVAL;
    if (n == 0) return 0;
    const DevBuf &b = which == 0 ? idx->sa_full : which == 1 ? idx->isa : idx->text;
    DeviceGuard g(idx->device);
    MICA_CUDA_TRY(cudaSetDevice(idx->device));
    MICA_CUDA_TRY(cudaMemcpy(out, (const uint32_t *)b.p + first, n * 4, cudaMemcpyDeviceToHost));
    return 0;
}
