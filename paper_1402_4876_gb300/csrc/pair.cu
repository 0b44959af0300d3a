// Mate pairing of a paired-end batch (the paper reports properly paired
// reads, Section 3, Table 1): for pair i (reads 2i and 2i + 1), every listed
// + strand hit of one mate against every listed - strand hit of the other
// whose fragment length b.pos + m_b - a.pos lies in the insert window.
//
// One thread per pair.  A read's hits are sorted by (pos, strand), so for a
// + strand hit a the - strand partners form one contiguous position range
// of the other mate's list: a binary search finds its start and a scan
// counts the partners and keeps the best (fewest substitutions, then the
// tie order of mica_pair).
#include "mica_internal.cuh"

namespace mica {
namespace {

struct Best {
    uint32_t n = 0, nbest = 0, mm = 0xffu, pp = 0, pm = 0, mate = 0;
};

// Offer combination (a = + strand hit of `amate`, b = - strand hit).
__device__ __forceinline__ void offer(Best &B, uint32_t mm, uint32_t pp, uint32_t amate, uint32_t pm)
{
    B.n = B.n == 0xffffffffu ? B.n : B.n + 1;
    bool better = mm < B.mm || (mm == B.mm && (pp < B.pp || (pp == B.pp && (amate < B.mate ||
                                                                              (amate == B.mate && pm < B.pm)))));
    if (mm < B.mm) B.nbest = 1;
    else if (mm == B.mm) B.nbest++;
    if (better) { B.mm = mm; B.pp = pp; B.pm = pm; B.mate = amate; }
}

// + strand hits of mate `amate` (list A) against - strand hits of the other
// mate (list Bl, its read length mb).
__device__ __forceinline__ void pair_lists(const Hit *A, uint64_t na, const Hit *Bl, uint64_t nb, uint32_t mb,
                                           uint32_t lmin, uint32_t lmax, uint32_t amate, Best &B)
{
    for (uint64_t i = 0; i < na; i++) {
        Hit a = A[i];
        if (a.strand != 0) continue;
        // partner positions p with lmin <= p + mb - a.pos <= lmax
        long long lo = (long long)a.pos + (long long)lmin - (long long)mb;
        long long hi = (long long)a.pos + (long long)lmax - (long long)mb;
        if (hi < 0) continue;
        uint32_t lo32 = lo < 0 ? 0u : (uint32_t)lo;
        uint64_t L = 0, R = nb;   // first hit with pos >= lo32
        while (L < R) {
            uint64_t M = (L + R) >> 1;
            if (Bl[M].pos < lo32) L = M + 1;
            else R = M;
        }
        for (uint64_t j = L; j < nb && (long long)Bl[j].pos <= hi; j++) {
            Hit b = Bl[j];
            if (b.strand == 1) offer(B, (uint32_t)a.mm + b.mm, a.pos, amate, b.pos);
        }
    }
}

__global__ void k_pair(const uint64_t *__restrict__ off, const Hit *__restrict__ hits,
                       const uint16_t *__restrict__ len, uint64_t n_pairs, uint32_t lmin, uint32_t lmax,
                       mica_pair *__restrict__ out)
{
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n_pairs;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r1 = 2 * p, r2 = 2 * p + 1;
        const uint64_t b1 = off[r1], e1 = off[r1 + 1], b2 = off[r2], e2 = off[r2 + 1];
        Best B;
        pair_lists(hits + b1, e1 - b1, hits + b2, e2 - b2, len[r2], lmin, lmax, 0, B);
        pair_lists(hits + b2, e2 - b2, hits + b1, e1 - b1, len[r1], lmin, lmax, 1, B);
        mica_pair o;
        o.n_concordant = B.n;
        o.n_best = B.n ? B.nbest : 0;
        o.pos_plus = B.n ? B.pp : 0;
        o.pos_minus = B.n ? B.pm : 0;
        o.plus_mate = (uint8_t)(B.n ? B.mate : 0);
        o.mm = (uint8_t)(B.n ? B.mm : 0);
        o.pad = 0;
        out[p] = o;
    }
}

}  // namespace
}  // namespace mica

using namespace mica;

extern "C" {

int mica_pair_device(const uint64_t *d_offsets, const mica_hit *d_hits, const uint16_t *d_lengths,
                     uint64_t n_pairs, uint32_t insert_min, uint32_t insert_max, mica_pair *d_out,
                     void *cuda_stream)
{
    if (insert_min > insert_max) return MICA_EINVAL;
    if (n_pairs == 0) return 0;
    if (!d_offsets || !d_hits || !d_lengths || !d_out) return MICA_EINVAL;
    unsigned g = (unsigned)std::min<uint64_t>((n_pairs + 127) / 128, 152ull * 32);
    k_pair<<<g, 128, 0, (cudaStream_t)cuda_stream>>>(d_offsets, (const Hit *)d_hits, d_lengths, n_pairs,
                                                      insert_min, insert_max, d_out);
    MICA_CUDA_TRY(cudaGetLastError());
    return 0;
}

int mica_pair_batch(int device, const uint64_t *offsets, const mica_hit *hits, const uint16_t *lengths,
                    uint64_t n_pairs, uint32_t insert_min, uint32_t insert_max, mica_pair *out)
{
    if (insert_min > insert_max) return MICA_EINVAL;
    if (n_pairs == 0) return 0;
    if (!offsets || !lengths || !out) return MICA_EINVAL;
    const uint64_t n_reads = 2 * n_pairs, nh = offsets[n_reads];
    if (nh && !hits) return MICA_EINVAL;
    for (uint64_t r = 0; r < n_reads; r++)
        if (offsets[r] > offsets[r + 1]) return MICA_EINVAL;
    DeviceGuard g(device);
    MICA_CUDA_TRY(cudaSetDevice(device));
    DevBuf doff, dhits, dlen, dout;
    int rc = dev_reserve(doff, (n_reads + 1) * 8);
    if (!rc) rc = dev_reserve(dhits, std::max<uint64_t>(nh, 1) * sizeof(mica_hit));
    if (!rc) rc = dev_reserve(dlen, n_reads * 2);
    if (!rc) rc = dev_reserve(dout, n_pairs * sizeof(mica_pair));
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaMemcpy(doff.p, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice);
    if (!rc && e == cudaSuccess && nh) e = cudaMemcpy(dhits.p, hits, nh * sizeof(mica_hit), cudaMemcpyHostToDevice);
    if (!rc && e == cudaSuccess) e = cudaMemcpy(dlen.p, lengths, n_reads * 2, cudaMemcpyHostToDevice);
    if (!rc && e != cudaSuccess) { set_last_cuda_error(e, "pair upload", __FILE__, __LINE__); rc = MICA_ECUDA; }
    if (!rc) rc = mica_pair_device((const uint64_t *)doff.p, (const mica_hit *)dhits.p, (const uint16_t *)dlen.p,
                                   n_pairs, insert_min, insert_max, (mica_pair *)dout.p, nullptr);
    if (!rc) {
        e = cudaMemcpy(out, dout.p, n_pairs * sizeof(mica_pair), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { set_last_cuda_error(e, "pair download", __FILE__, __LINE__); rc = MICA_ECUDA; }
    }
    dev_release(doff);
    dev_release(dhits);
    dev_release(dlen);
    dev_release(dout);
    return rc;
}

}  // extern "C"
