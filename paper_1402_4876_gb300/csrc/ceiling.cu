// Random-gather ceiling: the rate at which this GPU serves independent random
// loads of one occurrence-block size from a buffer of a given size.
//
// The paper names access to the index in memory as the bottleneck of the BWT
// phase once reads are short (Section 3), and the search here is a chain of
// dependent random 32-byte block reads.  A copy benchmark measures streaming
// bandwidth, which random sector reads cannot reach; this kernel measures
// the practical ceiling for the access pattern the search actually makes, so
// the search's achieved bytes/s can be stated as a fraction of it.  With a
// buffer well above L2 (129 MB) the loads are served by HBM; with a buffer
// the size of a small index they are mostly L2 hits.
#include "mica_internal.cuh"

namespace mica {
namespace {

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): a counter-based mix, so every load address is
// independent of every loaded value and many loads stay in flight.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Each thread makes `iters` loads of VEC x 16 bytes at uniformly random
// unit-aligned offsets; the XOR of what was read goes to `sink` only if it
// equals an unlikely value, which keeps the loads without a store per thread.
template <int VEC>
__global__ void __launch_bounds__(256) k_gather(const uint4 *__restrict__ buf, uint64_t n_units, uint32_t iters,
                                               uint64_t seed, unsigned int *sink)
{
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
#pragma unroll 8
    for (uint32_t it = 0; it < iters; it++) {
        uint64_t z = splitmix64(seed ^ (t * 0x100000001B3ull + it));
        uint64_t u = __umul64hi(z, n_units);   // uniform in [0, n_units)
        const uint4 *p = buf + u * VEC;
#pragma unroll
        for (int v = 0; v < VEC; v++) {
            uint4 q = __ldg(p + v);
            acc ^= q.x ^ q.y ^ q.z ^ q.w;
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);
}

__global__ void k_fill(uint4 *buf, uint64_t n)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        buf[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 32) ^ 0x5bd1e995u, (uint32_t)(i * 2654435761u), 7u);
}

}  // namespace
}  // namespace mica

using namespace mica;

extern "C" {

int mica_gather_ceiling(int device, uint64_t buffer_bytes, uint32_t load_bytes, uint64_t loads, uint32_t repeats,
                        double *gbs, double *ms)
{
    if (!gbs || (load_bytes != 16 && load_bytes != 32 && load_bytes != 64 && load_bytes != 128)) return MICA_EINVAL;
    if (buffer_bytes < 4096 || buffer_bytes % load_bytes || loads == 0) return MICA_EINVAL;
    if (repeats == 0) repeats = 1;
    DeviceGuard g(device);
    MICA_CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    MICA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    DevBuf buf, sink;
    int rc = dev_reserve(buf, buffer_bytes);
    if (!rc) rc = dev_reserve(sink, 16);
    if (rc) { dev_release(buf); dev_release(sink); return rc; }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    const uint32_t threads = 256;
    // 8 resident CTAs of 256 threads per SM: 64 warps, the SM's maximum
    const uint64_t grid = (uint64_t)sms * 8;
    const uint64_t per_launch = grid * threads;
    const uint32_t iters = (uint32_t)std::max<uint64_t>(1, (loads + per_launch - 1) / per_launch);
    const uint64_t n_units = buffer_bytes / load_bytes;
    auto launch = [&](uint64_t seed) {
        const uint4 *b = (const uint4 *)buf.p;
        unsigned int *s = (unsigned int *)sink.p;
        switch (load_bytes) {
        case 16: k_gather<1><<<(unsigned)grid, threads>>>(b, n_units, iters, seed, s); break;
        case 32: k_gather<2><<<(unsigned)grid, threads>>>(b, n_units, iters, seed, s); break;
        case 64: k_gather<4><<<(unsigned)grid, threads>>>(b, n_units, iters, seed, s); break;
        default: k_gather<8><<<(unsigned)grid, threads>>>(b, n_units, iters, seed, s); break;
        }
    };
    {
        cudaError_t e = cudaSuccess;
        k_fill<<<sms * 4, 256>>>((uint4 *)buf.p, buffer_bytes / 16);
        if ((e = cudaGetLastError()) == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        for (uint32_t r = 0; e == cudaSuccess && r <= repeats; r++) {
            launch(0x243F6A8885A308D3ull + r);   // the first launch warms up
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if (r == 0) { e = cudaDeviceSynchronize(); continue; }
            if ((e = cudaEventRecord(e0)) != cudaSuccess) break;
            launch(0x13198A2E03707344ull + r);
            if ((e = cudaEventRecord(e1)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float t = 0.f;
            if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
            best = std::min(best, t);
        }
        if (e != cudaSuccess) { set_last_cuda_error(e, "gather ceiling", __FILE__, __LINE__); rc = MICA_ECUDA; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_release(buf);
    dev_release(sink);
    if (rc) return rc;
    double bytes = (double)per_launch * iters * load_bytes;
    *gbs = bytes / (best * 1e-3) / 1e9;
    if (ms) *ms = best;
    return 0;
}

}  // extern "C"
