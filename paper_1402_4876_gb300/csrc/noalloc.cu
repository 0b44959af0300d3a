// Hit-list offsets without any device allocation.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is
// being captured, services whose device memory is owned by another
// framework's allocator or pool, and hosts that must keep their memory
// footprint fixed after start-up.  For them this file offers one entry point
// that turns per-read hit counts into the CSR offsets of the hit lists (the
// prefix-sum step of the search path) using a scratch array that exists from
// the moment the library's module is loaded on a device, instead of a buffer
// allocated per call.  The caller still passes the counts and the offsets.
#include <mutex>

#include "mica_internal.cuh"

namespace mica {
namespace {

// One tile sum per 2,048 counts, plus the grand total: 8,193 + 1 entries
// (64 KiB) for the maximum of MICA_NOALLOC_MAX_COUNTS counts per call.  Every
// GPU that loads the library holds this array until the process exits.
constexpr uint64_t NOALLOC_TILE = 2048;
constexpr uint64_t NOALLOC_SCRATCH = MICA_NOALLOC_MAX_COUNTS / NOALLOC_TILE + 2;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_SCRATCH];

// The array's device address, looked up once per device and context with
// that device current (in host code the symbol's name is only a host-side
// stand-in).  A device reset destroys the context and the module with it; the
// context that replaces it has a new id, so the address is looked up again.
constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
struct ScratchAddr {
    unsigned long long ctx_id = 0;   // 0: not looked up yet (context ids start at 1)
    unsigned long long *ptr = nullptr;
};
ScratchAddr g_noalloc_addr[MAX_DEVICES];

// Id of the calling thread's current context, through the driver's entry
// points (the library links only the runtime).
typedef int (*ctx_get_current_fn)(void **);
typedef int (*ctx_get_id_fn)(void *, unsigned long long *);

int current_context_id(unsigned long long *id)
{
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess || qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess) {
            if (e == cudaSuccess) e = cudaErrorNotSupported;
            set_last_cuda_error(e, "cudaGetDriverEntryPointByVersion(cuCtxGetCurrent, cuCtxGetId)", __FILE__, __LINE__);
            return MICA_ECUDA;
        }
        get_current = (ctx_get_current_fn)a;
        get_id = (ctx_get_id_fn)b;
    }
    void *ctx = nullptr;
    *id = 0;
    if (get_current(&ctx) != 0 || (ctx && get_id(ctx, id) != 0)) {
        set_last_cuda_error(cudaErrorDeviceUninitialized, "cuCtxGetCurrent / cuCtxGetId", __FILE__, __LINE__);
        return MICA_ECUDA;
    }
    return 0;   // *id stays 0 while the thread has no current context yet
}

int noalloc_scratch(int device, unsigned long long **out)
{
    if (device < 0 || device >= MAX_DEVICES) return MICA_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned long long ctx = 0;
    if (int rc = current_context_id(&ctx)) return rc;
    ScratchAddr &a = g_noalloc_addr[device];
    if (ctx == 0 || a.ctx_id != ctx || !a.ptr) {
        // the lookup makes the device's primary context current if no
        // context was yet, so the id is read after it
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            return MICA_ECUDA;
        }
        if (ctx == 0) {
            if (int rc = current_context_id(&ctx)) return rc;
            if (ctx == 0) {
                set_last_cuda_error(cudaErrorDeviceUninitialized, "no current context after the lookup", __FILE__, __LINE__);
                return MICA_ECUDA;
            }
        }
        a.ptr = (unsigned long long *)p;
        a.ctx_id = ctx;
    }
    *out = a.ptr;
    return 0;
}

}  // namespace
}  // namespace mica

extern "C" int mica_offsets_noalloc(const uint64_t *d_counts, uint64_t n, uint64_t *d_offsets, void *cuda_stream)
{
    if (!d_offsets || (n && !d_counts)) return MICA_EINVAL;
    if (n > MICA_NOALLOC_MAX_COUNTS) return MICA_EINVAL;   // the scratch array has room for no more
    int dev = 0;
    MICA_CUDA_TRY(cudaGetDevice(&dev));
    unsigned long long *scratch = nullptr;
    if (int rc = mica::noalloc_scratch(dev, &scratch)) return rc;
    // every tile sum and the grand total are written before they are read,
    // so nothing left from an earlier call needs clearing
    return mica::exclusive_scan_u64_scratch(d_counts, n, d_offsets, scratch, (cudaStream_t)cuda_stream);
}
