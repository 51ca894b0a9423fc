// hn_bruteforce_static: the FP32 brute-force scan with its per-query scratch
// in a fixed, library-owned device array instead of memory the library
// allocates on demand.
//
// Who needs this: callers that must not allocate device memory while they
// answer queries -- a latency-critical serving thread (cudaMalloc can block
// and implicitly synchronise the device), a process whose device memory is
// handed out by another framework's allocator or capped by a fixed budget, or
// a deployment whose rules forbid dynamic allocation after initialisation.
// They still pass their own queries and output buffers; the scratch below is
// the only other memory the call touches.
#include <mutex>

#include <cuda.h>

#include "hn_internal.cuh"

namespace hn {

// One 8-byte (score, index) key per query.  Every GPU that loads the library
// holds this array (512 KiB) until the process exits.
static __device__ __align__(256) unsigned long long g_static_keys[HN_STATIC_MAX_QUERIES];

constexpr int kMaxDevices = 64;
struct StaticSlot {
    unsigned long long ctx_id = 0;   // the CUDA context the address belongs to (0: none yet)
    unsigned long long *addr = nullptr;
};
static StaticSlot g_static_slot[kMaxDevices];
static std::mutex g_static_mu;

// Unique id of the current CUDA context (driver entry points looked up once through the
// runtime, so the library does not link the driver library); 0 if unavailable.
static unsigned long long current_ctx_id() {
    typedef CUresult (*GetCurrent)(CUcontext *);
    typedef CUresult (*GetId)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult r1, r2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &r1) == cudaSuccess &&
            r1 == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &r2) == cudaSuccess &&
            r2 == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(g);
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_static_keys in the current context.  In host code the symbol is
// only a host-side stand-in, so the address is looked up with the device current and
// cached per device together with the context's unique id: after a device reset (a new
// primary context) the id differs and the address is looked up again.
static hn_status static_keys(unsigned long long **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(HN_ERR_UNSUPPORTED, "device ordinal out of range");
    // 0 when this thread has no current context yet: then the address is looked up, which
    // also makes the device's primary context current for the next call
    const unsigned long long id = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticSlot &slot = g_static_slot[dev];
    if (!slot.addr || id == 0 || slot.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_keys);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_keys)");
        slot.addr = static_cast<unsigned long long *>(p);
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return HN_OK;
}

}  // namespace hn

using namespace hn;

extern "C" hn_status hn_bruteforce_static(const hn_index *index, const float *q, int64_t nq, int64_t *out_idx,
                                          double *out_sim, void *stream) {
    if (!index) return fail(HN_ERR_INVALID_ARG, "index is NULL");
    if (nq < 0) return fail(HN_ERR_INVALID_ARG, "nq < 0");
    if (nq > HN_STATIC_MAX_QUERIES)
        return fail(HN_ERR_INVALID_ARG, "nq exceeds HN_STATIC_MAX_QUERIES (65536): split the batch");
    if (nq == 0) return HN_OK;
    if (!q || !out_idx || !out_sim || ((uintptr_t)q & 15u)) return fail(HN_ERR_INVALID_ARG, "null or unaligned pointer");
    unsigned long long *keys = nullptr;
    hn_status st = static_keys(&keys);
    if (st != HN_OK) return st;
    HN_CUDA(launch_bruteforce_keys(*index_state(index), q, nq, keys, out_idx, out_sim, (cudaStream_t)stream));
    return HN_OK;
}
