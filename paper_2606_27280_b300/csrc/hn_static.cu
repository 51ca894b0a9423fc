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

#include "hn_internal.cuh"

namespace hn {

// One 8-byte (score, index) key per query.  Every GPU that loads the library
// holds this array (512 KiB) until the process exits.
static __device__ __align__(256) unsigned long long g_static_keys[HN_STATIC_MAX_QUERIES];

constexpr int kMaxDevices = 64;
static unsigned long long *g_static_addr[kMaxDevices] = {};
static std::mutex g_static_mu;

// Device address of g_static_keys on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and cached.
static hn_status static_keys(unsigned long long **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(HN_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_keys);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_keys)");
        g_static_addr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_static_addr[dev];
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
