// Self-test of the bounded device-side wait that every mbarrier wait of the dense
// scan uses (the paper has no counterpart).  One warp waits on an mbarrier that
// nothing ever arrives on; the wait must give up after `limit_ns` of global time,
// raise the shared abort flag and let the kernel return normally, so that the host
// reads HN_ERR_TIMEOUT from the status word and the context stays usable.
#include "hn_internal.cuh"
#include "hn_sm100.cuh"

namespace hn {
using namespace sm100;

__global__ void k_wait_selftest(uint64_t limit_ns, int32_t *status) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    // phase 0 of `bar` never completes: no thread arrives on it
    const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag, limit_ns);
    __syncthreads();
    if (threadIdx.x == 0) {
        status[0] = ok ? 0 : 1;
        status[1] = abort_flag;
    }
}

}  // namespace hn

using namespace hn;

extern "C" hn_status hn_selftest_wait_timeout(uint64_t limit_ns, void *stream) {
    if (limit_ns < 1000 || limit_ns > 10000000000ull)
        return fail(HN_ERR_INVALID_ARG, "need 1 us <= limit_ns <= 10 s");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *dstat = nullptr;
    HN_CUDA(cudaMallocAsync((void **)&dstat, 2 * sizeof(int32_t), s));
    int32_t h[2] = {-1, -1};
    cudaError_t e = cudaMemsetAsync(dstat, 0, 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, dstat);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, dstat, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dstat, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "hn_selftest_wait_timeout");
    if (h[0] == 1 && h[1] == 1) return fail(HN_ERR_TIMEOUT, "the bounded wait gave up as intended");
    return HN_OK;  // the wait completed: the mechanism did not fire
}
