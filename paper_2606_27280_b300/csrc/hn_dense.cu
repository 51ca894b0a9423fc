// tcgen05 dense prefix scan (placeholder until the tensor-core kernel lands).
#include "hn_internal.cuh"

namespace hn {
bool dense_scan_supported(const Index &) { return false; }
cudaError_t launch_dense_scan(const Index &, int64_t, int, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace hn
