// Merge step of the entry-range sharded search.
//
// The exact maximum of Theorem 1 is associative: with the database cut into
// contiguous entry ranges, one per GPU, each GPU's exact answer over its range
// (binary64 similarity, index) is a candidate, and the lexicographic maximum of
// the candidates -- similarity descending, global index ascending, the tie rule
// of Theorem 2 -- is the answer over the whole database.  For the top-k form each
// shard contributes its own k best in that order and the merge keeps the k best
// of the union.  After an all-gather of the per-shard results (nq * k * 16 bytes
// per shard) every rank can merge; the kernel merges device-resident results, the
// host function the same data in host memory (for a gather through host buffers).
#include <algorithm>

#include "hn_internal.cuh"

namespace hn {

// (s, i) comes before (s2, i2) in the answer order; i < 0 marks an empty slot
__host__ __device__ inline bool merge_before(double s, int64_t i, double s2, int64_t i2) {
    if (i < 0) return false;
    if (i2 < 0) return true;
    return s > s2 || (s == s2 && i < i2);
}

// One query: k rounds, each taking the best head among the shards' sorted lists.
__host__ __device__ inline void merge_one(const int64_t *idx, const double *sim, const int64_t *off, int32_t shards,
                                          int64_t nq, int32_t k, int64_t j, int64_t *out_idx, double *out_sim) {
    int32_t head[64];
    for (int32_t r = 0; r < shards; ++r) head[r] = 0;
    for (int32_t t = 0; t < k; ++t) {
        int32_t br = -1;
        double bs = 0.0;
        int64_t bi = -1;
        for (int32_t r = 0; r < shards; ++r) {
            if (head[r] >= k) continue;
            const int64_t p = ((int64_t)r * nq + j) * k + head[r];
            const int64_t li = idx[p];
            const int64_t gi = li < 0 ? -1 : li + off[r];
            if (merge_before(sim[p], gi, bs, bi)) {
                br = r;
                bs = sim[p];
                bi = gi;
            }
        }
        if (br >= 0) ++head[br];
        out_idx[j * k + t] = bi;
        out_sim[j * k + t] = bi >= 0 ? bs : -INFINITY;
    }
}

__global__ void k_merge_topk(const int64_t *__restrict__ idx, const double *__restrict__ sim,
                             const int64_t *__restrict__ off, int32_t shards, int64_t nq, int32_t k,
                             int64_t *__restrict__ out_idx, double *__restrict__ out_sim) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nq) merge_one(idx, sim, off, shards, nq, k, j, out_idx, out_sim);
}

static hn_status merge_args(const void *idx, const void *sim, const void *off, int32_t shards, int64_t nq, int32_t k,
                            const void *out_idx, const void *out_sim) {
    if (shards < 1 || shards > 64) return fail(HN_ERR_INVALID_ARG, "need 1 <= n_shards <= 64");
    if (nq < 0 || k < 1 || k > 32) return fail(HN_ERR_INVALID_ARG, "need nq >= 0 and 1 <= k <= 32");
    if (nq > 0 && (!idx || !sim || !off || !out_idx || !out_sim)) return fail(HN_ERR_INVALID_ARG, "NULL pointer");
    return HN_OK;
}

}  // namespace hn

using namespace hn;

extern "C" hn_status hn_merge_topk(const int64_t *idx, const double *sim, const int64_t *id_offset, int32_t n_shards,
                                   int64_t nq, int32_t k, int64_t *out_idx, double *out_sim, void *stream) {
    hn_status st = merge_args(idx, sim, id_offset, n_shards, nq, k, out_idx, out_sim);
    if (st != HN_OK || nq == 0) return st;
    k_merge_topk<<<(unsigned)((nq + 255) / 256), 256, 0, (cudaStream_t)stream>>>(idx, sim, id_offset, n_shards, nq, k,
                                                                              out_idx, out_sim);
    HN_CUDA(cudaGetLastError());
    return HN_OK;
}

extern "C" hn_status hn_merge_topk_host(const int64_t *idx, const double *sim, const int64_t *id_offset,
                                        int32_t n_shards, int64_t nq, int32_t k, int64_t *out_idx, double *out_sim) {
    hn_status st = merge_args(idx, sim, id_offset, n_shards, nq, k, out_idx, out_sim);
    if (st != HN_OK) return st;
    for (int64_t j = 0; j < nq; ++j) merge_one(idx, sim, id_offset, n_shards, nq, k, j, out_idx, out_sim);
    return HN_OK;
}
