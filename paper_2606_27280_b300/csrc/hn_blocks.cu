// Block partition of the database for the learned proposal.
//
// The proposal (an extension that seeds Algorithm 1's threshold) predicts
// which block of the database holds a query's nearest neighbour.  Blocks are
// made here, at index build time:
//   1. B centres: entries at positions floor(c*N/B), major prefix scaled to unit
//      length (spherical k-means on the K-dim prefixes, which is all the network sees);
//   2. Lloyd iterations: assign every entry to the centre of largest prefix
//      inner product (the streaming scan's Phase-1 argmax, ties to the lower
//      centre), then centre = normalised mean of its members.  Member sums are
//      accumulated in 2^-30 fixed point with int64 atomics, so the result does
//      not depend on the order of the atomics;
//   3. entries sorted by (nearest centre, entry id) -- a bitonic sort of 64-bit
//      keys -- and cut into B equal contiguous blocks:
//      block b = sorted positions [floor(b*N/B), floor((b+1)*N/B)).
// The index keeps the sorted ids (block_ids), the block starts and block_of[entry].
#include <math.h>

#include <vector>

#include "hn_internal.cuh"

namespace hn {

constexpr double kFix = 1073741824.0;  // 2^30

__global__ void k_centres_init(const float *__restrict__ rows, int64_t n, int k, int kp, int B,
                               float *__restrict__ cen) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    const int64_t e = (int64_t)c * n / B;
    double s = 0;
    for (int d = 0; d < k; ++d) s += (double)rows[e * kD + d] * rows[e * kD + d];
    const double inv = s > 0 ? 1.0 / sqrt(s) : 0.0;
    for (int d = 0; d < kp; ++d) cen[(int64_t)c * kp + d] = d < k ? (float)(rows[e * kD + d] * inv) : 0.f;
}

__global__ void k_prefix_f32(const float *__restrict__ rows, int64_t n, int k, int kp, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * kp) return;
    const int64_t e = i / kp;
    const int d = (int)(i % kp);
    out[i] = d < k ? rows[e * kD + d] : 0.f;
}

__global__ void k_centre_accumulate(const float *__restrict__ pre, int64_t n, int kp,
                                    const unsigned long long *__restrict__ key, long long *__restrict__ sums,
                                    int *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = best_idx(key[i]);
    for (int d = 0; d < kp; ++d)
        atomicAdd(reinterpret_cast<unsigned long long *>(sums + (int64_t)c * kp + d),
                  (unsigned long long)llrint((double)pre[i * kp + d] * kFix));
    atomicAdd(cnt + c, 1);
}

__global__ void k_centre_update(const long long *__restrict__ sums, const int *__restrict__ cnt, int B, int kp,
                                float *__restrict__ cen) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B || cnt[c] == 0) return;  // an empty cluster keeps its centre
    double s = 0;
    for (int d = 0; d < kp; ++d) {
        const double v = (double)sums[(int64_t)c * kp + d];
        s += v * v;
    }
    if (s == 0) return;
    const double inv = 1.0 / sqrt(s);
    for (int d = 0; d < kp; ++d) cen[(int64_t)c * kp + d] = (float)((double)sums[(int64_t)c * kp + d] * inv);
}

__global__ void k_sort_keys(const unsigned long long *__restrict__ key, int64_t n, int64_t n2,
                            unsigned long long *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    out[i] = i < n ? (((unsigned long long)best_idx(key[i])) << 32) | (unsigned long long)i : ~0ull;
}

// One compare-exchange pass of a bitonic sorting network (ascending).
__global__ void k_bitonic_pass(unsigned long long *__restrict__ a, int64_t n2, int64_t j, int64_t k) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const int64_t p = i ^ j;
    if (p <= i) return;
    const unsigned long long x = a[i], y = a[p];
    const bool up = (i & k) == 0;
    if ((x > y) == up) {
        a[i] = y;
        a[p] = x;
    }
}

// All passes with j < 2048 of one stage k, inside shared memory (2048 keys per CTA).
__global__ void __launch_bounds__(1024) k_bitonic_local(unsigned long long *__restrict__ a, int64_t n2, int64_t k,
                                                        int64_t j0) {
    __shared__ unsigned long long s[2048];
    const int64_t base = (int64_t)blockIdx.x * 2048;
    s[threadIdx.x] = a[base + threadIdx.x];
    s[threadIdx.x + 1024] = a[base + threadIdx.x + 1024];
    __syncthreads();
    for (int64_t j = j0; j > 0; j >>= 1) {
        for (int r = 0; r < 2; ++r) {
            const int64_t li = threadIdx.x + r * 1024;
            const int64_t lp = li ^ j;
            if (lp > li) {
                const bool up = ((base + li) & k) == 0;
                const unsigned long long x = s[li], y = s[lp];
                if ((x > y) == up) {
                    s[li] = y;
                    s[lp] = x;
                }
            }
        }
        __syncthreads();
    }
    a[base + threadIdx.x] = s[threadIdx.x];
    a[base + threadIdx.x + 1024] = s[threadIdx.x + 1024];
}

cudaError_t bitonic_sort(unsigned long long *a, int64_t n2, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n2 + 255) / 256);
    for (int64_t k = 2; k <= n2; k <<= 1) {
        int64_t j = k >> 1;
        for (; j >= 2048 || (j > 0 && n2 < 2048); j >>= 1) {
            k_bitonic_pass<<<blocks, 256, 0, st>>>(a, n2, j, k);
        }
        if (j > 0) k_bitonic_local<<<(unsigned)(n2 / 2048), 1024, 0, st>>>(a, n2, k, j);
    }
    return cudaGetLastError();
}

__global__ void k_blocks_from_sorted(const unsigned long long *__restrict__ sorted, int64_t n, int B,
                                     int32_t *__restrict__ block_ids, int32_t *__restrict__ block_of) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t e = (int32_t)(sorted[p] & 0xFFFFFFFFull);
    block_ids[p] = e;
    block_of[e] = (int32_t)(((p + 1) * B - 1) / n);  // largest b with floor(b*n/B) <= p
}

__global__ void k_block_starts(int64_t n, int B, int32_t *__restrict__ start) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b <= B) start[b] = (int32_t)((int64_t)b * n / B);
}

// Streaming-scan Phase 1 with explicit arrays (defined in hn_search.cu).
cudaError_t stream_argmax_f32(const float *db_pre, int64_t n_db, int64_t n_db_tiles, int kp, const float *q_pre,
                              int64_t nq, unsigned long long *keys, cudaStream_t st);

cudaError_t build_blocks(Index &ix, int B, int iters, cudaStream_t st) {
    const int64_t n = ix.n;
    const int kp = ix.k_pad4;
    const int64_t ct = (B + kTileE - 1) / kTileE;  // centre tiles
    float *cen = nullptr, *pre = nullptr;
    long long *sums = nullptr;
    int *cnt = nullptr;
    unsigned long long *key = nullptr, *sorted = nullptr;
    int64_t n2 = 2048;
    while (n2 < n) n2 <<= 1;
    cudaError_t e = cudaMalloc(&cen, sizeof(float) * ct * kTileE * kp);
    if (e == cudaSuccess) e = cudaMemsetAsync(cen, 0, sizeof(float) * ct * kTileE * kp, st);
    if (e == cudaSuccess) e = cudaMalloc(&sums, sizeof(long long) * B * kp);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(int) * B);
    if (e == cudaSuccess) e = cudaMalloc(&key, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&sorted, sizeof(unsigned long long) * n2);
    if (e == cudaSuccess && ix.pre32 == nullptr) e = cudaMalloc(&pre, sizeof(float) * n * kp);
    const float *prefix = ix.pre32 ? ix.pre32 : pre;
    if (e == cudaSuccess && pre) k_prefix_f32<<<(unsigned)((n * kp + 255) / 256), 256, 0, st>>>(ix.rows, n, ix.k, kp, pre);
    if (e == cudaSuccess) k_centres_init<<<(B + 127) / 128, 128, 0, st>>>(ix.rows, n, ix.k, kp, B, cen);
    for (int it = 0; e == cudaSuccess && it <= iters; ++it) {
        e = cudaMemsetAsync(key, 0, sizeof(unsigned long long) * n, st);
        if (e == cudaSuccess) e = stream_argmax_f32(cen, B, ct, kp, prefix, n, key, st);
        if (e != cudaSuccess || it == iters) break;
        e = cudaMemsetAsync(sums, 0, sizeof(long long) * B * kp, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int) * B, st);
        if (e == cudaSuccess) {
            k_centre_accumulate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(prefix, n, kp, key, sums, cnt);
            k_centre_update<<<(B + 127) / 128, 128, 0, st>>>(sums, cnt, B, kp, cen);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        k_sort_keys<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(key, n, n2, sorted);
        e = bitonic_sort(sorted, n2, st);
    }
    if (e == cudaSuccess) e = cudaMalloc(&ix.block_ids, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&ix.block_of, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&ix.block_start, sizeof(int32_t) * (B + 1));
    if (e == cudaSuccess) {
        k_blocks_from_sorted<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sorted, n, B, ix.block_ids, ix.block_of);
        k_block_starts<<<(B + 256) / 256, 256, 0, st>>>(n, B, ix.block_start);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(cen);
    cudaFree(pre);
    cudaFree(sums);
    cudaFree(cnt);
    cudaFree(key);
    cudaFree(sorted);
    if (e == cudaSuccess) ix.n_blocks = B;
    return e;
}

}  // namespace hn
