// Learned block proposal: a small MLP trained and run by this library's own
// kernels (an extension of the method; the paper has no network here).
//
//   x  = query major prefix (K values)
//   a1 = W1 x + b1, h1 = gelu(a1);  a2 = W2 h1 + b2, h2 = gelu(a2);  z = W3 h2 + b3
//   loss = mean_j logsumexp(z_j) - z_j[y_j]      (y_j = block of the exact NN)
//   gelu(a) = 0.5 a (1 + erf(a / sqrt 2))
// Training: FP32 master weights, FP32 arithmetic, Adam.  Inference: weights
// rounded to BF16 values (kept as FP32 numbers), FP32 accumulation, top-k
// blocks by (score desc, block asc).  Parameter layout (also the save format):
//   [W1 (H1 x K), b1 (H1), W2 (H2 x H1), b2 (H2), W3 (C x H2), b3 (C)], row-major.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "hn_internal.cuh"

namespace hn {

// ------------------------------------------------------------------ GEMM
// C(i,j) = sum_k A(i,k) B(k,j) [+ beta C(i,j)], A(i,k) = A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj],
// then optionally + bias[j] and an activation (ACT 1 = gelu, storing the pre-activation).
// 64 x 64 tile, 16-deep K slices in shared memory, 4 x 4 outputs per thread, FP32 FMA.
constexpr int GBM = 64, GBN = 64, GBK = 16;

__device__ inline float gelu_f(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }
__device__ inline float gelu_grad_f(float a) {
    return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}

__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float *__restrict__ A, int64_t sai,
                                              int64_t sak, const float *__restrict__ B, int64_t sbk, int64_t sbj,
                                              float *__restrict__ C, int64_t ldc, float beta,
                                              const float *__restrict__ bias, int act, float *__restrict__ pre) {
    __shared__ float As[GBK][GBM + 4];
    __shared__ __align__(16) float Bs[GBK][GBN + 4];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int i0 = blockIdx.y * GBM, j0 = blockIdx.x * GBN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;
            int ii, kk;
            if (sak == 1) { kk = e % GBK; ii = e / GBK; } else { ii = e % GBM; kk = e / GBM; }
            const int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < K) ? A[gi * sai + gk * sak] : 0.f;
            int jj, kb;
            if (sbj == 1) { jj = e % GBN; kb = e / GBN; } else { kb = e % GBK; jj = e / GBK; }
            const int gj = j0 + jj, gkb = k0 + kb;
            Bs[kb][jj] = (gj < N && gkb < K) ? B[gkb * sbk + gj * sbj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            b[0] = bv.x; b[1] = bv.y; b[2] = bv.z; b[3] = bv.w;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gi = i0 + ty * 4 + r;
        if (gi >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int gj = j0 + tx * 4 + c;
            if (gj >= N) continue;
            float v = acc[r][c];
            if (beta != 0.f) v += beta * C[gi * ldc + gj];
            if (bias) v += bias[gj];
            if (act == 1) {
                if (pre) pre[gi * ldc + gj] = v;
                v = gelu_f(v);
            }
            C[gi * ldc + gj] = v;
        }
    }
}

static cudaError_t gemm(int M, int N, int K, const float *A, int64_t sai, int64_t sak, const float *B, int64_t sbk,
                        int64_t sbj, float *C, int64_t ldc, cudaStream_t st, float beta = 0.f,
                        const float *bias = nullptr, int act = 0, float *pre = nullptr) {
    if (M == 0 || N == 0) return cudaSuccess;
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    k_gemm<<<grid, 256, 0, st>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, beta, bias, act, pre);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ elementwise / reductions
// Softmax cross-entropy, one warp per row: row_loss[i] = lse(z_i) - z_i[y_i];
// dz = (softmax(z_i) - onehot(y_i)) * inv_b.
// z and dz may be the same array (no __restrict__ on them).
__global__ void k_softmax_xent(const float *z, const int32_t *__restrict__ y, int B, int C, float inv_b, float *dz,
                               float *__restrict__ row_loss) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= B) return;
    const float *zi = z + i * C;
    float m = -INFINITY;
    for (int c = lane; c < C; c += 32) m = fmaxf(m, zi[c]);
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    float s = 0.f;
    for (int c = lane; c < C; c += 32) s += expf(zi[c] - m);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int yi = y[i];
    const float zy = zi[yi];  // read before dz (which may alias z) is written
    __syncwarp();
    if (dz) {
        const float inv_s = 1.f / s;
        for (int c = lane; c < C; c += 32) dz[i * C + c] = (expf(zi[c] - m) * inv_s - (c == yi ? 1.f : 0.f)) * inv_b;
    }
    if (lane == 0) row_loss[i] = m + logf(s) - zy;
}

__global__ void k_gelu_back(const float *__restrict__ dh, const float *__restrict__ pre, int64_t n,
                            float *__restrict__ da) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) da[i] = dh[i] * gelu_grad_f(pre[i]);
}

// Column sums (bias gradients), one thread per column, rows summed in order.
__global__ void k_colsum(const float *__restrict__ a, int rows, int cols, float *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int i = 0; i < rows; ++i) s += a[(int64_t)i * cols + j];
    out[j] = s;
}

// Deterministic sum of n values by one block (fixed tree).
__global__ void k_sum(const float *__restrict__ a, int n, float *__restrict__ out) {
    __shared__ float s[256];
    float v = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) v += a[i];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_round_bf16(const float *__restrict__ a, int64_t n, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __bfloat162float(__float2bfloat16_rn(a[i]));
}

// x[i, :] = the first k coordinates of row src_row(i) of q (128 wide); optional label gather.
__global__ void k_gather_prefix(const float *__restrict__ q, const int32_t *__restrict__ rows_idx, int64_t nrows, int k,
                                 float *__restrict__ x, const int32_t *__restrict__ lab_in, int32_t *__restrict__ lab_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nrows * k) return;
    const int64_t i = t / k;
    const int d = (int)(t % k);
    const int64_t r = rows_idx ? rows_idx[i] : i;
    x[t] = q[r * kD + d];
    if (d == 0 && lab_out) lab_out[i] = lab_in[r];
}

// Top-k columns per row by (score desc, column asc), one warp per row.
__global__ void k_topk(const float *__restrict__ z, int64_t rows, int C, int topk, int32_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= rows) return;
    const float *zi = z + i * C;
    unsigned long long taken = ~0ull;
    for (int r = 0; r < topk; ++r) {
        unsigned long long km = 0;
        for (int c = lane; c < C; c += 32) {
            const unsigned long long kk = pack_best(zi[c], (uint32_t)c);
            if (kk < taken && kk > km) km = kk;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, km, o);
            km = other > km ? other : km;
        }
        taken = km;
        if (lane == 0) out[i * topk + r] = (int32_t)best_idx(km);
    }
}

// Labels: block of each training query's exact nearest neighbour.
__global__ void k_labels(const int64_t *__restrict__ nn, const int32_t *__restrict__ block_of, int64_t n,
                         int32_t *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = block_of[nn[i]];
}

// Epoch shuffle keys: (hash(seed, epoch, i) << 32) | i, sorted to a permutation.
__global__ void k_shuffle_keys(int64_t n, int64_t n2, uint64_t salt, unsigned long long *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    uint64_t h = salt ^ (0x9E3779B97F4A7C15ull * (uint64_t)(i + 1));  // splitmix64 finaliser
    h ^= h >> 30;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 27;
    h *= 0x94D049BB133111EBull;
    h ^= h >> 31;
    keys[i] = i < n ? ((h & 0xFFFFFFFF00000000ull) | (unsigned long long)i) : ~0ull;
}

__global__ void k_low32(const unsigned long long *__restrict__ keys, int64_t n, int32_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)(keys[i] & 0xFFFFFFFFull);
}

cudaError_t bitonic_sort(unsigned long long *a, int64_t n2, cudaStream_t st);

// ------------------------------------------------------------------ network state
struct Net {
    int k = 0, h1 = 0, h2 = 0, c = 0;
    int64_t np = 0;
    int64_t o_w1 = 0, o_b1 = 0, o_w2 = 0, o_b2 = 0, o_w3 = 0, o_b3 = 0;
    void set(int k_, int h1_, int h2_, int c_) {
        k = k_; h1 = h1_; h2 = h2_; c = c_;
        o_w1 = 0; o_b1 = o_w1 + (int64_t)h1 * k; o_w2 = o_b1 + h1; o_b2 = o_w2 + (int64_t)h2 * h1;
        o_w3 = o_b2 + h2; o_b3 = o_w3 + (int64_t)c * h2; np = o_b3 + c;
    }
};

// Activations for a batch of up to `cap` rows.
struct Acts {
    int64_t cap = 0;
    float *x = nullptr, *a1 = nullptr, *h1 = nullptr, *a2 = nullptr, *h2 = nullptr, *z = nullptr;
    float *dh1 = nullptr, *dh2 = nullptr, *row_loss = nullptr;
    int32_t *y = nullptr;
    void release() {
        cudaFree(x); cudaFree(a1); cudaFree(h1); cudaFree(a2); cudaFree(h2); cudaFree(z);
        cudaFree(dh1); cudaFree(dh2); cudaFree(row_loss); cudaFree(y);
        *this = Acts();
    }
    cudaError_t ensure(const Net &n, int64_t rows, bool train) {
        if (rows <= cap) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&x, sizeof(float) * rows * n.k);
        if (e == cudaSuccess) e = cudaMalloc(&h1, sizeof(float) * rows * n.h1);
        if (e == cudaSuccess) e = cudaMalloc(&h2, sizeof(float) * rows * n.h2);
        if (e == cudaSuccess) e = cudaMalloc(&z, sizeof(float) * rows * n.c);
        if (e == cudaSuccess) e = cudaMalloc(&row_loss, sizeof(float) * rows);
        if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(int32_t) * rows);
        if (train) {
            if (e == cudaSuccess) e = cudaMalloc(&a1, sizeof(float) * rows * n.h1);
            if (e == cudaSuccess) e = cudaMalloc(&a2, sizeof(float) * rows * n.h2);
            if (e == cudaSuccess) e = cudaMalloc(&dh1, sizeof(float) * rows * n.h1);
            if (e == cudaSuccess) e = cudaMalloc(&dh2, sizeof(float) * rows * n.h2);
        }
        if (e == cudaSuccess) cap = rows;
        return e;
    }
};

// Forward pass of `rows` inputs already in a.x; with `train`, pre-activations are kept.
static cudaError_t forward(const Net &n, const float *w, Acts &a, int rows, bool train, cudaStream_t st) {
    cudaError_t e = gemm(rows, n.h1, n.k, a.x, n.k, 1, w + n.o_w1, 1, n.k, a.h1, n.h1, st, 0.f, w + n.o_b1, 1,
                         train ? a.a1 : nullptr);
    if (e == cudaSuccess)
        e = gemm(rows, n.h2, n.h1, a.h1, n.h1, 1, w + n.o_w2, 1, n.h1, a.h2, n.h2, st, 0.f, w + n.o_b2, 1,
                 train ? a.a2 : nullptr);
    if (e == cudaSuccess) e = gemm(rows, n.c, n.h2, a.h2, n.h2, 1, w + n.o_w3, 1, n.h2, a.z, n.c, st, 0.f, w + n.o_b3, 0);
    return e;
}

// Loss (row losses in a.row_loss) and parameter gradients g for labels a.y; a.z is overwritten by dz.
static cudaError_t backward(const Net &n, const float *w, Acts &a, int rows, float *g, cudaStream_t st) {
    const unsigned wb = (unsigned)((rows * 32 + 255) / 256);
    k_softmax_xent<<<wb, 256, 0, st>>>(a.z, a.y, rows, n.c, 1.f / rows, a.z, a.row_loss);
    float *dz = a.z;
    cudaError_t e = cudaGetLastError();
    // layer 3
    if (e == cudaSuccess) e = gemm(n.c, n.h2, rows, dz, 1, n.c, a.h2, n.h2, 1, g + n.o_w3, n.h2, st);
    if (e == cudaSuccess) { k_colsum<<<(n.c + 255) / 256, 256, 0, st>>>(dz, rows, n.c, g + n.o_b3); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = gemm(rows, n.h2, n.c, dz, n.c, 1, w + n.o_w3, n.h2, 1, a.dh2, n.h2, st);
    if (e == cudaSuccess) {
        k_gelu_back<<<(unsigned)(((int64_t)rows * n.h2 + 255) / 256), 256, 0, st>>>(a.dh2, a.a2, (int64_t)rows * n.h2, a.dh2);
        e = cudaGetLastError();
    }
    // layer 2
    if (e == cudaSuccess) e = gemm(n.h2, n.h1, rows, a.dh2, 1, n.h2, a.h1, n.h1, 1, g + n.o_w2, n.h1, st);
    if (e == cudaSuccess) { k_colsum<<<(n.h2 + 255) / 256, 256, 0, st>>>(a.dh2, rows, n.h2, g + n.o_b2); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = gemm(rows, n.h1, n.h2, a.dh2, n.h2, 1, w + n.o_w2, n.h1, 1, a.dh1, n.h1, st);
    if (e == cudaSuccess) {
        k_gelu_back<<<(unsigned)(((int64_t)rows * n.h1 + 255) / 256), 256, 0, st>>>(a.dh1, a.a1, (int64_t)rows * n.h1, a.dh1);
        e = cudaGetLastError();
    }
    // layer 1
    if (e == cudaSuccess) e = gemm(n.h1, n.k, rows, a.dh1, 1, n.h1, a.x, n.k, 1, g + n.o_w1, n.k, st);
    if (e == cudaSuccess) { k_colsum<<<(n.h1 + 255) / 256, 256, 0, st>>>(a.dh1, rows, n.h1, g + n.o_b1); e = cudaGetLastError(); }
    return e;
}

}  // namespace hn

using namespace hn;

struct hn_proposal {
    Net net;
    int32_t n_blocks = 0;      // = net.c, the index's block count
    float *w = nullptr;        // FP32 master parameters
    float *w_inf = nullptr;    // BF16-rounded copy used for inference
    float *m = nullptr, *v = nullptr;  // Adam moments
    int64_t step = 0;          // Adam steps taken
    int32_t epochs_done = 0;
    float last_loss = NAN;
    Acts acts;                 // scratch, grown on demand
    int32_t *blocks = nullptr; // inference output scratch for seeded search
    int64_t blocks_cap = 0;
};

namespace hn {

static void destroy_proposal(hn_proposal *p) {
    if (!p) return;
    cudaFree(p->w); cudaFree(p->w_inf); cudaFree(p->m); cudaFree(p->v); cudaFree(p->blocks);
    p->acts.release();
    delete p;
}

static cudaError_t alloc_proposal(hn_proposal *p) {
    cudaError_t e = cudaMalloc(&p->w, sizeof(float) * p->net.np);
    if (e == cudaSuccess) e = cudaMalloc(&p->w_inf, sizeof(float) * p->net.np);
    if (e == cudaSuccess) e = cudaMalloc(&p->m, sizeof(float) * p->net.np);
    if (e == cudaSuccess) e = cudaMalloc(&p->v, sizeof(float) * p->net.np);
    return e;
}

// He-normal initial weights from a seeded splitmix64 stream and the Box-Muller
// transform (u1, u2 uniform in (0,1]: r = sqrt(-2 ln u1), normal = r cos(2 pi u2)); zero biases.
static std::vector<float> init_weights(const Net &n, uint64_t seed) {
    std::vector<float> w(n.np, 0.f);
    uint64_t s = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    auto next = [&]() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uniform = [&]() { return ((next() >> 11) + 1) * 0x1.0p-53; };
    auto fill = [&](int64_t off, int64_t count, double stdv) {
        for (int64_t i = 0; i < count; ++i) {
            const double r = sqrt(-2.0 * log(uniform()));
            w[off + i] = (float)(stdv * r * cos(6.283185307179586 * uniform()));
        }
    };
    fill(n.o_w1, (int64_t)n.h1 * n.k, sqrt(2.0 / n.k));
    fill(n.o_w2, (int64_t)n.h2 * n.h1, sqrt(2.0 / n.h1));
    fill(n.o_w3, (int64_t)n.c * n.h2, sqrt(2.0 / n.h2));
    return w;
}

// Top-k blocks for nq queries (rows of q, 128 wide), in chunks of 8192 rows.
cudaError_t proposal_topk(hn_proposal *p, const float *q, int64_t nq, int topk, int32_t *out, cudaStream_t st) {
    const Net &n = p->net;
    const int64_t chunk = 8192;
    cudaError_t e = p->acts.ensure(n, std::min<int64_t>(chunk, std::max<int64_t>(nq, 1)), false);
    for (int64_t r0 = 0; e == cudaSuccess && r0 < nq; r0 += chunk) {
        const int rows = (int)std::min<int64_t>(chunk, nq - r0);
        k_gather_prefix<<<(unsigned)(((int64_t)rows * n.k + 255) / 256), 256, 0, st>>>(q + r0 * kD, nullptr, rows, n.k,
                                                                                        p->acts.x, nullptr, nullptr);
        e = forward(n, p->w_inf, p->acts, rows, false, st);
        if (e == cudaSuccess) {
            k_topk<<<(unsigned)(((int64_t)rows * 32 + 255) / 256), 256, 0, st>>>(p->acts.z, rows, n.c, topk, out + r0 * topk);
            e = cudaGetLastError();
        }
    }
    return e;
}

int32_t proposal_blocks(const hn_proposal *p) { return p ? p->n_blocks : 0; }
int32_t proposal_k(const hn_proposal *p) { return p ? p->net.k : 0; }

cudaError_t proposal_scratch(hn_proposal *p, int64_t n, int32_t **out) {
    if (n > p->blocks_cap) {
        cudaFree(p->blocks);
        p->blocks = nullptr;
        p->blocks_cap = 0;
        cudaError_t e = cudaMalloc(&p->blocks, sizeof(int32_t) * n);
        if (e != cudaSuccess) return e;
        p->blocks_cap = n;
    }
    *out = p->blocks;
    return cudaSuccess;
}

}  // namespace hn

extern "C" {

hn_status hn_proposal_train(const hn_index *index, const float *train_q, const int32_t *nn_block, int64_t npairs,
                            const hn_train_opts *opts, hn_proposal **out, void *stream) {
    if (!out) return fail(HN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!index) return fail(HN_ERR_INVALID_ARG, "index is NULL");
    const Index &ix = *index_state(index);
    if (ix.n_blocks <= 0) return fail(HN_ERR_INVALID_ARG, "the index was built without blocks (opts.n_blocks)");
    if (npairs < 1 || npairs > 0x7FFFFFFF) return fail(HN_ERR_INVALID_ARG, "need 1 <= npairs < 2^31");
    if (!train_q || ((uintptr_t)train_q & 15u)) return fail(HN_ERR_INVALID_ARG, "null or unaligned train_q");
    hn_train_opts o{};
    if (opts) o = *opts;
    const int h1 = o.hidden1 ? o.hidden1 : 256, h2 = o.hidden2 ? o.hidden2 : 256;
    const int epochs = o.epochs ? o.epochs : 4;
    const int batch = o.batch ? o.batch : 4096;
    const float lr = o.lr > 0 ? o.lr : 1e-3f;
    if (h1 < 1 || h2 < 1 || h1 > 4096 || h2 > 4096 || epochs < 0 || batch < 1 || batch > (1 << 20))
        return fail(HN_ERR_INVALID_ARG, "bad training options");
    if (o.init && (o.init->net.k != ix.k || o.init->n_blocks != ix.n_blocks))
        return fail(HN_ERR_INVALID_ARG, "init proposal does not match the index");
    cudaStream_t st = (cudaStream_t)stream;
    hn_proposal *p = new hn_proposal();
    if (o.init) p->net = o.init->net; else p->net.set(ix.k, h1, h2, ix.n_blocks);
    p->n_blocks = ix.n_blocks;
    const Net &n = p->net;
    int32_t *y_all = nullptr, *perm = nullptr;
    int64_t *nn = nullptr;
    double *nn_sim = nullptr;
    float *g = nullptr, *loss_dev = nullptr;
    unsigned long long *keys = nullptr;
    int64_t n2 = 2048;
    while (n2 < npairs) n2 <<= 1;
    cudaError_t e = alloc_proposal(p);
#define TRYE(call) do { if (e == cudaSuccess) e = (call); } while (0)
    TRYE(cudaMalloc(&y_all, sizeof(int32_t) * npairs));
    TRYE(cudaMalloc(&perm, sizeof(int32_t) * npairs));
    TRYE(cudaMalloc(&keys, sizeof(unsigned long long) * n2));
    TRYE(cudaMalloc(&g, sizeof(float) * n.np));
    TRYE(cudaMalloc(&loss_dev, sizeof(float)));
    hn_status hs = HN_OK;
    if (e == cudaSuccess) {
        if (o.init) {
            TRYE(cudaMemcpyAsync(p->w, o.init->w, sizeof(float) * n.np, cudaMemcpyDeviceToDevice, st));
            TRYE(cudaMemcpyAsync(p->m, o.init->m, sizeof(float) * n.np, cudaMemcpyDeviceToDevice, st));
            TRYE(cudaMemcpyAsync(p->v, o.init->v, sizeof(float) * n.np, cudaMemcpyDeviceToDevice, st));
            p->step = o.init->step;
            p->epochs_done = o.init->epochs_done;
        } else {
            std::vector<float> w0 = init_weights(n, o.seed);
            TRYE(cudaMemcpyAsync(p->w, w0.data(), sizeof(float) * n.np, cudaMemcpyHostToDevice, st));
            TRYE(cudaMemsetAsync(p->m, 0, sizeof(float) * n.np, st));
            TRYE(cudaMemsetAsync(p->v, 0, sizeof(float) * n.np, st));
            TRYE(cudaStreamSynchronize(st));  // w0 is a host temporary
        }
    }
    // labels: given, or the block of each query's exact NN from the plain search
    if (e == cudaSuccess) {
        if (nn_block) {
            TRYE(cudaMemcpyAsync(y_all, nn_block, sizeof(int32_t) * npairs, cudaMemcpyDeviceToDevice, st));
        } else {
            TRYE(cudaMalloc(&nn, sizeof(int64_t) * npairs));
            TRYE(cudaMalloc(&nn_sim, sizeof(double) * npairs));
            const int64_t chunk = 65536;
            for (int64_t r0 = 0; e == cudaSuccess && hs == HN_OK && r0 < npairs; r0 += chunk) {
                const int64_t rows = std::min(chunk, npairs - r0);
                hs = hn_search_batch(const_cast<hn_index *>(index), train_q + r0 * kD, rows, nullptr, nn + r0,
                                     nn_sim + r0, nullptr, stream);
            }
            if (e == cudaSuccess && hs == HN_OK) {
                k_labels<<<(unsigned)((npairs + 255) / 256), 256, 0, st>>>(nn, ix.block_of, npairs, y_all);
                e = cudaGetLastError();
            }
        }
    }
    // training
    if (e == cudaSuccess && hs == HN_OK) e = p->acts.ensure(n, std::min<int64_t>(batch, npairs), true);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; e == cudaSuccess && hs == HN_OK && ep < epochs; ++ep) {
        const uint64_t salt = ((uint64_t)o.seed << 32) ^ (uint64_t)(p->epochs_done + 1) * 0xD1B54A32D192ED03ull;
        k_shuffle_keys<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(npairs, n2, salt, keys);
        TRYE(bitonic_sort(keys, n2, st));
        if (e == cudaSuccess) {
            k_low32<<<(unsigned)((npairs + 255) / 256), 256, 0, st>>>(keys, npairs, perm);
            e = cudaGetLastError();
        }
        for (int64_t r0 = 0; e == cudaSuccess && r0 < npairs; r0 += batch) {
            const int rows = (int)std::min<int64_t>(batch, npairs - r0);
            k_gather_prefix<<<(unsigned)(((int64_t)rows * n.k + 255) / 256), 256, 0, st>>>(
                train_q, perm + r0, rows, n.k, p->acts.x, y_all, p->acts.y);
            TRYE(forward(n, p->w, p->acts, rows, true, st));
            TRYE(backward(n, p->w, p->acts, rows, g, st));
            ++p->step;
            const float c1 = 1.f - powf(b1, (float)p->step), c2 = 1.f - powf(b2, (float)p->step);
            k_adam<<<(unsigned)((n.np + 255) / 256), 256, 0, st>>>(p->w, g, p->m, p->v, n.np, lr, b1, b2, eps, c1, c2);
            TRYE(cudaGetLastError());
            if (r0 + batch >= npairs && e == cudaSuccess) {  // loss of the epoch's last batch
                k_sum<<<1, 256, 0, st>>>(p->acts.row_loss, rows, loss_dev);
                float h = 0;
                TRYE(cudaMemcpyAsync(&h, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st));
                TRYE(cudaStreamSynchronize(st));
                p->last_loss = h / rows;
            }
        }
        ++p->epochs_done;
    }
    if (e == cudaSuccess && hs == HN_OK) {
        k_round_bf16<<<(unsigned)((n.np + 255) / 256), 256, 0, st>>>(p->w, n.np, p->w_inf);
        TRYE(cudaGetLastError());
        TRYE(cudaStreamSynchronize(st));
    }
#undef TRYE
    cudaFree(y_all); cudaFree(perm); cudaFree(keys); cudaFree(g); cudaFree(loss_dev); cudaFree(nn); cudaFree(nn_sim);
    if (hs != HN_OK) { destroy_proposal(p); return hs; }
    if (e != cudaSuccess) { destroy_proposal(p); return cuda_fail(e, "hn_proposal_train"); }
    *out = p;
    return HN_OK;
}

hn_status hn_proposal_infer(const hn_proposal *prop, const float *q, int64_t nq, int32_t topk, int32_t *out_blocks,
                            void *stream) {
    if (!prop) return fail(HN_ERR_INVALID_ARG, "proposal is NULL");
    if (nq < 0 || topk < 1 || topk > 64 || topk > prop->n_blocks) return fail(HN_ERR_INVALID_ARG, "bad nq or topk");
    if (nq == 0) return HN_OK;
    if (!q || !out_blocks || ((uintptr_t)q & 15u)) return fail(HN_ERR_INVALID_ARG, "null or unaligned pointer");
    HN_CUDA(proposal_topk(const_cast<hn_proposal *>(prop), q, nq, topk, out_blocks, (cudaStream_t)stream));
    return HN_OK;
}

hn_status hn_proposal_get_info(const hn_proposal *p, hn_proposal_info *info) {
    if (!p || !info) return fail(HN_ERR_INVALID_ARG, "NULL argument");
    info->k = p->net.k;
    info->hidden1 = p->net.h1;
    info->hidden2 = p->net.h2;
    info->n_blocks = p->n_blocks;
    info->n_params = p->net.np;
    info->steps = p->step;
    info->epochs = p->epochs_done;
    info->last_loss = p->last_loss;
    return HN_OK;
}

hn_status hn_proposal_destroy(hn_proposal *p) {
    destroy_proposal(p);
    return HN_OK;
}

// File: "HNPROP01", int32 k, h1, h2, c, int64 step, int32 epochs, float last_loss,
// then np floats each of weights, Adam m, Adam v.
hn_status hn_proposal_save(const hn_proposal *p, const char *path) {
    if (!p || !path) return fail(HN_ERR_INVALID_ARG, "NULL argument");
    const Net &n = p->net;
    std::vector<float> buf((size_t)n.np * 3);
    HN_CUDA(cudaMemcpy(buf.data(), p->w, sizeof(float) * n.np, cudaMemcpyDeviceToHost));
    HN_CUDA(cudaMemcpy(buf.data() + n.np, p->m, sizeof(float) * n.np, cudaMemcpyDeviceToHost));
    HN_CUDA(cudaMemcpy(buf.data() + 2 * n.np, p->v, sizeof(float) * n.np, cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(HN_ERR_INVALID_ARG, std::string("cannot open ") + path);
    const int32_t hdr[4] = {n.k, n.h1, n.h2, n.c};
    bool ok = fwrite("HNPROP01", 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(&p->step, sizeof(int64_t), 1, f) == 1 && fwrite(&p->epochs_done, sizeof(int32_t), 1, f) == 1 &&
              fwrite(&p->last_loss, sizeof(float), 1, f) == 1 &&
              fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? HN_OK : fail(HN_ERR_INVALID_ARG, std::string("write failed: ") + path);
}

hn_status hn_proposal_load(const char *path, hn_proposal **out) {
    if (!path || !out) return fail(HN_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(HN_ERR_INVALID_ARG, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[4];
    hn_proposal *p = new hn_proposal();
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "HNPROP01", 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
              hdr[0] >= 1 && hdr[0] <= 64 && hdr[1] >= 1 && hdr[1] <= 4096 && hdr[2] >= 1 && hdr[2] <= 4096 &&
              hdr[3] >= 1 && hdr[3] <= (1 << 20) && fread(&p->step, sizeof(int64_t), 1, f) == 1 &&
              fread(&p->epochs_done, sizeof(int32_t), 1, f) == 1 && fread(&p->last_loss, sizeof(float), 1, f) == 1;
    std::vector<float> buf;
    if (ok) {
        p->net.set(hdr[0], hdr[1], hdr[2], hdr[3]);
        p->n_blocks = hdr[3];
        buf.resize((size_t)p->net.np * 3);
        ok = fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    }
    fclose(f);
    if (!ok) {
        delete p;
        return fail(HN_ERR_INVALID_ARG, std::string("not a proposal file: ") + path);
    }
    cudaError_t e = alloc_proposal(p);
    const int64_t np = p->net.np;
    if (e == cudaSuccess) e = cudaMemcpy(p->w, buf.data(), sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->m, buf.data() + np, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->v, buf.data() + 2 * np, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_round_bf16<<<(unsigned)((np + 255) / 256), 256>>>(p->w, np, p->w_inf);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        destroy_proposal(p);
        return cuda_fail(e, "hn_proposal_load");
    }
    *out = p;
    return HN_OK;
}

hn_status hn_mlp_loss_grad(const float *params, int32_t k, int32_t h1, int32_t h2, int32_t c, const float *x,
                           const int32_t *y, int32_t batch, float *loss, float *grads, void *stream) {
    if (!params || !x || !y || !loss || !grads) return fail(HN_ERR_INVALID_ARG, "NULL argument");
    if (k < 1 || h1 < 1 || h2 < 1 || c < 1 || batch < 1 || k > 4096 || h1 > 4096 || h2 > 4096 || c > (1 << 20))
        return fail(HN_ERR_INVALID_ARG, "bad sizes");
    cudaStream_t st = (cudaStream_t)stream;
    Net n;
    n.set(k, h1, h2, c);
    Acts a;
    float *loss_dev = nullptr;
    cudaError_t e = a.ensure(n, batch, true);
    if (e == cudaSuccess) e = cudaMalloc(&loss_dev, sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.x, x, sizeof(float) * batch * k, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.y, y, sizeof(int32_t) * batch, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = forward(n, params, a, batch, true, st);
    if (e == cudaSuccess) e = backward(n, params, a, batch, grads, st);
    if (e == cudaSuccess) {
        k_sum<<<1, 256, 0, st>>>(a.row_loss, batch, loss_dev);
        float h = 0;
        e = cudaMemcpyAsync(&h, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        *loss = h / batch;
    }
    cudaFree(loss_dev);
    a.release();
    if (e != cudaSuccess) return cuda_fail(e, "hn_mlp_loss_grad");
    return HN_OK;
}

}  // extern "C"
