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
#include "hn_sm100.cuh"

namespace hn {
using namespace sm100;

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

// ------------------------------------------------------------------ tensor-core linear layer
// Inference layers on the tensor cores: out[r][j] = act(sum_k bf16(in[r][k]) bf16(w[j][k]) + b[j]),
// act 0 = none, 1 = gelu.  Products of BF16 values are exact in FP32 and the tcgen05.mma
// accumulates in FP32, so a layer differs from an FP32 evaluation on BF16-rounded operands
// only by the accumulation order (error <= gamma_K sum_k |a_k w_k|).
//
// One CTA per 128 x 256 output tile (M = 128 rows of `in`, N = 256 rows of `w`), 8 warps.  K is
// taken in slices of 64: all threads stage the slice's A (128 x ks) and B (256 x ks) operands in
// shared memory, rounded to BF16, in the no-swizzle K-major core-matrix layout (8 rows x 16
// bytes per core matrix, K-adjacent core matrices 128 bytes apart); one thread issues ks / 16
// MMAs (M = 128, N = 256, K = 16) into a 256-column TMEM accumulator and commits.  Two
// slice buffers: the staging of slice s + 1 overlaps the MMAs of slice s.  The epilogue reads
// the accumulator (thread = row; warps 0-3 columns 0-127, warps 4-7 columns 128-255), adds the
// bias, applies the activation and stores FP32.
constexpr int kLinM = 128, kLinN = 256, kLinKs = 64, kLinThreads = 256;
constexpr uint32_t kLinA = kLinM * kLinKs * 2, kLinB = kLinN * kLinKs * 2;  // bytes of one slice
constexpr uint32_t kLinSmem = 2 * (kLinA + kLinB) + 64;

// Byte offset of element (r, k) of a rows x ks operand slice in the core-matrix layout.
__device__ __forceinline__ uint32_t lin_off(int r, int k, int ks) {
    return (uint32_t)((((r >> 3) * (ks >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Stage rows [r0, r0 + rows) x columns [k0, k0 + ks) of an FP32 operand (R x K, element (r, k)
// at src[r * sr + k * sk]) as BF16; zeros outside the matrix.  With `vec` (sk = 1, K and sr
// multiples of 4, a 16-byte aligned base) each thread moves four consecutive columns at a time --
// one 16-byte load, one 8-byte store (four consecutive k are contiguous in a core matrix) -- with
// four loads in flight before any store, so that the staging is not bound by one load's latency
// at a time.  Otherwise one element a thread, consecutive threads along the operand's contiguous
// direction (k when sk = 1, else r when sr = 1), so that the loads stay coalesced.
__device__ __forceinline__ void lin_stage(uint8_t *dst, const float *__restrict__ src, int64_t sr, int64_t sk,
                                          int R, int K, int r0, int rows, int k0, int ks, bool vec) {
    const int64_t ld = sr;
    if (vec) {
        const int kq = ks >> 2, total = rows * kq;
        for (int base = threadIdx.x; base < total; base += 4 * kLinThreads) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * kLinThreads;
                const int r = idx / kq, k = (idx - r * kq) << 2;
                const int gr = r0 + r, gk = k0 + k;
                v[u] = (idx < total && gr < R && gk < K) ? *reinterpret_cast<const float4 *>(src + (int64_t)gr * ld + gk)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * kLinThreads;
                if (idx >= total) break;
                const int r = idx / kq, k = (idx - r * kq) << 2;
                const __nv_bfloat162 lo = __floats2bfloat162_rn(v[u].x, v[u].y), hi = __floats2bfloat162_rn(v[u].z, v[u].w);
                uint2 packed;
                packed.x = *reinterpret_cast<const uint32_t *>(&lo);
                packed.y = *reinterpret_cast<const uint32_t *>(&hi);
                *reinterpret_cast<uint2 *>(dst + lin_off(r, k, ks)) = packed;
            }
        }
        return;
    }
    // strided operand (a transposed activation or weight): consecutive threads take consecutive
    // rows when rows are adjacent in memory; eight loads in flight per thread before any store
    const bool rows_fast = sk != 1 && sr == 1;
    const int total = rows * ks;
    for (int base = threadIdx.x; base < total; base += 8 * kLinThreads) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = base + u * kLinThreads;
            int r, k;
            if (rows_fast) { k = idx / rows; r = idx - k * rows; } else { r = idx / ks; k = idx - r * ks; }
            const int gr = r0 + r, gk = k0 + k;
            v[u] = (idx < total && gr < R && gk < K) ? src[(int64_t)gr * sr + (int64_t)gk * sk] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = base + u * kLinThreads;
            if (idx >= total) break;
            int r, k;
            if (rows_fast) { k = idx / rows; r = idx - k * rows; } else { r = idx / ks; k = idx - r * ks; }
            *reinterpret_cast<__nv_bfloat16 *>(dst + lin_off(r, k, ks)) = __float2bfloat16_rn(v[u]);
        }
    }
}

// Running top-TK of one thread's columns, (score desc, column asc): a value enters only if it
// beats the current last (strict, and columns come in increasing order, so on equal scores the
// earlier column stays), then bubbles up.
template <int TK>
__device__ __forceinline__ void topk_insert(float (&ts)[TK], int (&ti)[TK], float x, int j) {
    if (!(x > ts[TK - 1])) return;
#pragma unroll
    for (int p = 0; p < TK; ++p) {
        if (x > ts[p]) {
            const float tx = ts[p];
            const int tj = ti[p];
            ts[p] = x;
            ti[p] = j;
            x = tx;
            j = tj;
        }
    }
}

// TK = 0: store out.  TK = 4 or 8 (the proposal's last layer): no output matrix; each row's
// TK best columns of this CTA's 256 (score desc, column asc) go to cand[row][blockIdx.x][TK] as
// pack_best keys, 0 for none, and k_topk_keys picks the row's best among its tiles.
// in: element (r, k) at in[r * sai + k * sak]; w: element (j, k) at w[j * swj + k * swk].
// pre (TK = 0, act 1, may be NULL): the pre-activation values, stored like out.
template <int TK>
__global__ void __launch_bounds__(kLinThreads) k_linear_bf16(int M, int N, int K, const float *__restrict__ in,
                                                             int64_t sai, int64_t sak, const float *__restrict__ w,
                                                             int64_t swj, int64_t swk,
                                                             const float *__restrict__ bias, int act,
                                                             float *__restrict__ out, int64_t ldo,
                                                             float *__restrict__ pre,
                                                             unsigned long long *__restrict__ cand,
                                                             int32_t *__restrict__ status, int kper,
                                                             float *__restrict__ part) {
    extern __shared__ __align__(1024) uint8_t lsm[];
    uint8_t *sa = lsm, *sb = lsm + 2 * kLinA;
    uint64_t *done = reinterpret_cast<uint64_t *>(lsm + 2 * (kLinA + kLinB));  // [2] MMA completion per slice buffer
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.y * kLinM, c0 = blockIdx.x * kLinN;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&done[0]), 1);
        mbar_init(smem_u32(&done[1]), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), kLinN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = idesc_bf16_f32(kLinM, kLinN);
    // this CTA's share of K: [kbeg, kend), a multiple of 16 wide (kper is a multiple of kLinKs)
    const int kp = (K + 15) & ~15;
    const int kbeg = (int)min((int64_t)blockIdx.z * kper, (int64_t)kp), kend = (int)min((int64_t)kbeg + kper, (int64_t)kp);
    const bool vec_in = sak == 1 && (K & 3) == 0 && (sai & 3) == 0 && ((uintptr_t)in & 15u) == 0;
    const bool vec_w = swk == 1 && (K & 3) == 0 && (swj & 3) == 0 && ((uintptr_t)w & 15u) == 0;
    const int slices = (kend - kbeg + kLinKs - 1) / kLinKs;
    constexpr uint64_t kLimit = 2000000000ull;
    bool ok = true;
    int issued = 0;  // slices whose MMAs were issued (and committed)
    for (int s = 0; s < slices; ++s) {
        const int buf = s & 1, k0 = kbeg + s * kLinKs, ks = min(kLinKs, kend - k0);
        // the MMAs of slice s - 2 read this buffer: wait for their commit
        if (s >= 2) {
            ok = mbar_wait(smem_u32(&done[buf]), (uint32_t)(((s - 2) >> 1) & 1), abort_flag, kLimit);
            if (!__syncthreads_and(ok)) break;
        }
        lin_stage(sa + buf * kLinA, in, sai, sak, M, K, r0, kLinM, k0, ks, vec_in);
        lin_stage(sb + buf * kLinB, w, swj, swk, N, K, c0, kLinN, k0, ks, vec_w);
        // generic-proxy stores must be visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a = smem_u32(sa + buf * kLinA), b = smem_u32(sb + buf * kLinB);
            for (int kk = 0; kk < ks / 16; ++kk) {
                const uint64_t ad = smem_desc(a + kk * 256, 128, ks * 16);
                const uint64_t bd = smem_desc(b + kk * 256, 128, ks * 16);
                umma_bf16(tmem, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit(smem_u32(&done[buf]));
        }
        ++issued;
    }
    // the last commit covers every MMA issued before it
    if (issued > 0) {
        const int last = issued - 1;
        if (ok) ok = mbar_wait(smem_u32(&done[last & 1]), (uint32_t)((last >> 1) & 1), abort_flag, kLimit);
        else mbar_drain(smem_u32(&done[last & 1]), (uint32_t)((last >> 1) & 1), kLimit);
    }
    ok = __syncthreads_and(ok);  // uniform: the epilogue below has a block-wide barrier
    tc_fence_after();
    if (ok && issued == slices) {
        const int quarter = warp & 3, colhalf = warp >> 2;  // TMEM lanes 32 quarter .., columns 128 colhalf ..
        const int rl = quarter * 32 + lane, r = r0 + rl;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        if constexpr (TK == 0) {
            // a K split writes its plain partial sums to its own (M x N) slab of `part`
            float *o = part ? part + (int64_t)blockIdx.z * M * N : out;
            const int64_t ldd = part ? N : ldo;
            for (int cb = colhalf * (kLinN / 2); cb < (colhalf + 1) * (kLinN / 2); cb += 32) {
                float v[32];
                tmem_ld32(tmem + cb + lane_addr, v);
                if (r < M && part) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int j = c0 + cb + i;
                        if (j < N) o[(int64_t)r * ldd + j] = v[i];
                    }
                } else if (r < M) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int j = c0 + cb + i;
                        if (j < N) {
                            float x = v[i] + (bias ? bias[j] : 0.f);
                            if (act == 1) {
                                if (pre) pre[(int64_t)r * ldo + j] = x;
                                x = gelu_f(x);
                            }
                            out[(int64_t)r * ldo + j] = x;
                        }
                    }
                }
            }
        } else {
            float ts[TK];
            int ti[TK];
#pragma unroll
            for (int t = 0; t < TK; ++t) {
                ts[t] = -INFINITY;
                ti[t] = -1;
            }
            for (int cb = colhalf * (kLinN / 2); cb < (colhalf + 1) * (kLinN / 2); cb += 32) {
                float v[32];
                tmem_ld32(tmem + cb + lane_addr, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int j = c0 + cb + i;
                    if (j < N) topk_insert<TK>(ts, ti, v[i] + (bias ? bias[j] : 0.f), j);
                }
            }
            // the two column halves of a row meet in shared memory (the slice buffers are free:
            // every MMA has completed); the colhalf-0 thread merges them
            unsigned long long *mk = reinterpret_cast<unsigned long long *>(lsm);  // [128 rows][2 halves][TK]
#pragma unroll
            for (int t = 0; t < TK; ++t)
                mk[(rl * 2 + colhalf) * TK + t] = ti[t] >= 0 ? pack_best(ts[t], (uint32_t)ti[t]) : 0ull;
            __syncthreads();
            if (colhalf == 0 && r < M) {
                const unsigned long long *a = mk + rl * 2 * TK, *b = a + TK;
                int ia = 0, ib = 0;
                unsigned long long *dst = cand + ((int64_t)r * gridDim.x + blockIdx.x) * TK;
#pragma unroll
                for (int t = 0; t < TK; ++t) {
                    const unsigned long long ka = ia < TK ? a[ia] : 0ull, kb = ib < TK ? b[ib] : 0ull;
                    if (ka >= kb) { dst[t] = ka; ++ia; } else { dst[t] = kb; ++ib; }
                }
            }
        }
    }
    if (threadIdx.x == 0 && *abort_flag && status) atomicExch(status, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kLinN);
}

// Top-k of every row from its tiles' candidates (pack_best keys, 0 = none): one warp per row,
// topk rounds of a warp maximum below the previous round's key (keys are distinct).
__global__ void k_topk_keys(const unsigned long long *__restrict__ cand, int64_t rows, int per_row, int topk,
                            int32_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= rows) return;
    const unsigned long long *ci = cand + i * per_row;
    unsigned long long taken = ~0ull;
    for (int r = 0; r < topk; ++r) {
        unsigned long long km = 0;
        for (int c = lane; c < per_row; c += 32) {
            const unsigned long long k = ci[c];
            if (k < taken && k > km) km = k;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, km, o);
            km = other > km ? other : km;
        }
        taken = km;
        if (lane == 0) out[i * topk + r] = km ? (int32_t)best_idx(km) : -1;
    }
}

template <int TK>
static cudaError_t launch_linear(int M, int N, int K, const float *in, int64_t sai, int64_t sak, const float *w,
                                 int64_t swj, int64_t swk, const float *bias, int act, float *out, int64_t ldo,
                                 float *pre, unsigned long long *cand, int32_t *status, cudaStream_t st,
                                 int splits = 1, int kper = 1 << 30, float *part = nullptr) {
    static bool ready = false;
    if (!ready) {
        cudaError_t e = cudaFuncSetAttribute(k_linear_bf16<TK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinSmem);
        if (e != cudaSuccess) return e;
        ready = true;
    }
    dim3 grid((unsigned)((N + kLinN - 1) / kLinN), (unsigned)((M + kLinM - 1) / kLinM), (unsigned)splits);
    k_linear_bf16<TK><<<grid, kLinThreads, kLinSmem, st>>>(M, N, K, in, sai, sak, w, swj, swk, bias, act, out, ldo, pre,
                                                           cand, status, kper, part);
    return cudaGetLastError();
}

cudaError_t linear_bf16(int M, int N, int K, const float *in, int64_t ldi, const float *w, int64_t ldw,
                        const float *bias, int act, float *out, int64_t ldo, int32_t *status, cudaStream_t st) {
    if (M == 0 || N == 0) return cudaSuccess;
    if (M < 0 || N < 0 || K < 1) return cudaErrorInvalidValue;
    return launch_linear<0>(M, N, K, in, ldi, 1, w, ldw, 1, bias, act, out, ldo, nullptr, nullptr, status, st);
}

static int g_lin_sms = 0;
static int lin_sms() {
    if (g_lin_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_lin_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_lin_sms <= 0) g_lin_sms = 148;
    }
    return g_lin_sms;
}

// K split of a tensor-core GEMM whose output tiles alone would leave SMs idle (a weight
// gradient: K is the batch, M x N the weight): enough splits for about two CTAs per SM, each
// at least four K slices.  Returns the split count; *kper = K elements per split, a multiple of
// kLinKs, every split non-empty.
static int lin_splits(int M, int N, int K, int *kper) {
    const int64_t tiles = (int64_t)((M + kLinM - 1) / kLinM) * ((N + kLinN - 1) / kLinN);
    const int kp = (K + 15) & ~15;
    const int64_t want = std::min<int64_t>((kp + 4 * kLinKs - 1) / (4 * kLinKs), std::max<int64_t>(1, 2 * lin_sms() / tiles));
    if (want <= 1) {
        *kper = 1 << 30;
        return 1;
    }
    int per = (int)((kp + want - 1) / want);
    per = (per + kLinKs - 1) / kLinKs * kLinKs;
    *kper = per;
    return (kp + per - 1) / per;
}

// Partial-sum floats any split GEMM needs at most: splits x M x N <= 2 SMs x tiles x tile area.
static int64_t lin_split_cap() { return (int64_t)2 * lin_sms() * kLinM * kLinN; }

// C = the partial slabs summed in split order (deterministic).
__global__ void k_splitk_sum(const float *__restrict__ part, int splits, int M, int N, float *__restrict__ C,
                             int64_t ldc) {
    const int64_t mn = (int64_t)M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < mn; e += (int64_t)gridDim.x * blockDim.x) {
        float v = part[e];
        for (int z = 1; z < splits; ++z) v += part[z * mn + e];
        const int64_t i = e / N;
        C[i * ldc + (e - i * N)] = v;
    }
}

// The training GEMMs on the tensor cores, with the FP32 gemm()'s operand convention:
// C(i,j) = sum_k bf16(A(i,k)) bf16(B(k,j)) [+ bias[j], act, pre], A(i,k) = A[i*sai + k*sak],
// B(k,j) = B[k*sbk + j*sbj]; products exact, summed in FP32.  Without bias or activation and
// given a partial-sum buffer of lin_split_cap() floats, K is split across CTAs.
static cudaError_t gemm_bf16(int M, int N, int K, const float *A, int64_t sai, int64_t sak, const float *B, int64_t sbk,
                             int64_t sbj, float *C, int64_t ldc, int32_t *status, cudaStream_t st,
                             const float *bias = nullptr, int act = 0, float *pre = nullptr, float *part = nullptr) {
    if (M == 0 || N == 0) return cudaSuccess;
    if (M < 0 || N < 0 || K < 1) return cudaErrorInvalidValue;
    int kper = 1 << 30, splits = 1;
    if (part && !bias && act == 0 && !pre) splits = lin_splits(M, N, K, &kper);
    if (splits == 1)
        return launch_linear<0>(M, N, K, A, sai, sak, B, sbj, sbk, bias, act, C, ldc, pre, nullptr, status, st);
    cudaError_t e = launch_linear<0>(M, N, K, A, sai, sak, B, sbj, sbk, nullptr, 0, C, ldc, nullptr, nullptr, status, st,
                                     splits, kper, part);
    if (e != cudaSuccess) return e;
    const int64_t mn = (int64_t)M * N;
    k_splitk_sum<<<(unsigned)std::min<int64_t>((mn + 255) / 256, 8 * lin_sms()), 256, 0, st>>>(part, splits, M, N, C, ldc);
    return cudaGetLastError();
}

// Last layer with its top-k fused (topk <= 8): per row the topk best columns of
// in . w^T + bias, (score desc, column asc), into out (rows x topk int32).  cand: scratch of
// M * ceil(N / 256) * 8 keys.
static cudaError_t linear_bf16_topk(int M, int N, int K, const float *in, int64_t ldi, const float *w, int64_t ldw,
                                    const float *bias, int topk, unsigned long long *cand, int32_t *out,
                                    int32_t *status, cudaStream_t st) {
    if (M == 0) return cudaSuccess;
    const int tiles = (N + kLinN - 1) / kLinN;
    const int tk = topk <= 4 ? 4 : 8;
    cudaError_t e = tk == 4 ? launch_linear<4>(M, N, K, in, ldi, 1, w, ldw, 1, bias, 0, nullptr, 0, nullptr, cand, status, st)
                            : launch_linear<8>(M, N, K, in, ldi, 1, w, ldw, 1, bias, 0, nullptr, 0, nullptr, cand, status, st);
    if (e != cudaSuccess) return e;
    k_topk_keys<<<(unsigned)(((int64_t)M * 32 + 255) / 256), 256, 0, st>>>(cand, M, tiles * tk, topk, out);
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
    bool has_z = false;                     // z allocated (rows x c); the fused top-k needs none
    unsigned long long *cand = nullptr;     // fused top-k candidates
    int64_t cand_cap = 0;
    void release() {
        cudaFree(x); cudaFree(a1); cudaFree(h1); cudaFree(a2); cudaFree(h2); cudaFree(z);
        cudaFree(dh1); cudaFree(dh2); cudaFree(row_loss); cudaFree(y); cudaFree(cand);
        *this = Acts();
    }
    cudaError_t ensure_cand(int64_t count) {
        if (count <= cand_cap) return cudaSuccess;
        cudaFree(cand);
        cand = nullptr;
        cand_cap = 0;
        cudaError_t e = cudaMalloc(&cand, sizeof(unsigned long long) * count);
        if (e == cudaSuccess) cand_cap = count;
        return e;
    }
    cudaError_t ensure(const Net &n, int64_t rows, bool train, bool need_z = true) {
        if (rows <= cap && (has_z || !need_z) && (!train || a1)) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&x, sizeof(float) * rows * n.k);
        if (e == cudaSuccess) e = cudaMalloc(&h1, sizeof(float) * rows * n.h1);
        if (e == cudaSuccess) e = cudaMalloc(&h2, sizeof(float) * rows * n.h2);
        if (e == cudaSuccess && need_z) {
            e = cudaMalloc(&z, sizeof(float) * rows * n.c);
            has_z = e == cudaSuccess;
        }
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

// Inference forward pass of `rows` inputs already in a.x (weights already BF16-rounded): the
// three layers on the tensor cores, BF16 operands, FP32 accumulation.  `status` (device, may be
// NULL) is set to 1 if a layer's bounded wait gave up.
static cudaError_t forward_infer(const Net &n, const float *w, Acts &a, int rows, int32_t *status, cudaStream_t st) {
    cudaError_t e = linear_bf16(rows, n.h1, n.k, a.x, n.k, w + n.o_w1, n.k, w + n.o_b1, 1, a.h1, n.h1, status, st);
    if (e == cudaSuccess)
        e = linear_bf16(rows, n.h2, n.h1, a.h1, n.h1, w + n.o_w2, n.h1, w + n.o_b2, 1, a.h2, n.h2, status, st);
    if (e == cudaSuccess)
        e = linear_bf16(rows, n.c, n.h2, a.h2, n.h2, w + n.o_w3, n.h2, w + n.o_b3, 0, a.z, n.c, status, st);
    return e;
}

// The training GEMMs: with `bf16` on the tensor cores (BF16 operands, FP32 accumulation, the
// precision the proposal is specified in), otherwise FP32 CUDA-core tiles (the gradient check
// against the binary64 oracle).  status: device word set to 1 if a tensor-core wait gave up.
struct TrainGemm {
    bool bf16;
    int32_t *status;
    cudaStream_t st;
    float *part = nullptr;  // lin_split_cap() floats: K-split partial sums (weight gradients)
    cudaError_t operator()(int M, int N, int K, const float *A, int64_t sai, int64_t sak, const float *B, int64_t sbk,
                           int64_t sbj, float *C, int64_t ldc, const float *bias = nullptr, int act = 0,
                           float *pre = nullptr) const {
        return bf16 ? gemm_bf16(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, status, st, bias, act, pre, part)
                    : gemm(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, st, 0.f, bias, act, pre);
    }
};

// Training forward pass; with `train`, pre-activations are kept.
static cudaError_t forward(const Net &n, const float *w, Acts &a, int rows, bool train, const TrainGemm &G) {
    cudaError_t e = G(rows, n.h1, n.k, a.x, n.k, 1, w + n.o_w1, 1, n.k, a.h1, n.h1, w + n.o_b1, 1, train ? a.a1 : nullptr);
    if (e == cudaSuccess)
        e = G(rows, n.h2, n.h1, a.h1, n.h1, 1, w + n.o_w2, 1, n.h1, a.h2, n.h2, w + n.o_b2, 1, train ? a.a2 : nullptr);
    if (e == cudaSuccess) e = G(rows, n.c, n.h2, a.h2, n.h2, 1, w + n.o_w3, 1, n.h2, a.z, n.c, w + n.o_b3, 0);
    return e;
}

// Loss (row losses in a.row_loss) and parameter gradients g for labels a.y; a.z is overwritten by dz.
static cudaError_t backward(const Net &n, const float *w, Acts &a, int rows, float *g, const TrainGemm &G) {
    cudaStream_t st = G.st;
    const unsigned wb = (unsigned)((rows * 32 + 255) / 256);
    k_softmax_xent<<<wb, 256, 0, st>>>(a.z, a.y, rows, n.c, 1.f / rows, a.z, a.row_loss);
    float *dz = a.z;
    cudaError_t e = cudaGetLastError();
    // layer 3
    if (e == cudaSuccess) e = G(n.c, n.h2, rows, dz, 1, n.c, a.h2, n.h2, 1, g + n.o_w3, n.h2);
    if (e == cudaSuccess) { k_colsum<<<(n.c + 255) / 256, 256, 0, st>>>(dz, rows, n.c, g + n.o_b3); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = G(rows, n.h2, n.c, dz, n.c, 1, w + n.o_w3, n.h2, 1, a.dh2, n.h2);
    if (e == cudaSuccess) {
        k_gelu_back<<<(unsigned)(((int64_t)rows * n.h2 + 255) / 256), 256, 0, st>>>(a.dh2, a.a2, (int64_t)rows * n.h2, a.dh2);
        e = cudaGetLastError();
    }
    // layer 2
    if (e == cudaSuccess) e = G(n.h2, n.h1, rows, a.dh2, 1, n.h2, a.h1, n.h1, 1, g + n.o_w2, n.h1);
    if (e == cudaSuccess) { k_colsum<<<(n.h2 + 255) / 256, 256, 0, st>>>(a.dh2, rows, n.h2, g + n.o_b2); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = G(rows, n.h1, n.h2, a.dh2, n.h2, 1, w + n.o_w2, n.h1, 1, a.dh1, n.h1);
    if (e == cudaSuccess) {
        k_gelu_back<<<(unsigned)(((int64_t)rows * n.h1 + 255) / 256), 256, 0, st>>>(a.dh1, a.a1, (int64_t)rows * n.h1, a.dh1);
        e = cudaGetLastError();
    }
    // layer 1
    if (e == cudaSuccess) e = G(n.h1, n.k, rows, a.dh1, 1, n.h1, a.x, n.k, 1, g + n.o_w1, n.k);
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
cudaError_t proposal_topk(hn_proposal *p, const float *q, int64_t nq, int topk, int32_t *out, int32_t *status,
                          cudaStream_t st) {
    const Net &n = p->net;
    if (topk <= 8) {
        // top-k fused into the last layer: no score matrix, so large chunks (the hidden layers then
        // fill the GPU)
        const int64_t chunk = 65536;
        const int64_t rows_max = std::min<int64_t>(chunk, std::max<int64_t>(nq, 1));
        cudaError_t e = p->acts.ensure(n, rows_max, false, false);
        if (e == cudaSuccess) e = p->acts.ensure_cand(rows_max * ((n.c + 255) / 256) * 8);
        for (int64_t r0 = 0; e == cudaSuccess && r0 < nq; r0 += chunk) {
            const int rows = (int)std::min<int64_t>(chunk, nq - r0);
            k_gather_prefix<<<(unsigned)(((int64_t)rows * n.k + 255) / 256), 256, 0, st>>>(
                q + r0 * kD, nullptr, rows, n.k, p->acts.x, nullptr, nullptr);
            const float *w = p->w_inf;
            Acts &a = p->acts;
            e = linear_bf16(rows, n.h1, n.k, a.x, n.k, w + n.o_w1, n.k, w + n.o_b1, 1, a.h1, n.h1, status, st);
            if (e == cudaSuccess)
                e = linear_bf16(rows, n.h2, n.h1, a.h1, n.h1, w + n.o_w2, n.h1, w + n.o_b2, 1, a.h2, n.h2, status, st);
            if (e == cudaSuccess)
                e = linear_bf16_topk(rows, n.c, n.h2, a.h2, n.h2, w + n.o_w3, n.h2, w + n.o_b3, topk, a.cand,
                                     out + r0 * topk, status, st);
        }
        return e;
    }
    const int64_t chunk = 8192;
    cudaError_t e = p->acts.ensure(n, std::min<int64_t>(chunk, std::max<int64_t>(nq, 1)), false);
    for (int64_t r0 = 0; e == cudaSuccess && r0 < nq; r0 += chunk) {
        const int rows = (int)std::min<int64_t>(chunk, nq - r0);
        k_gather_prefix<<<(unsigned)(((int64_t)rows * n.k + 255) / 256), 256, 0, st>>>(q + r0 * kD, nullptr, rows, n.k,
                                                                                        p->acts.x, nullptr, nullptr);
        e = forward_infer(n, p->w_inf, p->acts, rows, status, st);
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
    if (o.precision != 0 && o.precision != 1) return fail(HN_ERR_INVALID_ARG, "precision must be 0 or 1");
    if (o.reserved[0]) return fail(HN_ERR_INVALID_ARG, "reserved option fields must be zero");
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
    int32_t *gstatus = nullptr;  // set by a tensor-core GEMM whose bounded wait gave up
    if (e == cudaSuccess && hs == HN_OK) e = cudaMalloc(&gstatus, sizeof(int32_t));
    if (e == cudaSuccess && hs == HN_OK) e = cudaMemsetAsync(gstatus, 0, sizeof(int32_t), st);
    float *gpart = nullptr;  // K-split partial sums of the tensor-core weight gradients
    if (e == cudaSuccess && hs == HN_OK && o.precision == 0) e = cudaMalloc(&gpart, sizeof(float) * lin_split_cap());
    const TrainGemm G{o.precision == 0, gstatus, st, gpart};
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
            TRYE(forward(n, p->w, p->acts, rows, true, G));
            TRYE(backward(n, p->w, p->acts, rows, g, G));
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
        int32_t hstat = 0;
        TRYE(cudaMemcpyAsync(&hstat, gstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TRYE(cudaStreamSynchronize(st));
        if (e == cudaSuccess && hstat) hs = fail(HN_ERR_TIMEOUT, "a tensor-core training GEMM's device-side wait timed out");
    }
#undef TRYE
    cudaFree(gstatus);
    cudaFree(gpart);
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
    HN_CUDA(proposal_topk(const_cast<hn_proposal *>(prop), q, nq, topk, out_blocks, nullptr, (cudaStream_t)stream));
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

static hn_status mlp_loss_grad(const float *params, int32_t k, int32_t h1, int32_t h2, int32_t c, const float *x,
                               const int32_t *y, int32_t batch, float *loss, float *grads, bool bf16, void *stream) {
    if (!params || !x || !y || !loss || !grads) return fail(HN_ERR_INVALID_ARG, "NULL argument");
    if (k < 1 || h1 < 1 || h2 < 1 || c < 1 || batch < 1 || k > 4096 || h1 > 4096 || h2 > 4096 || c > (1 << 20))
        return fail(HN_ERR_INVALID_ARG, "bad sizes");
    cudaStream_t st = (cudaStream_t)stream;
    Net n;
    n.set(k, h1, h2, c);
    Acts a;
    float *loss_dev = nullptr;
    int32_t *status = nullptr;
    cudaError_t e = a.ensure(n, batch, true);
    if (e == cudaSuccess) e = cudaMalloc(&loss_dev, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.x, x, sizeof(float) * batch * k, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.y, y, sizeof(int32_t) * batch, cudaMemcpyDeviceToDevice, st);
    float *part = nullptr;
    if (e == cudaSuccess && bf16) e = cudaMalloc(&part, sizeof(float) * lin_split_cap());
    const TrainGemm G{bf16, status, st, part};
    if (e == cudaSuccess) e = forward(n, params, a, batch, true, G);
    if (e == cudaSuccess) e = backward(n, params, a, batch, grads, G);
    int32_t hstat = 0;
    if (e == cudaSuccess) {
        k_sum<<<1, 256, 0, st>>>(a.row_loss, batch, loss_dev);
        float h = 0;
        e = cudaMemcpyAsync(&h, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        *loss = h / batch;
    }
    cudaFree(loss_dev);
    cudaFree(status);
    cudaFree(part);
    a.release();
    if (e != cudaSuccess) return cuda_fail(e, "hn_mlp_loss_grad");
    if (hstat) return fail(HN_ERR_TIMEOUT, "a tensor-core GEMM's device-side wait timed out");
    return HN_OK;
}

hn_status hn_mlp_loss_grad(const float *params, int32_t k, int32_t h1, int32_t h2, int32_t c, const float *x,
                           const int32_t *y, int32_t batch, float *loss, float *grads, void *stream) {
    return mlp_loss_grad(params, k, h1, h2, c, x, y, batch, loss, grads, false, stream);
}

hn_status hn_mlp_loss_grad_bf16(const float *params, int32_t k, int32_t h1, int32_t h2, int32_t c, const float *x,
                                const int32_t *y, int32_t batch, float *loss, float *grads, void *stream) {
    return mlp_loss_grad(params, k, h1, h2, c, x, y, batch, loss, grads, true, stream);
}

hn_status hn_gemm_bf16(int32_t m, int32_t n, int32_t k, const float *a, int64_t sai, int64_t sak, const float *b,
                       int64_t sbk, int64_t sbj, float *c, int64_t ldc, void *stream) {
    if (m < 0 || n < 0 || k < 1 || k > 65536) return fail(HN_ERR_INVALID_ARG, "need m, n >= 0 and 1 <= k <= 65536");
    if (m == 0 || n == 0) return HN_OK;
    if (!a || !b || !c) return fail(HN_ERR_INVALID_ARG, "NULL argument");
    if (sai < 0 || sak < 0 || sbk < 0 || sbj < 0 || ldc < n) return fail(HN_ERR_INVALID_ARG, "bad strides");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = nullptr;
    int32_t hstat = 0;
    float *part = nullptr;
    cudaError_t e = cudaMalloc(&status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(float) * lin_split_cap());
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = gemm_bf16(m, n, k, a, sai, sak, b, sbk, sbj, c, ldc, status, st, nullptr, 0, nullptr, part);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(status);
    cudaFree(part);
    if (e != cudaSuccess) return cuda_fail(e, "hn_gemm_bf16");
    if (hstat) return fail(HN_ERR_TIMEOUT, "a device-side wait timed out");
    return HN_OK;
}

hn_status hn_linear_bf16(const float *in, int32_t m, int32_t k, const float *w, int32_t n, const float *bias,
                         int32_t act, float *out, void *stream) {
    if (m < 0 || n < 0 || k < 1 || k > 65536 || (act != 0 && act != 1)) return fail(HN_ERR_INVALID_ARG, "bad sizes or act");
    if (m == 0 || n == 0) return HN_OK;
    if (!in || !w || !out) return fail(HN_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = nullptr, h = 0;
    cudaError_t e = cudaMalloc(&status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = linear_bf16(m, n, k, in, k, w, k, bias, act, out, n, status, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(status);
    if (e != cudaSuccess) return cuda_fail(e, "hn_linear_bf16");
    if (h) return fail(HN_ERR_TIMEOUT, "a device-side wait timed out");
    return HN_OK;
}

hn_status hn_proposal_logits(const hn_proposal *prop, const float *q, int64_t nq, float *out_z, void *stream) {
    if (!prop) return fail(HN_ERR_INVALID_ARG, "proposal is NULL");
    if (nq < 0) return fail(HN_ERR_INVALID_ARG, "nq < 0");
    if (nq == 0) return HN_OK;
    if (!q || !out_z || ((uintptr_t)q & 15u)) return fail(HN_ERR_INVALID_ARG, "null or unaligned pointer");
    hn_proposal *p = const_cast<hn_proposal *>(prop);
    const Net &n = p->net;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t chunk = 8192;
    cudaError_t e = p->acts.ensure(n, std::min<int64_t>(chunk, nq), false);
    for (int64_t r0 = 0; e == cudaSuccess && r0 < nq; r0 += chunk) {
        const int rows = (int)std::min<int64_t>(chunk, nq - r0);
        k_gather_prefix<<<(unsigned)(((int64_t)rows * n.k + 255) / 256), 256, 0, st>>>(q + r0 * kD, nullptr, rows, n.k,
                                                                                        p->acts.x, nullptr, nullptr);
        e = forward_infer(n, p->w_inf, p->acts, rows, nullptr, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_z + r0 * n.c, p->acts.z, sizeof(float) * rows * n.c, cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "hn_proposal_logits");
    return HN_OK;
}

}  // extern "C"
