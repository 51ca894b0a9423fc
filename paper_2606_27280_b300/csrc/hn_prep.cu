// HN normalisation (Eq. 1), index packing (§6.1 SoA layout) and query preparation.
#include <math.h>

#include <cuda_fp8.h>

#include "hn_internal.cuh"

namespace hn {

// ------------------------------------------------------------------ Eq. 1
// One thread per row, so that each sum of squares runs in dimension order
// exactly as defined: binary64, products of binary32 values are exact, then
// sqrt and division correctly rounded, each output rounded once to binary32.
// Rows are staged through shared memory (stride 129 words: conflict-free).
constexpr int kNormRows = 64;

__global__ void __launch_bounds__(kNormRows) k_normalize(const float *__restrict__ in,
                                                         float *__restrict__ out, int64_t n, int k,
                                                         double alpha, int32_t *status) {
    __shared__ float s[kNormRows * (kD + 1)];
    const int64_t r0 = (int64_t)blockIdx.x * kNormRows;
    const int rows = (int)min64(kNormRows, n - r0);
    const float *src = in + r0 * kD;
    for (int i = threadIdx.x; i < rows * kD; i += blockDim.x) s[(i / kD) * (kD + 1) + (i % kD)] = src[i];
    __syncthreads();
    const int t = threadIdx.x;
    if (t < rows) {
        float *f = s + t * (kD + 1);
        double s_maj = 0.0, s_min = 0.0;
        for (int c = 0; c < k; ++c) s_maj = fma((double)f[c], (double)f[c], s_maj);
        for (int c = k; c < kD; ++c) s_min = fma((double)f[c], (double)f[c], s_min);
        const bool bad = !isfinite(s_maj) || !isfinite(s_min);
        const bool zero = s_maj == 0.0 || (alpha > 0.0 && s_min == 0.0);
        if (bad || zero) {
            if (status) atomicExch(status + (bad ? ST_NOT_NORMALIZED : ST_ZERO_NORM), 1);
        } else {
            const double c_maj = sqrt(1.0 - alpha) / sqrt(s_maj);
            for (int c = 0; c < k; ++c) f[c] = __double2float_rn((double)f[c] * c_maj);
            if (alpha == 0.0) {
                for (int c = k; c < kD; ++c) f[c] = 0.0f;
            } else {
                const double c_min = sqrt(alpha) / sqrt(s_min);
                for (int c = k; c < kD; ++c) f[c] = __double2float_rn((double)f[c] * c_min);
            }
        }
    }
    __syncthreads();
    float *dst = out + r0 * kD;
    for (int i = threadIdx.x; i < rows * kD; i += blockDim.x) dst[i] = s[(i / kD) * (kD + 1) + (i % kD)];
}

cudaError_t launch_normalize(const float *in, float *out, int64_t n, int k, double alpha,
                             int32_t *status, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + kNormRows - 1) / kNormRows;
    k_normalize<<<(unsigned)blocks, kNormRows, 0, st>>>(in, out, n, k, alpha, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ helpers
__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_max(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// An upper bound, in binary32, on sqrt(s) where s is a binary64 sum of <= 128
// non-negative terms carrying relative error <= 128 * 2^-53 < 2^-45.
__device__ inline float sqrt_up(double s) {
    return __double2float_ru(__dsqrt_ru(s * (1.0 + 0x1p-44)));
}
// An upper bound on the sum over the warp of non-negative binary32 values: every addition
// rounded up (each lane's tree differs, every lane's result is an upper bound).
__device__ inline float warp_sum_up(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// The same bound as sqrt_up, from the binary64 sum, without a binary64 square root.
__device__ inline float sqrt_up32(double s) { return __fsqrt_ru(__double2float_ru(s * (1.0 + 0x1p-44))); }
// Relative tolerance of the norm identities for binary32-stored coordinates.
__device__ inline bool hn_ok(double maj2, double min2, double alpha) {
    const double tol = (kD + 4) * 0x1p-24;
    return fabs(maj2 - (1.0 - alpha)) <= tol * (1.0 - alpha) && fabs(min2 - alpha) <= tol * alpha;
}

__device__ inline float4 bf16_round4(float4 v) {
    return make_float4(__bfloat162float(__float2bfloat16_rn(v.x)), __bfloat162float(__float2bfloat16_rn(v.y)),
                       __bfloat162float(__float2bfloat16_rn(v.z)), __bfloat162float(__float2bfloat16_rn(v.w)));
}

// ------------------------------------------------------------------ FP8 e4m3
// Per-entry scale of the FP8 prefix: the smallest power of two s with
// amax / s <= 448 (the largest finite e4m3 value), x~ = s * x^ exact.  The index
// passes the entry's prefix norm (rounded up) as amax, which bounds every
// component, so no code saturates; HN entries all have prefix norm sqrt(1 - alpha),
// so they share one scale, and the one-pass dense scan can bound a group's largest
// score from its largest raw accumulator without loss.  Relative to a scale from the
// largest component this moves codes down by at most two binades, where e4m3 keeps
// its relative precision (the per-entry error term b_i holds the actual residual).
// amax = 0 (padding) -> 1.
__device__ inline float f8_entry_scale(float amax) {
    if (!(amax > 0.f)) return 1.f;
    int ex;
    frexp((double)amax / 448.0, &ex);
    double s = ldexp(1.0, ex);
    if ((double)amax > 448.0 * s) s *= 2.0;
    return (float)fmax(s, 0x1p-126);
}
__device__ inline uint8_t f8_encode(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ inline float f8_decode(uint8_t b) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3)));
}

// ------------------------------------------------------------------ int8 fixed point
// Code scale of the int8 prefix: the smallest power of two s (>= 2^-100) with
// amax / s <= 127, from frexp, so every code RN(v / s) lies in [-127, 127] and
// the dequantised value s * code is exact.  amax = 0 -> 1.
__device__ inline float i8_scale(float amax) {
    if (!(amax > 0.f)) return 1.f;
    int ex;
    frexp((double)amax / 127.0, &ex);
    return (float)ldexp(1.0, ex < -100 ? -100 : ex);
}
// the code of v at scale s (v / s is exact: s is a power of two)
__device__ inline uint32_t i8_code(float v, float s) {
    return (uint32_t)(uint8_t)(int8_t)__float2int_rn(v / s);
}

// max |x_d| over the prefix columns d < k of all n entries -> dev_max[5]: the
// int8 index takes its one code scale from it (non-negative floats order like
// their bit patterns, so atomicMax on the bits is a float max)
__global__ void __launch_bounds__(256) k_prefix_amax(const float *__restrict__ x, int64_t n, int k,
                                                     float *dev_max) {
    float m = 0.f;
    const int64_t total = n * kD;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        if ((int)(i % kD) < k) m = fmaxf(m, fabsf(x[i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(dev_max) + 5, __float_as_int(m));
}

// ------------------------------------------------------------------ index build
// One warp per entry (grid-stride).  Lane l owns dimensions 4l..4l+3.  Writes
// the FP32 master row, the prefix in the index precision, |x_minor| rounded up,
// and checks the norm identities.  Block maxima of the norms go to dev_max via
// one atomicMax per block (non-negative floats order like their bit patterns).
__global__ void __launch_bounds__(256) k_pack(const float *__restrict__ x, int64_t n, int k, double alpha,
                                              int prefix, int k_pad4, int k_pad16, int64_t n_pad,
                                              float *__restrict__ rows, float *__restrict__ pre32,
                                              __nv_bfloat16 *__restrict__ pre16,
                                              uint8_t *__restrict__ pre8, int8_t *__restrict__ prei8, float qt,
                                              float *__restrict__ mx, float *dev_max, int32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float m_min = 0.f, m_maj = 0.f, m_res = 0.f, m_pre = 0.f, m_full = 0.f;
    const float s8 = prefix == HN_PREFIX_I8 ? i8_scale(dev_max[5]) : 1.f;  // k_prefix_amax ran before
    for (int64_t e = warp; e < n_pad; e += nwarps) {
        const int c0 = lane * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < n) v = reinterpret_cast<const float4 *>(x + e * kD)[lane];
        if (e < n) reinterpret_cast<float4 *>(rows + e * kD)[lane] = v;
        float vv[4] = {v.x, v.y, v.z, v.w};
        double maj2 = 0, min2 = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double d = vv[j];
            if (c0 + j < k) maj2 += d * d; else min2 += d * d;
        }
        // prefix in storage precision (zero beyond k)
        float pv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) pv[j] = (c0 + j < k) ? vv[j] : 0.f;
        float4 p4 = make_float4(pv[0], pv[1], pv[2], pv[3]);
        if (prefix == HN_PREFIX_BF16) p4 = bf16_round4(p4);
        float sc = 1.f;
        uint32_t f8 = 0;  // this lane's 4 e4m3 codes
        if (prefix == HN_PREFIX_FP8_E4M3) {
            const double pn2 = warp_sum((double)pv[0] * pv[0] + (double)pv[1] * pv[1] + (double)pv[2] * pv[2] +
                                        (double)pv[3] * pv[3]);
            sc = f8_entry_scale(sqrt_up(pn2));
            float dq[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint8_t b = f8_encode(pv[j] / sc);  // division by a power of two: exact
                f8 |= (uint32_t)b << (8 * j);
                dq[j] = f8_decode(b) * sc;                // exact
            }
            p4 = make_float4(dq[0], dq[1], dq[2], dq[3]);
        }
        uint32_t i8w = 0;  // this lane's 4 int8 codes
        if (prefix == HN_PREFIX_I8) {
            float dq[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t b = i8_code(pv[j], s8);
                i8w |= b << (8 * j);
                dq[j] = (float)(int8_t)b * s8;  // exact
            }
            p4 = make_float4(dq[0], dq[1], dq[2], dq[3]);
        }
        const float pp[4] = {p4.x, p4.y, p4.z, p4.w};
        double res2 = 0, pre2 = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double r = (double)pv[j] - (double)pp[j];  // exact: both binary32
            res2 += r * r;
            pre2 += (double)pp[j] * (double)pp[j];
        }
        if (prefix == HN_PREFIX_F32 && c0 < k_pad4)
            reinterpret_cast<float4 *>(pre32 + e * k_pad4)[lane] = p4;
        if (prefix == HN_PREFIX_BF16 && c0 < k_pad16) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(p4.x, p4.y), hi = __floats2bfloat162_rn(p4.z, p4.w);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t *>(&lo);
            pk.y = *reinterpret_cast<uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(reinterpret_cast<char *>(pre16) + pre16_offset(e, c0, k_pad16)) = pk;
        }
        if (prefix == HN_PREFIX_I8 && c0 < k_pad16)
            *reinterpret_cast<uint32_t *>(prei8 + e * k_pad16 + c0) = i8w;
        uint8_t *tile8 = nullptr;
        if (prefix == HN_PREFIX_FP8_E4M3) {
            tile8 = pre8 + (e >> 7) * kF8TileBytes(k_pad16);
            if (c0 < k_pad16) *reinterpret_cast<uint32_t *>(tile8 + umma8_offset(e & 127, c0, k_pad16)) = f8;
        }
        maj2 = warp_sum(maj2);
        min2 = warp_sum(min2);
        res2 = warp_sum(res2);
        pre2 = warp_sum(pre2);
        if (tile8 && lane == 0) {
            // per-entry scale and error term b_i = RU(qt * r_i) (a product of two binary32 values is
            // exact in binary64); padding rows get b = 0 and are never reported
            float *sc2 = reinterpret_cast<float *>(tile8 + f8_scale_off(k_pad16));
            const int r = (int)(e & 127);
            sc2[r] = sc / kF8QScale;
            sc2[kF8Tile + r] = e < n ? __double2float_ru((double)qt * (double)sqrt_up(res2)) : 0.f;
        }
        if (e < n) {
            const float umin = sqrt_up(min2), umaj = sqrt_up(maj2), ures = sqrt_up(res2);
            const float upre = sqrt_up(pre2), ufull = sqrt_up(maj2 + min2);
            if (lane == 0) {
                mx[e] = umin;
                if (!hn_ok(maj2, min2, alpha)) {
                    atomicExch(status + ST_NOT_NORMALIZED, 1);
                    atomicMin(status + ST_BAD_ROW, (int32_t)min64(e, 0x7FFFFFFF));
                }
            }
            m_min = fmaxf(m_min, umin);
            m_maj = fmaxf(m_maj, umaj);
            m_res = fmaxf(m_res, ures);
            m_pre = fmaxf(m_pre, upre);
            m_full = fmaxf(m_full, ufull);
        }
    }
    __shared__ float red[5][8];
    const int w = threadIdx.x >> 5;
    if (lane == 0) { red[0][w] = m_min; red[1][w] = m_maj; red[2][w] = m_res; red[3][w] = m_pre; red[4][w] = m_full; }
    __syncthreads();
    if (threadIdx.x < 5) {
        float m = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[threadIdx.x][i]);
        atomicMax(reinterpret_cast<int *>(dev_max) + threadIdx.x, __float_as_int(m));
    }
}

// Per 32-entry group of an FP8 tile: (max s_i, min s_i) / kF8QScale and max b_i over the
// group's real entries (i < n).  A score u_i = RN(acc_i * s_i / 256 + b_i) of the group is
// at most max(RU(A * smax + bmax), RU(A * smin + bmax)) with A = max_i acc_i: the product
// with a positive scale is increasing in acc_i, and linear in the scale, so its largest
// value over the group's scales is at an end of their range.  One thread per group.
__global__ void __launch_bounds__(256) k_f8_group_bounds(uint8_t *__restrict__ pre8, int64_t n, int64_t n_groups,
                                                         int kp) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    uint8_t *tile8 = pre8 + (g >> 2) * kF8TileBytes(kp);
    const float *sc2 = reinterpret_cast<const float *>(tile8 + f8_scale_off(kp));
    const int r0 = (int)(g & 3) * 32;
    float smax = 0.f, smin = INFINITY, bmax = 0.f;
    for (int r = 0; r < 32; ++r) {
        if ((g >> 2) * kF8Tile + r0 + r >= n) break;
        smax = fmaxf(smax, sc2[r0 + r]);
        smin = fminf(smin, sc2[r0 + r]);
        bmax = fmaxf(bmax, sc2[kF8Tile + r0 + r]);
    }
    if (smin == INFINITY) smin = 0.f;
    reinterpret_cast<float4 *>(tile8 + f8_group_off(kp))[g & 3] = make_float4(smax, smin, bmax, 0.f);
}

// The rescore's FP16 rows: every FP32 master row rounded to nearest FP16 (padding rows
// stay zero).  Eight values a thread: two 16-byte loads, one 16-byte store.
__global__ void __launch_bounds__(256) k_rows_f16(const float *__restrict__ rows, __half *__restrict__ rows16,
                                                  int64_t n8) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = reinterpret_cast<const float4 *>(rows)[2 * i];
        const float4 b = reinterpret_cast<const float4 *>(rows)[2 * i + 1];
        const __half2 h0 = __floats2half2_rn(a.x, a.y), h1 = __floats2half2_rn(a.z, a.w);
        const __half2 h2 = __floats2half2_rn(b.x, b.y), h3 = __floats2half2_rn(b.z, b.w);
        uint4 o;
        o.x = *reinterpret_cast<const uint32_t *>(&h0);
        o.y = *reinterpret_cast<const uint32_t *>(&h1);
        o.z = *reinterpret_cast<const uint32_t *>(&h2);
        o.w = *reinterpret_cast<const uint32_t *>(&h3);
        reinterpret_cast<uint4 *>(rows16)[i] = o;
    }
}

cudaError_t launch_pack(Index &ix, const float *x, cudaStream_t st) {
    const int64_t n_pad = ix.n_tiles * kTileE;
    int64_t blocks = (n_pad * 32 + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    if (ix.prefix == HN_PREFIX_I8) {
        k_prefix_amax<<<148 * 8, 256, 0, st>>>(x, ix.n, ix.k, ix.dev_max);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_pack<<<(unsigned)blocks, 256, 0, st>>>(x, ix.n, ix.k, ix.alpha, ix.prefix, ix.k_pad4, ix.k_pad16, n_pad,
                                             ix.rows, ix.pre32, ix.pre16, ix.pre8, ix.prei8, ix.qt, ix.mx,
                                             ix.dev_max,
                                             ix.ws.status);
    if (ix.prefix == HN_PREFIX_FP8_E4M3) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t n_groups = n_pad / 32;
        k_f8_group_bounds<<<(unsigned)((n_groups + 255) / 256), 256, 0, st>>>(ix.pre8, ix.n, n_groups, ix.k_pad16);
    }
    if (ix.rows16) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_rows_f16<<<148 * 16, 256, 0, st>>>(ix.rows, ix.rows16, n_pad * kD / 8);
    }
    return cudaGetLastError();
}

cudaError_t launch_check_hn(const float *, int64_t, int, double, int32_t *, cudaStream_t) {
    return cudaSuccess;  // the check is fused into k_pack and k_query_prep
}

// ------------------------------------------------------------------ queries
// One warp per query.  Produces the query prefix in the scan precision (exact
// FP32 for an FP8 index), the UMMA A-tile copies (BF16 and FP16, or the e4m3
// operands of an FP8 index), |q| rounded up, and the Phase-2 slack
//   E_q >= scan error + |q_minor| * max_i |x_i,minor| + binary64 rounding of the oracle,
// rounded up to binary32.  Scan error:
//   FP32 prefix: gamma_kp * |q_major| * max|x_major|  (recursive FMA summation, Higham Thm 3.1)
//   BF16 prefix: |q_major| * max r(x) + r(q) * max|x^| + gamma' * |q^| * max|x^|,
//     with r(.) the residual norm of the BF16 rounding and gamma' = (kp+2) 2^-20,
//     a deliberately loose accumulation term for the tensor cores' FP32 adder.
//   FP8 prefix: the per-query part of the bound derived below; the per-entry part
//     b_i rides with the entry and is added inside the scan.
__global__ void __launch_bounds__(256) k_query_prep(const float *__restrict__ q, int64_t nq, int64_t nq_pad,
                                                    int k, double alpha, int prefix, int k_pad4, int k_pad16,
                                                    float qt, float minor_scale,
                                                    const float *__restrict__ dev_max, float *__restrict__ qpre32,
                                                    __nv_bfloat16 *__restrict__ qpre16, __half *__restrict__ qpre16h,
                                                    float *__restrict__ qeps, float *__restrict__ qeps32,
                                                    float *__restrict__ qnorm, int32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nq_pad) return;
    const int c0 = lane * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < nq) v = reinterpret_cast<const float4 *>(q + j * kD)[lane];
    const float vv[4] = {v.x, v.y, v.z, v.w};
    // the norm identities need binary64 sums; the bound terms below are upper bounds formed in
    // binary32 with every operation rounded up (binary64 is slow on this GPU)
    double maj2 = 0, min2 = 0;
    float res2 = 0.f, pre2 = 0.f;
    float pv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const double d = vv[t];
        if (c0 + t < k) maj2 += d * d; else min2 += d * d;
        pv[t] = (c0 + t < k) ? vv[t] : 0.f;
    }
    float4 p4 = make_float4(pv[0], pv[1], pv[2], pv[3]);
    if (prefix == HN_PREFIX_BF16) p4 = bf16_round4(p4);
    const float pp[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float r = pv[t] - pp[t];  // exact: the BF16 rounding residual
        res2 = __fmaf_ru(r, r, res2);
        pre2 = __fmaf_ru(pp[t], pp[t], pre2);
    }
    if (c0 < k_pad4) reinterpret_cast<float4 *>(qpre32 + j * k_pad4)[lane] = p4;
    // FP8 index: Phase-2 A operand = e4m3 hi and lo parts of 256 q (q~ = (hi + lo) / 256 carries
    // about 8 significant bits), Phase-1 A operand = e4m3 of 16 q with the lo slots zero.
    // A row holds 2 * k_pad16 bytes: for every 16 prefix columns, 16 hi bytes then 16 lo bytes.
    float rq2 = 0.f, hi2 = 0.f, lo2 = 0.f, qt2 = 0.f;
    if (prefix == HN_PREFIX_FP8_E4M3) {
        uint32_t hw = 0, lw = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float a = pv[t] * kF8QScale;                   // exact
            const uint8_t hb = f8_encode(a);
            const float hf = f8_decode(hb);
            const uint8_t lb = f8_encode(a - hf);                 // a - hf is exact
            const float lf = f8_decode(lb);
            hw |= (uint32_t)hb << (8 * t);
            lw |= (uint32_t)lb << (8 * t);
            const float qq = (hf + lf) / kF8QScale;  // exact
            const float r = pv[t] - qq;               // exact
            rq2 = __fmaf_ru(r, r, rq2);
            hi2 = __fmaf_ru(hf, hf, hi2);
            lo2 = __fmaf_ru(lf, lf, lo2);
            qt2 = __fmaf_ru(qq, qq, qt2);
        }
        if (c0 < k_pad16) {
            const int bc = 32 * (c0 >> 4) + (c0 & 15);
            uint8_t *a2 = reinterpret_cast<uint8_t *>(qpre16);
            *reinterpret_cast<uint32_t *>(a2 + umma8_offset(j, bc, 2 * k_pad16)) = hw;
            *reinterpret_cast<uint32_t *>(a2 + umma8_offset(j, bc + 16, 2 * k_pad16)) = lw;
        }
        rq2 = warp_sum_up(rq2);
        hi2 = warp_sum_up(hi2);
        lo2 = warp_sum_up(lo2);
        qt2 = warp_sum_up(qt2);
    }
    // int8 index: codes q^ = RN(q / t_q) with the query's own power-of-two scale t_q, written as
    // k_pad16 bytes a query into qpre16, and 1 / (t_q s) (a power of two) into qpre16h read as
    // float: the stream scan turns tau_q into an integer threshold with it
    if (prefix == HN_PREFIX_I8) {
        const float tq = i8_scale(warp_max(fmaxf(fmaxf(fabsf(pv[0]), fabsf(pv[1])), fmaxf(fabsf(pv[2]), fabsf(pv[3])))));
        uint32_t w8 = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t b = i8_code(pv[t], tq);
            w8 |= b << (8 * t);
            const float qq = (float)(int8_t)b * tq;  // exact
            const float r = pv[t] - qq;              // exact
            rq2 = __fmaf_ru(r, r, rq2);
            qt2 = __fmaf_ru(qq, qq, qt2);
        }
        if (c0 < k_pad16) *reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(qpre16) + j * k_pad16 + c0) = w8;
        if (lane == 0) reinterpret_cast<float *>(qpre16h)[j] = (float)(1.0 / ((double)tq * (double)i8_scale(dev_max[5])));
        rq2 = warp_sum_up(rq2);
        qt2 = warp_sum_up(qt2);
    }
    if (prefix == HN_PREFIX_BF16 && c0 < k_pad16) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(p4.x, p4.y), hi = __floats2bfloat162_rn(p4.z, p4.w);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t *>(&lo);
        pk.y = *reinterpret_cast<uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(reinterpret_cast<char *>(qpre16) + pre16_offset(j, c0, k_pad16)) = pk;
    }
    maj2 = warp_sum(maj2);
    min2 = warp_sum(min2);
    res2 = warp_sum_up(res2);
    pre2 = warp_sum_up(pre2);
    if (lane != 0 || j >= nq) return;
    if (!hn_ok(maj2, min2, alpha)) atomicExch(status + ST_NOT_NORMALIZED, 1);
    // binary32, every operation rounded up: each term an upper bound of its exact value
    const float qmaj = sqrt_up32(maj2), qmin = sqrt_up32(min2), qres = __fsqrt_ru(res2), qhat = __fsqrt_ru(pre2);
    const float xmin = dev_max[0], xmaj = dev_max[1], xres = dev_max[2], xhat = dev_max[3];
    // gamma_n = n u / (1 - n u), u = 2^-24
    auto gamma = [](int n) { return __fdiv_ru((float)n * 0x1p-24f, __fsub_rd(1.f, (float)n * 0x1p-24f)); };
    float scan;
    if (prefix == HN_PREFIX_F32) {
        scan = __fmul_ru(__fmul_ru(gamma(k_pad4), qmaj), xmaj);
    } else if (prefix == HN_PREFIX_FP8_E4M3) {
        // With x~_i = s_i x^_i (exact), q~ = (hi + lo) / 256 and b_i = RU(qt r_i):
        //   q.x_i = q~.x~_i + (q - q~).x_i + q~.(x_i - x~_i)
        //        <= q~.x~_i + r(q) max|x_major| + |q~| r_i,      |q~| r_i <= b_i + (|q~| - qt)+ max r.
        // The tensor-core scan forms u_i = fma(acc_i, s_i / 256, b_i) with acc_i = (hi + lo).x^_i
        // summed from 2 kp exact products (accumulation error <= (2kp+2) 2^-20 Qa |x~_i|,
        // Qa = (|hi| + |lo|) / 256, the same deliberately loose term as for BF16), one rounding;
        // the CUDA-core scan forms RN(sum_d q_d x~_d + b_i) with the exact FP32 q (FMA chain
        // error <= gamma_kp |q| |x~_i|).  One slack covers both.
        const float qa = __fdiv_ru(__fadd_ru(__fsqrt_ru(hi2), __fsqrt_ru(lo2)), kF8QScale);
        const float qtil = __fsqrt_ru(qt2), rq = __fsqrt_ru(rq2);
        const float acc = fmaxf(__fmul_ru(__fmul_ru((float)(2 * k_pad16 + 2) * 0x1p-20f, qa), xhat),
                                __fmul_ru(__fmul_ru(gamma(k_pad16), qmaj), xhat));
        const float excess = __fmul_ru(fmaxf(0.f, __fsub_ru(fmaxf(qtil, qmaj), qt)), xres);
        const float u_round = __fmul_ru(0x1p-23f, __fadd_ru(__fmul_ru(__fmul_ru(fmaxf(qa, qmaj), xhat), 1.f + 0x1p-10f),
                                                            __fmul_ru(qt, xres)));
        scan = __fadd_ru(__fadd_ru(acc, __fmul_ru(rq, xmaj)), __fadd_ru(excess, u_round));
    } else if (prefix == HN_PREFIX_I8) {
        // With q~ = t_q q^ and x~_i = s x^_i (both exact):
        //   q.x_i = q~.x~_i + (q - q~).x_i + q~.(x_i - x~_i) <= q~.x~_i + r(q) max|x_major| + |q~| max r_i.
        // The scan forms q~.x~_i = t_q s (q^ . x^_i) in integers and tests it against tau_q
        // exactly (an integer threshold), so no rounding term enters.
        scan = __fadd_ru(__fmul_ru(__fsqrt_ru(rq2), xmaj), __fmul_ru(__fsqrt_ru(qt2), xres));
    } else {
        const float g = (float)(k_pad16 + 2) * 0x1p-20f;
        scan = __fadd_ru(__fadd_ru(__fmul_ru(qmaj, xres), __fmul_ru(qres, xhat)), __fmul_ru(__fmul_ru(g, qhat), xhat));
    }
    // the oracle's own binary64 rounding: <= 128 * 2^-53 * |q| |x| < 1e-13 for unit vectors
    // (soft ANN mode: minor_scale = beta / alpha < 1 relaxes the minor bound; 1 is exact)
    const float minor = __fmul_ru(__fmul_ru(minor_scale, qmin), xmin);
    qeps[j] = __fadd_ru(__fadd_ru(scan, minor), 1e-12f);
    // the best-first rescore's bound: an FP32 FMA chain over the K prefix dimensions of the
    // exact query and master row, error <= gamma_K |q_maj| max|x_maj|, plus the full minor
    // bound (alpha, never the soft mode's beta: the rescore keeps the best survivor exactly)
    qeps32[j] = __fadd_ru(__fadd_ru(__fmul_ru(__fmul_ru(gamma(k), qmaj), xmaj), __fmul_ru(qmin, xmin)), 1e-12f);
    qnorm[j] = sqrt_up32(maj2 + min2);
}

cudaError_t launch_query_prep(const Index &ix, const float *q, int64_t nq, float minor_scale, cudaStream_t st) {
    const int64_t nq_pad = (nq + kQPad - 1) / kQPad * kQPad;
    const int64_t blocks = (nq_pad * 32 + 255) / 256;
    k_query_prep<<<(unsigned)blocks, 256, 0, st>>>(q, nq, nq_pad, ix.k, ix.alpha, ix.prefix, ix.k_pad4, ix.k_pad16,
                                                   ix.qt, minor_scale, ix.dev_max, ix.ws.qpre32, ix.ws.qpre16, ix.ws.qpre16h, ix.ws.qeps, ix.ws.qeps32,
                                                   ix.ws.qnorm, ix.ws.status);
    return cudaGetLastError();
}

}  // namespace hn
