// Streaming prefix scan (Phase 1 / Phase 2 of Algorithm 1 on CUDA cores), the
// Phase-1 threshold, the survivor rescore with binary64 near-tie resolution,
// and the FP32 brute-force baseline.
#include <math.h>

#include <algorithm>

#include <cuda_fp8.h>

#include "hn_internal.cuh"

namespace hn {

// ------------------------------------------------------------------ stream scan
// CTA = 64 queries x a contiguous range of 256-entry tiles.  Thread (w, lane)
// owns queries 8w..8w+7 and the tile entries 64 jj + 2 lane + {0, 1} (jj < 4),
// so every thread holds an 8x8 block of prefix scores in registers.  Each score is the FMA
// chain acc = fma(q_c, x_c, acc), c = 0..KT-1 from acc = 0 (zero padding adds
// exact zeros), whose error is bounded by gamma_KT * sum |q_c x_c|.
//   PHASE 1: per-query best (score, lowest index) -> atomicMax on key1[q].
//   PHASE 2: every entry with score >= tau[q] is appended to q's survivor slots.
// FMT selects the stored prefix: 0 FP32, 1 BF16 (UMMA order), 2 FP8 e4m3 tiles,
// dequantised exactly (x~ = s_i x^) while staging; in Phase 2 the FP8 score is
// RN(acc + b_i) with the entry's error term b_i (see the FP8 slack in hn_prep.cu).
// 3 int8 rows: D = q^ . x^ by dp4a, exact.  The accumulator starts at 0x4B400000,
// the bits of 1.5 * 2^23, so while |D| < 2^22 its bits read as the float
// 1.5 * 2^23 + D exactly: the float epilogue below then orders by D unchanged, and
// Phase 2 compares against 1.5 * 2^23 + ceil(tau_q / (t_q s)), which keeps exactly
// the entries with t_q s D >= tau_q.
// The same kernel with KT = 128 over the full rows is the brute-force baseline.
constexpr int kSQ = 64;     // queries per CTA
constexpr int kSE = 256;    // entries per tile
constexpr int kKC = 16;     // prefix columns staged per step

enum { FMT_F32 = 0, FMT_BF16 = 1, FMT_FP8 = 2, FMT_I8 = 3 };
constexpr int kI8Bias = 0x4B400000;  // bits of 1.5 * 2^23

// Phase-2 threshold of an int8 scan: D >= ceil(tau * inv) <=> t_q s D >= tau, with inv =
// 1 / (t_q s) a power of two (the product is exact in binary64); clamped to |.| < 2^22,
// beyond which every D (|D| <= 64 * 127^2) lies on one side anyway
__device__ inline float i8_threshold(float tau, float inv) {
    if (!(tau > -INFINITY)) return -INFINITY;
    const double v = fmin(fmax(ceil((double)tau * (double)inv), -4194303.0), 4194303.0);
    return (float)(12582912.0 + v);
}

template <int KT, int FMT, int PHASE>
__global__ void __launch_bounds__(256, 2)
k_stream_scan(const float *__restrict__ e32, const void *__restrict__ e16, int64_t n, int64_t n_tiles,
              int64_t tiles_per_cta, const float *__restrict__ qpre, int64_t nq, const float *__restrict__ tau,
              unsigned long long *__restrict__ key1, int32_t *__restrict__ bucket, int32_t *__restrict__ count,
              int cap, unsigned long long *__restrict__ cand, const float *__restrict__ qinv) {
    constexpr int KC = KT < kKC ? KT : kKC;
    // staging buffers: two for KT <= 32 (one barrier per staged slice; a buffer is refilled only
    // after the barrier that follows the next slice's staging, which every thread reaches after
    // its last read of it), one for the wider prefixes (48 KB static shared-memory limit)
    constexpr int NB = KT <= 32 ? 2 : 1;
    __shared__ float sq[KT][kSQ];
    // staged entries of the tile, in entry order: thread tid stages entry tid (conflict-free
    // stores), and lane reads its pairs 64 jj + 2 lane + {0, 1} with one 8-byte load each
    __shared__ __align__(16) float se[NB][KC][kSE];
    // FP8 Phase 2: error terms of the tile, by tile parity (written after a barrier that follows
    // every thread's last read of the same parity two tiles back)
    __shared__ __align__(16) float sb[FMT == FMT_FP8 ? 2 : 1][FMT == FMT_FP8 ? kSE : 2];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * kSQ;
    if (FMT == FMT_I8) {
        // int8 codes: KT / 4 words a query, word-column-major in sq's first rows
        constexpr int KW = KT / 4;
        const uint32_t *qw = reinterpret_cast<const uint32_t *>(qpre);
        uint32_t(*sqw)[kSQ] = reinterpret_cast<uint32_t(*)[kSQ]>(&sq[0][0]);
        for (int i = tid; i < kSQ * KW; i += 256) {
            const int qq = i / KW, c = i % KW;
            sqw[c][qq] = (q0 + qq < nq) ? qw[(q0 + qq) * KW + c] : 0u;
        }
    } else {
        for (int i = tid; i < kSQ * KT; i += 256) {
            const int qq = i / KT, c = i % KT;
            sq[c][qq] = (q0 + qq < nq) ? qpre[(q0 + qq) * KT + c] : 0.f;
        }
    }
    float thr[8], best[8];
    uint32_t bidx[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t qg = q0 + w * 8 + i;
        thr[i] = (PHASE == 2 && qg < nq) ? (FMT == FMT_I8 ? i8_threshold(tau[qg], qinv[qg]) : tau[qg]) : INFINITY;
        best[i] = -INFINITY;
        bidx[i] = 0xFFFFFFFFu;
    }
    const int64_t t_begin = (int64_t)blockIdx.y * tiles_per_cta;
    const int64_t t_end = min64(n_tiles, t_begin + tiles_per_cta);
    const int sp = tid;
    int buf = 0;
    // int8: the codes of the next staged slice, loaded one slice ahead so that the load's
    // latency overlaps the current slice's dp4a work (4 registers)
    const int8_t *codes = static_cast<const int8_t *>(e16);
    uint4 i8next = make_uint4(0u, 0u, 0u, 0u);
    if (FMT == FMT_I8 && t_begin < t_end)
        i8next = *reinterpret_cast<const uint4 *>(codes + (t_begin * kSE + tid) * KT);
    for (int64_t t = t_begin; t < t_end; ++t) {
        // acc2[i][jj] = scores of query 8w+i with entries 64 jj + 2 lane (.x) and 64 jj + 2 lane + 1 (.y):
        // packed FMA (fma.rn.f32x2), each half the same FMA chain as a scalar fmaf.  Measured on
        // B300, the packed form runs no more FMAs per second than the scalar one; it pays here
        // because it halves the instructions issued per FMA (8-byte pair loads, one issue per two)
        // (c1, FP32 prefix: Phase 1 15.3 -> 12.1 ms, Phase 2 16.3 -> 12.9 ms).
        float2 acc2[8][4];
        int acci[8][8];  // int8 scan: kI8Bias + D, entry 64 (j / 2) + 2 lane + j % 2
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc2[i][jj] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acci[i][j] = kI8Bias;
        }
        const int64_t e = t * kSE + tid;  // entry staged by this thread
        const uint8_t *tile8 = FMT == FMT_FP8
                                   ? static_cast<const uint8_t *>(e16) + (e >> 7) * kF8TileBytes(KT) : nullptr;
        float esc = 1.f, bterm = 0.f;
        if (FMT == FMT_FP8) {
            const float *sc2 = reinterpret_cast<const float *>(tile8 + f8_scale_off(KT));
            esc = sc2[e & 127] * kF8QScale;  // exact: powers of two
            if (PHASE == 2) bterm = sc2[kF8Tile + (e & 127)];
        }
#pragma unroll 1
        for (int c0 = 0; c0 < KT; c0 += KC) {
            if (NB == 1) __syncthreads();  // every thread has finished reading the single buffer
            if (FMT == FMT_FP8 && PHASE == 2 && c0 == 0) sb[t & 1][tid] = bterm;
            float (*const sx)[kSE] = se[buf];
            uint32_t(*const sxw)[kSE] = reinterpret_cast<uint32_t(*)[kSE]>(&sx[0][0]);
            if (FMT == FMT_I8) {
                // 16 codes = 4 words of this thread's entry, one word-column each
                const uint4 raw = i8next;
                const int64_t tn = c0 + KC < KT ? t : t + 1;  // the slice after this one
                const int cn = c0 + KC < KT ? c0 + KC : 0;
                if (tn < t_end) i8next = *reinterpret_cast<const uint4 *>(codes + (tn * kSE + tid) * KT + cn);
                sxw[0][sp] = raw.x;
                sxw[1][sp] = raw.y;
                sxw[2][sp] = raw.z;
                sxw[3][sp] = raw.w;
            } else if (FMT == FMT_FP8) {
                const uint4 raw = *reinterpret_cast<const uint4 *>(tile8 + umma8_offset(e & 127, c0, KT));
                const __nv_fp8x2_storage_t *h = reinterpret_cast<const __nv_fp8x2_storage_t *>(&raw);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h[u], __NV_E4M3)));
                    sx[2 * u][sp] = f.x * esc;
                    sx[2 * u + 1][sp] = f.y * esc;
                }
            } else if (FMT == FMT_BF16) {
#pragma unroll
                for (int c = 0; c < KC; c += 8) {
                    const uint4 raw = *reinterpret_cast<const uint4 *>(
                        static_cast<const char *>(e16) + pre16_offset(e, c0 + c, KT));
                    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 f = __bfloat1622float2(h[u]);
                        sx[c + 2 * u][sp] = f.x;
                        sx[c + 2 * u + 1][sp] = f.y;
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < KC; c += 4) {
                    const float4 f = *reinterpret_cast<const float4 *>(e32 + e * KT + c0 + c);
                    sx[c][sp] = f.x;
                    sx[c + 1][sp] = f.y;
                    sx[c + 2][sp] = f.z;
                    sx[c + 3][sp] = f.w;
                }
            }
            __syncthreads();
            if (FMT == FMT_I8) {
                const uint32_t(*sqw)[kSQ] = reinterpret_cast<const uint32_t(*)[kSQ]>(&sq[0][0]);
#pragma unroll
                for (int cw = 0; cw < KC / 4; ++cw) {
                    int qa[8];
                    uint2 xb[4];
#pragma unroll
                    for (int i = 0; i < 8; ++i) qa[i] = (int)sqw[c0 / 4 + cw][w * 8 + i];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) xb[jj] = *reinterpret_cast<const uint2 *>(&sxw[cw][jj * 64 + lane * 2]);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            acci[i][2 * jj] = __dp4a(qa[i], (int)xb[jj].x, acci[i][2 * jj]);
                            acci[i][2 * jj + 1] = __dp4a(qa[i], (int)xb[jj].y, acci[i][2 * jj + 1]);
                        }
                }
            } else {
#pragma unroll
            for (int c = 0; c < KC; ++c) {
                float2 a2[8], b2[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float a = sq[c0 + c][w * 8 + i];
                    a2[i] = make_float2(a, a);
                }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) b2[jj] = *reinterpret_cast<const float2 *>(&sx[c][jj * 64 + lane * 2]);
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc2[i][jj] = __ffma2_rn(a2[i], b2[jj], acc2[i][jj]);
            }
            }
            if (NB == 2) buf ^= 1;
        }
        float acc[8][8];  // acc[i][j]: entry 64 (j / 2) + 2 lane + j % 2, increasing in j
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                acc[i][2 * jj] = FMT == FMT_I8 ? __int_as_float(acci[i][2 * jj]) : acc2[i][jj].x;
                acc[i][2 * jj + 1] = FMT == FMT_I8 ? __int_as_float(acci[i][2 * jj + 1]) : acc2[i][jj].y;
            }
        const int64_t ebase = t * kSE + 2 * lane;
        const bool tail = (t + 1) * kSE > n;
        if (FMT == FMT_FP8 && PHASE == 2) {
            float b[8];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const float2 bb = *reinterpret_cast<const float2 *>(&sb[t & 1][64 * jj + 2 * lane]);
                b[2 * jj] = bb.x;
                b[2 * jj + 1] = bb.y;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += b[j];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float m = acc[i][0];
#pragma unroll
            for (int j = 1; j < 8; ++j) m = fmaxf(m, acc[i][j]);
            if (PHASE == 1) {
                if (m > best[i] || tail) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int64_t ei = ebase + 64 * (j >> 1) + (j & 1);
                        if (ei < n && acc[i][j] > best[i]) { best[i] = acc[i][j]; bidx[i] = (uint32_t)ei; }
                    }
                }
            } else {
                if (m >= thr[i]) {
                    const int64_t qg = q0 + w * 8 + i;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int64_t ei = ebase + 64 * (j >> 1) + (j & 1);
                        if (ei < n && acc[i][j] >= thr[i]) {
                            const int slot = atomicAdd(count + qg, 1);
                            if (slot < cap) bucket[qg * cap + slot] = (int32_t)ei;
                        }
                    }
                }
            }
        }
    }
    if (PHASE == 1) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            unsigned long long kbest = bidx[i] == 0xFFFFFFFFu ? 0ull : pack_best(best[i], bidx[i]);
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, kbest, o);
                kbest = other > kbest ? other : kbest;
            }
            const int64_t qg = q0 + w * 8 + i;
            // top-1: the query's best entry; top-k: one best entry per entry range (CTA column)
            if (lane == 0 && qg < nq) {
                if (cand) cand[qg * (int64_t)gridDim.y + blockIdx.y] = kbest;
                else if (kbest) atomicMax(key1 + qg, kbest);
            }
        }
    }
}

// Entry ranges (CTA columns) of the stream scan for nq queries: enough CTAs for ~8 per
// SM; consecutive CTAs share an entry range (L2 reuse).
static void stream_split(int64_t n_tiles, int64_t nq, int64_t *splits_out, int64_t *tpc_out) {
    const int64_t qt = (nq + kSQ - 1) / kSQ;
    int64_t splits = (148 * 8 + qt - 1) / qt;
    splits = max64(1, min64(splits, n_tiles));
    const int64_t tpc = (n_tiles + splits - 1) / splits;
    *splits_out = (n_tiles + tpc - 1) / tpc;
    *tpc_out = tpc;
}

int64_t stream_cand_slots(const Index &ix, int64_t nq) {
    int64_t splits = 0, tpc = 0;
    stream_split(ix.n_tiles, nq, &splits, &tpc);
    return splits;
}

template <int KT, int FMT>
static cudaError_t stream_scan_kt(const float *e32, const void *e16, int64_t n, int64_t n_tiles,
                                  const float *qpre, int64_t nq, int phase, const Workspace &ws, cudaStream_t st,
                                  unsigned long long *cand = nullptr, const float *qinv = nullptr) {
    const int64_t qt = (nq + kSQ - 1) / kSQ;
    int64_t splits = 0, tpc = 0;
    stream_split(n_tiles, nq, &splits, &tpc);
    if (qt > 0x7FFFFFFF || splits > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)qt, (unsigned)splits);
    if (phase == 1)
        k_stream_scan<KT, FMT, 1><<<grid, 256, 0, st>>>(e32, e16, n, n_tiles, tpc, qpre, nq, ws.tau, ws.key1,
                                                         ws.bucket, ws.count, ws.bucket_cap, cand, qinv);
    else
        k_stream_scan<KT, FMT, 2><<<grid, 256, 0, st>>>(e32, e16, n, n_tiles, tpc, qpre, nq, ws.tau, ws.key1,
                                                         ws.bucket, ws.count, ws.bucket_cap, nullptr, qinv);
    return cudaGetLastError();
}

cudaError_t launch_stream_scan(const Index &ix, int64_t nq, int phase, cudaStream_t st, unsigned long long *cand) {
    const Workspace &ws = ix.ws;
    if (ix.prefix == HN_PREFIX_BF16) {
        switch (ix.k_pad16) {
            case 16: return stream_scan_kt<16, FMT_BF16>(nullptr, ix.pre16, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
            case 32: return stream_scan_kt<32, FMT_BF16>(nullptr, ix.pre16, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
            case 64: return stream_scan_kt<64, FMT_BF16>(nullptr, ix.pre16, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
        }
    } else if (ix.prefix == HN_PREFIX_I8) {
        // int8 query codes (qpre16, k_pad16 bytes a query) against the int8 rows
        const float *qc = reinterpret_cast<const float *>(ws.qpre16);
        const float *qi = reinterpret_cast<const float *>(ws.qpre16h);
        switch (ix.k_pad16) {
            case 16: return stream_scan_kt<16, FMT_I8>(nullptr, ix.prei8, ix.n, ix.n_tiles, qc, nq, phase, ws, st, cand, qi);
            case 32: return stream_scan_kt<32, FMT_I8>(nullptr, ix.prei8, ix.n, ix.n_tiles, qc, nq, phase, ws, st, cand, qi);
            case 64: return stream_scan_kt<64, FMT_I8>(nullptr, ix.prei8, ix.n, ix.n_tiles, qc, nq, phase, ws, st, cand, qi);
        }
    } else if (ix.prefix == HN_PREFIX_FP8_E4M3) {
        // exact FP32 query prefix (k_pad16 wide) against the dequantised FP8 prefix
        switch (ix.k_pad16) {
            case 16: return stream_scan_kt<16, FMT_FP8>(nullptr, ix.pre8, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
            case 32: return stream_scan_kt<32, FMT_FP8>(nullptr, ix.pre8, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
            case 64: return stream_scan_kt<64, FMT_FP8>(nullptr, ix.pre8, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
        }
    } else {
        switch (ix.k_pad4) {
            case 8: return stream_scan_kt<8, FMT_F32>(ix.pre32, nullptr, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
            case 16: return stream_scan_kt<16, FMT_F32>(ix.pre32, nullptr, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
            case 32: return stream_scan_kt<32, FMT_F32>(ix.pre32, nullptr, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
            case 64: return stream_scan_kt<64, FMT_F32>(ix.pre32, nullptr, ix.n, ix.n_tiles, ws.qpre32, nq, phase, ws, st, cand);
        }
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ threshold
// Algorithm 1, step 2, with more than one Phase-1 candidate.  Phase 1 leaves S
// candidate keys (prefix score, id) per query: for the stream scan S = 1 (top-1)
// or one per entry range (top-k), the id being an entry; for the dense scan
// S = 2 x chunks (one per entry chunk and tile parity) and the id names a 32-entry
// group whose largest prefix score is the key.  One warp per query takes up to
// R keys, R from 4 to kSeedR = 32 growing with N (see seed_candidates): the R largest
// among each lane's two largest of every 32nd slot (the R largest of all when S <= 64); for a group it recomputes the group's prefix
// scores (FP32 FMA over the BF16 prefix, or the FP8 prefix times its scale) and keeps the
// best valid entry, so the entries are distinct.  Each chosen entry is scored in full in
// FP32, giving the certified lower bound RD(fp32_j - eps_r) <= <q, x_j> (binary64, the
// oracle's value; eps_r bounds the FP32 error of a 128-term sum in any order).  T_q is
// the kk-th largest of these bounds (the largest for the 1-NN): at least kk entries
// score >= T_q, so the kk-th best similarity is >= T_q (-inf when fewer than kk entries
// were found).  Any entry is a valid candidate and the order they are scored in does not
// matter: the choice only decides how tight T_q is.  The Phase-2 prefix threshold is
//   tau_q = RD(T_q - E_q),
// so that prefix_score < tau_q  =>  prefix_score + E_q < T_q  =>  the entry cannot
// be among the kk best.
// Scoring: lane r holds candidate r; kCandLanes lanes score one candidate (the group's
// entries split among them, then kD / kCandLanes dimensions each), 32 / kCandLanes
// candidates at a time, so that their gathers are in flight together.
constexpr int kSeedR = 32;
constexpr int kCandLanes = 8;

__device__ inline float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline float rescore_eps(float qn, float xn_max) {
    return __fmul_ru(__fmul_ru(qn, xn_max), 128 * 0x1p-24 / (1 - 128 * 0x1p-24) + 1e-12f);
}

// FP32 prefix score of entry e read from its master row: qp is zero beyond k, so
// the minor coordinates the loop also reads contribute exact zeros (FP8 index)
__device__ inline float prefix_score_rows(const float *__restrict__ rows, int64_t e, const float *qp, int kp) {
    const float *x = rows + e * kD;
    float s = 0.f;
    for (int c = 0; c < kp; c += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(x + c);
        s = fmaf(qp[c], v.x, s);
        s = fmaf(qp[c + 1], v.y, s);
        s = fmaf(qp[c + 2], v.z, s);
        s = fmaf(qp[c + 3], v.w, s);
    }
    return s;
}

// FP32 prefix score of entry e against the query prefix qp (BF16 values, k_pad16 wide)
__device__ inline float prefix_score16(const __nv_bfloat16 *__restrict__ pre16, int64_t e, const float *qp, int kp) {
    float s = 0.f;
    for (int c = 0; c < kp; c += 8) {
        const uint4 raw = *reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(pre16) + pre16_offset(e, c, kp));
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float2 f = __bfloat1622float2(h[u]);
            s = fmaf(qp[c + 2 * u], f.x, s);
            s = fmaf(qp[c + 2 * u + 1], f.y, s);
        }
    }
    return s;
}

// An FP8 entry's prefix score, s_i * sum_d q_d x^_d (e4m3 codes, the first kp columns;
// kp16 = the tile's row width), from the 128-entry tiles described in hn_internal.cuh.
__device__ inline float prefix_score8(const uint8_t *__restrict__ pre8, int64_t e, const float *qp, int kp, int kp16) {
    const uint8_t *tile = pre8 + (e >> 7) * kF8TileBytes(kp16);
    const int r = (int)(e & 127);
    float s = 0.f;
    for (int c = 0; c < kp; c += 16) {
        const uint4 raw = *reinterpret_cast<const uint4 *>(tile + umma8_offset(r, c, kp16));
        const __nv_fp8x2_storage_t *h = reinterpret_cast<const __nv_fp8x2_storage_t *>(&raw);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h[u], __NV_E4M3)));
            if (c + 2 * u < kp) s = fmaf(qp[c + 2 * u], f.x, s);
            if (c + 2 * u + 1 < kp) s = fmaf(qp[c + 2 * u + 1], f.y, s);
        }
    }
    return s * *reinterpret_cast<const float *>(tile + f8_scale_off(kp16) + 4 * r);
}

__global__ void __launch_bounds__(256) k_seed_threshold(const float *__restrict__ rows, const float *__restrict__ q,
                                                        int64_t nq, int64_t n, const unsigned long long *__restrict__ cand,
                                                        int S, int seg_entries, const __nv_bfloat16 *__restrict__ pre16,
                                                        const uint8_t *__restrict__ pre8, int kp16,
                                                        int kp, const float *__restrict__ qpre32,
                                                        const float *__restrict__ qeps,
                                                        const float *__restrict__ qnorm, float xnorm_max, int kk,
                                                        float *__restrict__ tau, float *__restrict__ tlow,
                                                        int32_t *__restrict__ count,
                                                        int32_t *__restrict__ bucket, int cap, int keep_best, int R) {
    __shared__ unsigned long long s_keys[8][kSeedR];  // 256 threads: eight warps
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nq) return;
    if (lane == 0) count[j] = 0;
    const unsigned long long *cj = cand + j * (int64_t)S;
    // 1. the candidate keys, lane r holding the r-th (0: none); nc = how many lanes hold one
    unsigned long long mine = 0ull;
    int nc = 0;
    {
        // each lane's two largest keys among slots lane, lane + 32, ... (all of them when
        // S <= 64); of these, the non-empty keys of rank < R (rank = larger keys, equal keys
        // by slot), compacted in slot order
        unsigned long long k0 = 0ull, k1 = 0ull;
        for (int s = lane; s < S; s += 32) {
            const unsigned long long k = cj[s];
            if (k > k0) {
                k1 = k0;
                k0 = k;
            } else if (k > k1) {
                k1 = k;
            }
        }
        int r0 = 0, r1 = 0;
        for (int o = 0; o < 32; ++o) {
            const unsigned long long a0 = __shfl_sync(0xffffffffu, k0, o), a1 = __shfl_sync(0xffffffffu, k1, o);
            r0 += (a0 > k0 || (a0 == k0 && o < lane)) + (a1 > k0);
            r1 += (a0 >= k1) + (a1 > k1 || (a1 == k1 && o < lane));
        }
        const bool keep0 = k0 != 0ull && r0 < R, keep1 = k1 != 0ull && r1 < R;
        const unsigned m0 = __ballot_sync(0xffffffffu, keep0), m1 = __ballot_sync(0xffffffffu, keep1);
        const unsigned below = (1u << lane) - 1u;
        if (keep0) s_keys[wib][__popc(m0 & below)] = k0;
        if (keep1) s_keys[wib][__popc(m0) + __popc(m1 & below)] = k1;
        __syncwarp();
        nc = __popc(m0) + __popc(m1);
        mine = lane < nc ? s_keys[wib][lane] : 0ull;
        __syncwarp();
    }
    // 2. score them, four at a time; lane c ends with candidate c's bound and entry
    float lb = -INFINITY;  // lane c: the certified bound of candidate c's entry
    int64_t lb_e = -1;     // and that entry (-1: none)
    const float *qp = qpre32 + j * kp;
    const float eps_r = rescore_eps(qnorm[j], xnorm_max);
    static_assert(32 % kCandLanes == 0 && kCandLanes <= 32, "whole candidates per warp");
    const int g = lane / kCandLanes, t = lane % kCandLanes;
    constexpr int kPerBatch = 32 / kCandLanes;
    for (int c0 = 0; c0 < nc; c0 += kPerBatch) {
        const int c = c0 + g;
        const unsigned long long key = __shfl_sync(0xffffffffu, mine, c & 31);
        int64_t e = (c < nc && key != 0ull) ? (int64_t)best_idx(key) : -1;
        if (seg_entries > 1) {
            // best valid entry of the group by recomputed prefix score (lowest index on ties)
            unsigned long long kb = 0;
            if (e >= 0) {
                const int64_t e0 = e * seg_entries;
                for (int i = t; i < seg_entries; i += kCandLanes) {
                    const int64_t ei = e0 + i;
                    if (ei < n) {
                        const float sc = pre16  ? prefix_score16(pre16, ei, qp, kp)
                                         : pre8 ? prefix_score8(pre8, ei, qp, kp, kp16)
                                                : prefix_score_rows(rows, ei, qp, kp);
                        const unsigned long long k2 = pack_best(sc, (uint32_t)ei);
                        kb = k2 > kb ? k2 : kb;
                    }
                }
            }
#pragma unroll
            for (int o = kCandLanes / 2; o; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, kb, o);
                kb = other > kb ? other : kb;
            }
            e = kb ? (int64_t)best_idx(kb) : -1;
        }
        // full FP32 score: kD / kCandLanes dimensions a lane, then a sum over the candidate's lanes
        constexpr int kRowF4 = kD / 4 / kCandLanes;  // float4 pieces of the row a lane takes
        static_assert(kRowF4 * 4 * kCandLanes == kD, "the candidate's lanes cover the row exactly");
        float sim = 0.f;
        if (e >= 0) {
            const float4 *qr = reinterpret_cast<const float4 *>(q + j * kD) + kRowF4 * t;
            const float4 *xr = reinterpret_cast<const float4 *>(rows + e * kD) + kRowF4 * t;
#pragma unroll
            for (int u = 0; u < kRowF4; ++u) {
                const float4 a = qr[u], x = xr[u];
                sim = fmaf(a.x, x.x, sim);
                sim = fmaf(a.y, x.y, sim);
                sim = fmaf(a.z, x.z, sim);
                sim = fmaf(a.w, x.w, sim);
            }
        }
#pragma unroll
        for (int o = kCandLanes / 2; o; o >>= 1) sim += __shfl_xor_sync(0xffffffffu, sim, o);
        const float bound = __fsub_rd(sim, eps_r);
#pragma unroll
        for (int gi = 0; gi < kPerBatch; ++gi) {
            const float v = __shfl_sync(0xffffffffu, bound, gi * kCandLanes);
            const int64_t ve = __shfl_sync(0xffffffffu, e, gi * kCandLanes);
            if (lane == c0 + gi && ve >= 0) {
                lb = v;
                lb_e = ve;
            }
        }
    }
    const unsigned vmask = __ballot_sync(0xffffffffu, lb_e >= 0);
    const int found = __popc(vmask);
    // the kk-th largest bound: the lane whose value has exactly kk-1 larger ones (ties by lane)
    float t_low = -INFINITY;
    if (found >= kk) {
        int rank = 0;
        for (int o = 0; o < 32; ++o) {
            const float v = __shfl_sync(0xffffffffu, lb, o);
            rank += (((vmask >> o) & 1u) && (v > lb || (v == lb && o < lane))) ? 1 : 0;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, lb_e >= 0 && rank == kk - 1);
        t_low = __shfl_sync(0xffffffffu, lb, __ffs(hit) - 1);
    }
    if (lane == 0) {
        tau[j] = t_low == -INFINITY ? -INFINITY : __fsub_rd(t_low, qeps[j]);
        tlow[j] = t_low;
    }
    if (keep_best && found > 0) {
        // soft ANN mode: the relaxed bound may prune every entry, the scored candidates
        // included; like Algorithm 1's Phase-1 winner, the best candidate is always kept
        // (survivor slot 0; Phase 2 appends after it)
        float bv = lb;
        int64_t be = lb_e;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int64_t oe = __shfl_xor_sync(0xffffffffu, be, o);
            if (oe >= 0 && (be < 0 || ov > bv || (ov == bv && oe < be))) { bv = ov; be = oe; }
        }
        if (lane == 0 && be >= 0 && cap > 0) {
            bucket[j * (int64_t)cap] = (int32_t)be;
            count[j] = 1;
        }
    }
}

// Threshold from the learned proposal: for each of the query's top-k blocks, the
// entry of best prefix score (FP32 FMA over the stored prefix, lowest id on
// ties) is scored in full; T_q and tau_q follow as for the Phase-1 candidates.
__global__ void __launch_bounds__(256) k_seed_blocks(const float *__restrict__ rows, const float *__restrict__ q,
                                                     int64_t nq, const float *__restrict__ pre32,
                                                     const __nv_bfloat16 *__restrict__ pre16, int kp,
                                                     const float *__restrict__ qpre32, const int32_t *__restrict__ blocks,
                                                     int topk, const int32_t *__restrict__ block_start,
                                                     const int32_t *__restrict__ block_ids, const float *__restrict__ qeps,
                                                     const float *__restrict__ qnorm, float xnorm_max,
                                                     float *__restrict__ tau, float *__restrict__ tlow,
                                                     int32_t *__restrict__ count,
                                                     int32_t *__restrict__ bucket, int cap, int keep_best) {
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nq) return;
    if (lane == 0) count[j] = 0;
    const float4 qv = reinterpret_cast<const float4 *>(q + j * kD)[lane];
    const float *qp = qpre32 + j * kp;
    const float eps_r = rescore_eps(qnorm[j], xnorm_max);
    float t_low = -INFINITY;
    int64_t t_e = -1;  // the entry giving t_low
    for (int r = 0; r < topk; ++r) {
        const int32_t b = blocks[j * topk + r];
        unsigned long long kb = 0;
        for (int32_t p = block_start[b] + lane; p < block_start[b + 1]; p += 32) {
            const int32_t e = block_ids[p];
            float sc;
            if (pre16) {
                sc = prefix_score16(pre16, e, qp, kp);
            } else if (!pre32) {
                sc = prefix_score_rows(rows, e, qp, kp);
            } else {
                sc = 0.f;
                const float *xe = pre32 + (int64_t)e * kp;
                for (int c = 0; c < kp; ++c) sc = fmaf(qp[c], xe[c], sc);
            }
            const unsigned long long kk = pack_best(sc, (uint32_t)e);
            kb = kk > kb ? kk : kb;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, kb, o);
            kb = other > kb ? other : kb;
        }
        if (kb == 0ull) continue;
        const float4 xv = reinterpret_cast<const float4 *>(rows + (int64_t)best_idx(kb) * kD)[lane];
        const float sim = warp_sum_f(fmaf(qv.x, xv.x, fmaf(qv.y, xv.y, fmaf(qv.z, xv.z, qv.w * xv.w))));
        const float lbv = __fsub_rd(sim, eps_r);
        if (lbv > t_low) { t_low = lbv; t_e = best_idx(kb); }
    }
    if (lane == 0) {
        tau[j] = t_low == -INFINITY ? -INFINITY : __fsub_rd(t_low, qeps[j]);
        tlow[j] = t_low;
        if (keep_best && t_e >= 0 && cap > 0) {  // soft ANN mode: keep the best candidate (see above)
            bucket[j * (int64_t)cap] = (int32_t)t_e;
            count[j] = 1;
        }
    }
}

cudaError_t launch_seed_blocks(const Index &ix, const float *q, int64_t nq, const int32_t *blocks, int topk,
                               bool keep_best, cudaStream_t st) {
    const Workspace &ws = ix.ws;
    const int64_t gblocks = (nq * 32 + 255) / 256;
    // FP32 and BF16 indexes score candidates on their stored prefix, an FP8 index on its master rows
    k_seed_blocks<<<(unsigned)gblocks, 256, 0, st>>>(ix.rows, q, nq, ix.pre32, ix.pre16, ix.k_pad4, ws.qpre32, blocks, topk,
                                                     ix.block_start, ix.block_ids, ws.qeps, ws.qnorm, ix.host_max[4],
                                                     ws.tau, ws.tlow, ws.count, ws.bucket, ws.bucket_cap,
                                                     keep_best ? 1 : 0);
    return cudaGetLastError();
}

// Phase-1 argmax of the stream scan over explicit FP32 arrays (k-means assignment).
cudaError_t stream_argmax_f32(const float *db_pre, int64_t n_db, int64_t n_db_tiles, int kp, const float *q_pre,
                              int64_t nq, unsigned long long *keys, cudaStream_t st) {
    Workspace w{};
    w.key1 = keys;
    switch (kp) {
        case 8: return stream_scan_kt<8, FMT_F32>(db_pre, nullptr, n_db, n_db_tiles, q_pre, nq, 1, w, st);
        case 16: return stream_scan_kt<16, FMT_F32>(db_pre, nullptr, n_db, n_db_tiles, q_pre, nq, 1, w, st);
        case 32: return stream_scan_kt<32, FMT_F32>(db_pre, nullptr, n_db, n_db_tiles, q_pre, nq, 1, w, st);
        case 64: return stream_scan_kt<64, FMT_F32>(db_pre, nullptr, n_db, n_db_tiles, q_pre, nq, 1, w, st);
    }
    return cudaErrorInvalidValue;
}

// Candidates scored per query: each costs the same at any N, while the survivors a tighter
// threshold removes grow with N -- one per 2^17 entries, 4 to 32, and at least kk.
static int seed_candidates(int64_t n, int kk) {
    const int64_t r = std::min<int64_t>(kSeedR, std::max<int64_t>(4, n >> 17));
    return (int)std::max<int64_t>(r, std::min(kk, kSeedR));
}

cudaError_t launch_seed_threshold(const Index &ix, const float *q, int64_t nq, bool dense, int kk, bool keep_best,
                                  cudaStream_t st) {
    const Workspace &ws = ix.ws;
    const int64_t blocks = (nq * 32 + 255) / 256;
    // candidates: the dense Phase 1's 32-entry groups, or (top-k) the stream scan's per-range
    // entries, or its best entry
    const bool multi = dense || kk > 1;
    const int S = dense ? (int)dense_phase1_slots(ix, nq) : multi ? ws.cand_slots : 1;
    k_seed_threshold<<<(unsigned)blocks, 256, 0, st>>>(ix.rows, q, nq, ix.n, multi ? ws.cand : ws.key1,
                                                       S, dense ? 32 : 1, ix.pre16, ix.pre8, ix.k_pad16,
                                                       ix.k_pad4, ws.qpre32, ws.qeps, ws.qnorm, ix.host_max[4], kk,
                                                       ws.tau, ws.tlow, ws.count, ws.bucket, ws.bucket_cap,
                                                       keep_best ? 1 : 0, seed_candidates(ix.n, kk));
    return cudaGetLastError();
}

cudaError_t launch_seed_threshold_at(const Index &ix, const float *q, int64_t q0, int64_t nq, int S, int seg_entries,
                                     int kk, bool keep_best, cudaStream_t st) {
    const Workspace &ws = ix.ws;
    const int64_t blocks = (nq * 32 + 255) / 256;
    const int cap = ws.bucket_cap;
    k_seed_threshold<<<(unsigned)blocks, 256, 0, st>>>(ix.rows, q + q0 * kD, nq, ix.n, ws.cand + q0 * S, S, seg_entries,
                                                       ix.pre16, ix.pre8, ix.k_pad16, ix.k_pad4,
                                                       ws.qpre32 + q0 * ix.k_pad4, ws.qeps + q0,
                                                       ws.qnorm + q0, ix.host_max[4], kk, ws.tau + q0, ws.tlow + q0,
                                                       ws.count + q0, ws.bucket + q0 * cap, cap, keep_best ? 1 : 0,
                                                       seed_candidates(ix.n, kk));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ rescore
// One warp per query.  For every survivor i: FP32 128-dim score (lane l owns
// dims 4l..4l+3, then a butterfly sum), error <= eps_r = gamma_128 |q| max|x|
// (any summation order of 128 terms).  The winner w.r.t. the oracle's binary64
// value must lie in the band  fp32_i >= best_fp32 - 2 eps_r;  band members are
// re-scored in binary64 in dimension order (bit-identical to the oracle) and
// the (score desc, index asc) maximum is the answer.  The band is kept in
// lane-distributed registers (<= 32 members); a larger band falls back to
// binary64 for every survivor of that query.
__device__ inline double dot64_seq(const float *__restrict__ a, const float *__restrict__ b) {
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < kD; ++c) s = fma((double)a[c], (double)b[c], s);
    return s;
}

// FP32 prefix score over the K leading dimensions of a master row (FMA chain in order),
// the query's prefix in qs (exact FP32 values); error <= gamma_K |q_maj| |x_maj|.
__device__ inline float prefix_score32(const float *__restrict__ x, const float *qs, int k) {
    float s = 0.f;
    for (int c = 0; c < k; ++c) s = fmaf(qs[c], x[c], s);
    return s;
}

// One FP32 full score v of entry id (warp-uniform) into the rescore state: the FP32
// best, and the band members (FP32 score within 2 eps_r of the best) held one per lane.
__device__ __forceinline__ void band_push(float v, int32_t id, float band, int lane, float &best32, float &cval,
                                          int32_t &cidx, int &ncand, bool &spill) {
    if (v > best32) {
        // new FP32 best: keep only band members still within 2 eps_r of it
        best32 = v;
        const bool keep = lane < ncand && cval >= __fsub_rd(best32, band);
        const unsigned mk = __ballot_sync(0xffffffffu, keep);
        const int nk = __popc(mk);
        unsigned rest = mk;  // clear the `lane` lowest set bits: the next one is member #lane
        for (int p = 0; p < lane && rest; ++p) rest &= rest - 1;
        const int src = rest ? __ffs(rest) - 1 : 0;
        const float nv = __shfl_sync(0xffffffffu, cval, src);
        const int32_t ni = __shfl_sync(0xffffffffu, cidx, src);
        cval = lane < nk ? nv : -INFINITY;
        cidx = lane < nk ? ni : -1;
        ncand = nk;
    }
    if (v >= __fsub_rd(best32, band)) {
        if (ncand < 32) {
            if (lane == ncand) { cval = v; cidx = id; }
            ++ncand;
        } else {
            spill = true;
        }
    }
}

// The binary64 step: band members (or, after a spill, every survivor) scored in the
// oracle's order, and the (score desc, index asc) maximum written out.
__device__ __forceinline__ void rescore_finish(const float *__restrict__ rows, const float *__restrict__ q, int64_t j,
                                               const int32_t *bk, int cnt, int lane, bool spill, int ncand,
                                               int32_t cidx, int64_t *__restrict__ out_idx,
                                               double *__restrict__ out_sim, long long *__restrict__ counters) {
    double bs = -INFINITY;
    int64_t bi = -1;
    if (!spill) {
        if (lane < ncand) { bs = dot64_seq(q + j * kD, rows + (int64_t)cidx * kD); bi = cidx; }
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_FP64), (unsigned long long)ncand);
    } else {
        for (int s = lane; s < cnt; s += 32) {
            const int32_t id = bk[s];
            const double v = dot64_seq(q + j * kD, rows + (int64_t)id * kD);
            if (v > bs || (v == bs && id < bi)) { bs = v; bi = id; }
        }
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_FP64), (unsigned long long)cnt);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, bs, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || os > bs || (os == bs && oi < bi))) { bs = os; bi = oi; }
    }
    if (lane == 0) {
        out_idx[j] = bi;
        out_sim[j] = bs;
    }
}

__global__ void __launch_bounds__(256) k_rescore(const float *__restrict__ rows, const float *__restrict__ q,
                                                 int64_t nq, const int32_t *__restrict__ bucket,
                                                 const int32_t *__restrict__ count, int cap,
                                                 const float *__restrict__ qnorm, float xnorm_max,
                                                 int64_t *__restrict__ out_idx, double *__restrict__ out_sim,
                                                 int32_t *__restrict__ status, long long *__restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nq) return;
    const int cnt = count[j];
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_SURVIVORS), (unsigned long long)cnt);
        atomicMax(reinterpret_cast<unsigned long long *>(counters + CT_MAXSURV), (unsigned long long)cnt);
    }
    if (cnt > cap) {  // survivors were dropped: the host re-runs with more slots
        if (lane == 0) atomicExch(status + ST_OVERFLOW, 1);
        return;
    }
    const float4 qv = reinterpret_cast<const float4 *>(q + j * kD)[lane];
    const float eps = rescore_eps(qnorm[j], xnorm_max);
    const float band = __fmul_ru(2.f, eps);
    const int32_t *bk = bucket + j * (int64_t)cap;
    float best32 = -INFINITY;
    float cval = -INFINITY;   // band member held by this lane
    int32_t cidx = -1;
    int ncand = 0;
    bool spill = false;
    constexpr int U = 8;  // survivor rows in flight per warp
    for (int s0 = 0; s0 < cnt; s0 += U) {
        float part[U];
        int32_t id[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            id[u] = (s0 + u < cnt) ? bk[s0 + u] : -1;
            float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (id[u] >= 0) xv = reinterpret_cast<const float4 *>(rows + (int64_t)id[u] * kD)[lane];
            part[u] = fmaf(qv.x, xv.x, fmaf(qv.y, xv.y, fmaf(qv.z, xv.z, qv.w * xv.w)));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
#pragma unroll
            for (int u = 0; u < U; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], o);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (id[u] >= 0) band_push(part[u], id[u], band, lane, best32, cval, cidx, ncand, spill);
    }
    rescore_finish(rows, q, j, bk, cnt, lane, spill, ncand, cidx, out_idx, out_sim, counters);
}

// Best-first rescore (the early exit of a sorted Phase 2 that the remark after
// Algorithm 1 describes).  A sorted Phase 2 reaches a good full score early and then
// drops every entry whose bound cannot beat it.  Here the threshold kernel has already
// scored the best prefix candidates in full: their best certified lower bound T_q
// starts the cut, and a survivor is scored in full only if its bound, an FP32 prefix
// score over the master row plus eps32, reaches cut = max(T_q, RD(best32 - eps_r)),
// which rises with every better FP32 score.  A survivor below the cut has similarity
// < cut <= max, so it can neither win nor tie the winner: the answer is unchanged, and
// each such survivor costs a read of its K prefix values instead of its whole row.
__global__ void __launch_bounds__(256) k_rescore_bf(const float *__restrict__ rows, const float *__restrict__ q,
                                                    int64_t nq, const int32_t *__restrict__ bucket,
                                                    const int32_t *__restrict__ count, int cap,
                                                    const float *__restrict__ qnorm, float xnorm_max,
                                                    const float *__restrict__ qeps32, const float *__restrict__ tlow,
                                                    int k, int64_t *__restrict__ out_idx, double *__restrict__ out_sim,
                                                    int32_t *__restrict__ status, long long *__restrict__ counters) {
    __shared__ float qsh[8][64];  // the query prefix of each warp (zeros beyond K)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nq) return;
    const int cnt = count[j];
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_SURVIVORS), (unsigned long long)cnt);
        atomicMax(reinterpret_cast<unsigned long long *>(counters + CT_MAXSURV), (unsigned long long)cnt);
    }
    if (cnt > cap) {
        if (lane == 0) atomicExch(status + ST_OVERFLOW, 1);
        return;
    }
    const float4 qv = reinterpret_cast<const float4 *>(q + j * kD)[lane];
    const float eps = rescore_eps(qnorm[j], xnorm_max);
    const float band = __fmul_ru(2.f, eps);
    const int32_t *bk = bucket + j * (int64_t)cap;
    float best32 = -INFINITY;
    float cval = -INFINITY;
    int32_t cidx = -1;
    int ncand = 0;
    bool spill = false;
    constexpr int U = 8;
    for (int c = lane; c < 64; c += 32) qsh[wib][c] = c < k ? q[j * kD + c] : 0.f;
    __syncwarp();
    const float *qs = qsh[wib];
    const float e32 = qeps32[j];
    float cut = tlow[j];
    long long skipped = 0;
    for (int s0 = 0; s0 < cnt; s0 += 32) {
        const int s = s0 + lane;
        bool keep = false;
        if (s < cnt) {
            keep = __fadd_ru(prefix_score32(rows + (int64_t)bk[s] * kD, qs, k), e32) >= cut;
            skipped += keep ? 0 : 1;
        }
        unsigned mk = __ballot_sync(0xffffffffu, keep);
        while (mk) {
            // up to U kept survivors: FP32 full scores (warp-cooperative rows)
            int32_t id[U];
            float part[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int src = mk ? __ffs(mk) - 1 : -1;
                if (mk) mk &= mk - 1;
                id[u] = src >= 0 ? bk[s0 + src] : -1;
                float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (id[u] >= 0) xv = reinterpret_cast<const float4 *>(rows + (int64_t)id[u] * kD)[lane];
                part[u] = fmaf(qv.x, xv.x, fmaf(qv.y, xv.y, fmaf(qv.z, xv.z, qv.w * xv.w)));
            }
#pragma unroll
            for (int o = 16; o; o >>= 1)
#pragma unroll
                for (int u = 0; u < U; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], o);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (id[u] >= 0) band_push(part[u], id[u], band, lane, best32, cval, cidx, ncand, spill);
        }
        cut = fmaxf(cut, __fsub_rd(best32, eps));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) skipped += __shfl_xor_sync(0xffffffffu, skipped, o);
    if (lane == 0 && skipped)
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_SKIPPED), (unsigned long long)skipped);
    rescore_finish(rows, q, j, bk, cnt, lane, spill, ncand, cidx, out_idx, out_sim, counters);
}

// The default 1-NN rescore: a certified FP16 filter in front of Algorithm 1's Phase-2 full
// scores.  Eq. 3 lets through every entry whose prefix bound reaches the threshold, and most
// of them end far below the best full score.  Each survivor's binary64 similarity is bounded
// from above by the FP32 dot of the query against the entry's FP16 row (256 B instead of the
// 512 B FP32 row): with x~_d = RN_fp16(x_d),
//   |x~_d - x_d| <= 2^-11 |x_d| + 2^-25          (normal and subnormal FP16 spacing)
//   |sum q_d x~_d - sum q_d x_d| <= 2^-11 |q||x| + 2^-25 sqrt(128) |q|
//   |FP32 dot - sum q_d x~_d| <= gamma_128 (1 + 2^-11) |q||x|  (any summation order)
// so ub = RU(dot + e16) >= the similarity, e16 = RU(|q| (|x|max c1 + c2)).  Only survivors
// with ub >= cut are read in FP32 and pass through the band and binary64 steps of k_rescore;
// cut starts at T_q (the threshold candidates' certified lower bound) and rises with the
// FP32 best as in k_rescore_bf.  A survivor with ub < cut has similarity < cut <= the best
// similarity, so it can neither win nor tie the winner: the answer is unchanged.
__device__ inline float rescore16_slack(float qn, float xn_max) {
    constexpr float c1 = 4.96e-4f;   // >= 2^-11 + gamma_128 (1 + 2^-11) + 1e-12
    constexpr float c2 = 3.4e-7f;    // >= 2^-25 sqrt(128)
    return __fmul_ru(qn, __fadd_ru(__fmul_ru(xn_max, c1), c2));
}

// Up to 32 kept survivors of one query (bit src of mk: the survivor whose id lane src holds):
// their FP32 full scores, eight warp-cooperative rows at a time, into the band state.
__device__ __forceinline__ void rescore_kept(unsigned mk, int32_t lane_id, const float *__restrict__ rows,
                                             float4 qv, float band, int lane, float &best32, float &cval,
                                             int32_t &cidx, int &ncand, bool &spill) {
    constexpr int V = 8;
    while (mk) {
        int32_t id[V];
        float full[V];
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const int src = mk ? __ffs(mk) - 1 : 0;
            const bool live = mk != 0;
            if (mk) mk &= mk - 1;
            id[t] = __shfl_sync(0xffffffffu, lane_id, src);
            if (!live) id[t] = -1;
            float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (id[t] >= 0) xv = reinterpret_cast<const float4 *>(rows + (int64_t)id[t] * kD)[lane];
            full[t] = fmaf(qv.x, xv.x, fmaf(qv.y, xv.y, fmaf(qv.z, xv.z, qv.w * xv.w)));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
#pragma unroll
            for (int t = 0; t < V; ++t) full[t] += __shfl_xor_sync(0xffffffffu, full[t], o);
#pragma unroll
        for (int t = 0; t < V; ++t)
            if (id[t] >= 0) band_push(full[t], id[t], band, lane, best32, cval, cidx, ncand, spill);
    }
}

// Queries with at most this many survivors bound them one per lane (each lane reads its
// row's 256 B itself); queries with more give each survivor eight lanes (32 B of the row a
// lane, four survivors per load instruction, so a row costs two cache-line requests instead
// of sixteen).  Measured on B300: one per lane is faster at a few hundred survivors a query
// (c2), eight lanes at thousands (c4's K = 8, alpha = 1/8 indexes, about 17 thousand a
// query).  Both forms stay in one launch (a second launch for the large queries left them
// as a serial tail), bounded to four blocks per SM.
constexpr int kRescoreLaneMax = 2048;

__global__ void __launch_bounds__(256, 4) k_rescore16(const float *__restrict__ rows, const __half *__restrict__ rows16,
                                                   const float *__restrict__ q, int64_t nq,
                                                   const int32_t *__restrict__ bucket,
                                                   const int32_t *__restrict__ count, int cap,
                                                   const float *__restrict__ qnorm, float xnorm_max,
                                                   const float *__restrict__ tlow, int64_t *__restrict__ out_idx,
                                                   double *__restrict__ out_sim, int32_t *__restrict__ status,
                                                   long long *__restrict__ counters) {
    __shared__ float4 qsh[8][kD / 4];  // each warp's query, read by broadcast (one survivor a lane)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nq) return;
    const int cnt = count[j];
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_SURVIVORS), (unsigned long long)cnt);
        atomicMax(reinterpret_cast<unsigned long long *>(counters + CT_MAXSURV), (unsigned long long)cnt);
    }
    if (cnt > cap) {
        if (lane == 0) atomicExch(status + ST_OVERFLOW, 1);
        return;
    }
    // lane l holds query coordinates 4l .. 4l+3 (warp-cooperative FP32 rows)
    const float4 qv = reinterpret_cast<const float4 *>(q + j * kD)[lane];
    const float eps = rescore_eps(qnorm[j], xnorm_max);
    const float e16 = rescore16_slack(qnorm[j], xnorm_max);
    const float band = __fmul_ru(2.f, eps);
    const int32_t *bk = bucket + j * (int64_t)cap;
    float best32 = -INFINITY;
    float cval = -INFINITY;
    int32_t cidx = -1;
    int ncand = 0;
    bool spill = false;
    float cut = tlow[j];
    int kept_total = 0;
    qsh[wib][lane] = qv;
    __syncwarp();
    const float4 *qs = qsh[wib];
    if (cnt <= kRescoreLaneMax) {
        for (int s0 = 0; s0 < cnt; s0 += 32) {
            const int s = s0 + lane;
            const int32_t my_id = s < cnt ? bk[s] : -1;
            bool keep = false;
            if (my_id >= 0) {
                // this lane's survivor: FP32 dot over its FP16 row, four partial sums
                const uint4 *r = reinterpret_cast<const uint4 *>(rows16 + (int64_t)my_id * kD);
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                for (int i = 0; i < kD / 8; ++i) {
                    const uint4 v = __ldg(r + i);
                    const float4 qa = qs[2 * i], qb = qs[2 * i + 1];
                    const float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
                    const float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
                    const float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&v.z));
                    const float2 f3 = __half22float2(*reinterpret_cast<const __half2 *>(&v.w));
                    a0 = fmaf(qa.x, f0.x, fmaf(qa.y, f0.y, a0));
                    a1 = fmaf(qa.z, f1.x, fmaf(qa.w, f1.y, a1));
                    a2 = fmaf(qb.x, f2.x, fmaf(qb.y, f2.y, a2));
                    a3 = fmaf(qb.z, f3.x, fmaf(qb.w, f3.y, a3));
                }
                keep = __fadd_ru((a0 + a1) + (a2 + a3), e16) >= cut;
            }
            const unsigned mk = __ballot_sync(0xffffffffu, keep);
            kept_total += __popc(mk);
            rescore_kept(mk, my_id, rows, qv, band, lane, best32, cval, cidx, ncand, spill);
            cut = fmaxf(cut, __fsub_rd(best32, eps));
        }
    } else {
        // eight lanes a survivor: lane 8g + t reads bytes 32t .. 32t+31 of the FP16 row of
        // survivor 4u + g of the batch against query coordinates 16t .. 16t+15 (shared memory)
        const int g = lane >> 3, t = lane & 7;
        const float4 *qt = qs + 4 * t;
        constexpr int U = 4;  // 16 survivors a batch, two 16-byte loads a lane each
        for (int s0 = 0; s0 < cnt; s0 += 4 * U) {
            int32_t sid[U];
            float part[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int s = s0 + 4 * u + g;
                sid[u] = s < cnt ? bk[s] : -1;
                uint4 v0 = make_uint4(0u, 0u, 0u, 0u), v1 = v0;
                if (sid[u] >= 0) {
                    const uint4 *r = reinterpret_cast<const uint4 *>(rows16 + (int64_t)sid[u] * kD + 16 * t);
                    v0 = __ldg(r);
                    v1 = __ldg(r + 1);
                }
                const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const float4 qa = qt[i >> 1];
                    const float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&w[i]));
                    const float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&w[i + 1]));
                    a0 = fmaf(qa.x, f0.x, fmaf(qa.y, f0.y, a0));
                    a1 = fmaf(qa.z, f1.x, fmaf(qa.w, f1.y, a1));
                }
                part[u] = a0 + a1;
            }
            // the octet's butterfly leaves the same sum in its eight lanes
#pragma unroll
            for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                for (int u = 0; u < U; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], o);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                // lanes 0, 8, 16, 24 vote for survivors 4u .. 4u+3 and hold their ids
                const bool keep = t == 0 && sid[u] >= 0 && __fadd_ru(part[u], e16) >= cut;
                const unsigned mk = __ballot_sync(0xffffffffu, keep);
                kept_total += __popc(mk);
                rescore_kept(mk, sid[u], rows, qv, band, lane, best32, cval, cidx, ncand, spill);
            }
            cut = fmaxf(cut, __fsub_rd(best32, eps));
        }
    }
    if (lane == 0 && cnt > kept_total)
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_SKIPPED), (unsigned long long)(cnt - kept_total));
    rescore_finish(rows, q, j, bk, cnt, lane, spill, ncand, cidx, out_idx, out_sim, counters);
}

// Exact top-kk (1 <= kk <= 32), one warp per query.  Pass 1 finds f_k, the kk-th
// largest FP32 score among the survivors (lane r holds the r-th largest value).
// Every entry of the exact top-kk has binary64 score >= f_k - eps_r (kk survivors
// score at least that), so its FP32 score is >= f_k - 2 eps_r: pass 2 scores the
// survivors in that band in binary64 in dimension order (the oracle's value) and the
// kk largest by (score desc, index asc) are the answer.  Band members sit two per
// lane (<= 64); a larger band falls back to binary64 for every survivor.
__device__ inline bool topk_before(double s, int64_t i, double s2, int64_t i2) {
    return i2 < 0 || (i >= 0 && (s > s2 || (s == s2 && i < i2)));
}

// The binary64 step of the top-kk rescore: the band members (member m at lane m % 32, slot
// m / 32), or after a spill every survivor, scored in the oracle's order, and the kk best
// by (score desc, index asc) written out.
__device__ __forceinline__ void topk_finish(const float *__restrict__ rows, const float *__restrict__ q, int64_t j,
                                            const int32_t *bk, int cnt, int kk, int lane, bool spill, int nm,
                                            int32_t m0, int32_t m1, int64_t *__restrict__ out_idx,
                                            double *__restrict__ out_sim, long long *__restrict__ counters) {
    const float *qj = q + j * kD;
    double prev_s = INFINITY;
    int64_t prev_i = -1;
    if (!spill) {
        double v0 = -INFINITY, v1 = -INFINITY;
        if (m0 >= 0) v0 = dot64_seq(qj, rows + (int64_t)m0 * kD);
        if (m1 >= 0) v1 = dot64_seq(qj, rows + (int64_t)m1 * kD);
        bool t0 = m0 < 0, t1 = m1 < 0;  // taken (or empty)
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_FP64), (unsigned long long)nm);
        for (int r = 0; r < kk; ++r) {
            double bs = -INFINITY;
            int64_t bi = -1;
            if (!t0) { bs = v0; bi = m0; }
            if (!t1 && topk_before(v1, m1, bs, bi)) { bs = v1; bi = m1; }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const double os = __shfl_xor_sync(0xffffffffu, bs, o);
                const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (topk_before(os, oi, bs, bi)) { bs = os; bi = oi; }
            }
            if (!t0 && bi == m0) t0 = true;
            else if (!t1 && bi == m1) t1 = true;
            if (lane == 0) {
                out_idx[j * kk + r] = bi;
                out_sim[j * kk + r] = bi >= 0 ? bs : -INFINITY;
            }
        }
    } else {
        // more than 64 band members: binary64 for every survivor, one rank per sweep
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_FP64), (unsigned long long)cnt * kk);
        for (int r = 0; r < kk; ++r) {
            double bs = -INFINITY;
            int64_t bi = -1;
            for (int t = lane; t < cnt; t += 32) {
                const int32_t id = bk[t];
                const double v = dot64_seq(qj, rows + (int64_t)id * kD);
                // eligible: after the previous rank in (score desc, index asc) order
                if (prev_i >= 0 && !topk_before(prev_s, prev_i, v, id)) continue;
                if (topk_before(v, id, bs, bi)) { bs = v; bi = id; }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const double os = __shfl_xor_sync(0xffffffffu, bs, o);
                const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (topk_before(os, oi, bs, bi)) { bs = os; bi = oi; }
            }
            prev_s = bs;
            prev_i = bi;
            if (lane == 0) {
                out_idx[j * kk + r] = bi;
                out_sim[j * kk + r] = bi >= 0 ? bs : -INFINITY;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_rescore_topk(const float *__restrict__ rows, const float *__restrict__ q,
                                                      int64_t nq, const int32_t *__restrict__ bucket,
                                                      const int32_t *__restrict__ count, int cap,
                                                      const float *__restrict__ qnorm, float xnorm_max, int kk,
                                                      int64_t *__restrict__ out_idx, double *__restrict__ out_sim,
                                                      int32_t *__restrict__ status, long long *__restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nq) return;
    const int cnt = count[j];
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_SURVIVORS), (unsigned long long)cnt);
        atomicMax(reinterpret_cast<unsigned long long *>(counters + CT_MAXSURV), (unsigned long long)cnt);
    }
    if (cnt > cap) {  // survivors were dropped: the host re-runs with more slots
        if (lane == 0) atomicExch(status + ST_OVERFLOW, 1);
        return;
    }
    const float4 qv = reinterpret_cast<const float4 *>(q + j * kD)[lane];
    const float eps = rescore_eps(qnorm[j], xnorm_max);
    const float band = __fmul_ru(2.f, eps);
    const int32_t *bk = bucket + j * (int64_t)cap;
    constexpr int U = 8;  // survivor rows in flight per warp
    // FP32 scores of survivors s0 .. s0+U-1 (warp-uniform after the butterfly)
    auto scores = [&](int s0, float (&part)[U], int32_t (&id)[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            id[u] = (s0 + u < cnt) ? bk[s0 + u] : -1;
            float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (id[u] >= 0) xv = reinterpret_cast<const float4 *>(rows + (int64_t)id[u] * kD)[lane];
            part[u] = fmaf(qv.x, xv.x, fmaf(qv.y, xv.y, fmaf(qv.z, xv.z, qv.w * xv.w)));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
#pragma unroll
            for (int u = 0; u < U; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], o);
    };
    // pass 1: the kk largest FP32 scores, descending over lanes 0 .. kk-1
    float top = -INFINITY;
    int filled = 0;
    for (int s0 = 0; s0 < cnt; s0 += U) {
        float part[U];
        int32_t id[U];
        scores(s0, part, id);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (id[u] < 0) continue;
            const float v = part[u];
            const float kth = __shfl_sync(0xffffffffu, top, kk - 1);
            if (filled < kk || v > kth) {
                const int p = __popc(__ballot_sync(0xffffffffu, lane < filled && top >= v));
                const float up = __shfl_up_sync(0xffffffffu, top, 1);
                if (lane > p && lane < kk) top = up;
                if (lane == p) top = v;
                filled = filled < kk ? filled + 1 : kk;
            }
        }
    }
    const float fk = filled >= kk ? __shfl_sync(0xffffffffu, top, kk - 1) : -INFINITY;
    const float lo = fk == -INFINITY ? -INFINITY : __fsub_rd(fk, band);
    // pass 2: band members, member m at lane m % 32, slot m / 32
    int32_t m0 = -1, m1 = -1;
    int nm = 0;
    bool spill = false;
    for (int s0 = 0; s0 < cnt; s0 += U) {
        float part[U];
        int32_t id[U];
        scores(s0, part, id);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (id[u] < 0 || part[u] < lo) continue;
            if (nm < 64) {
                if (lane == (nm & 31)) {
                    if (nm < 32) m0 = id[u]; else m1 = id[u];
                }
                ++nm;
            } else {
                spill = true;
            }
        }
    }
    topk_finish(rows, q, j, bk, cnt, kk, lane, spill, nm, m0, m1, out_idx, out_sim, counters);
}

// Exact top-kk with the FP16-row filter (the default): a survivor whose FP16-row bound stays
// below cut = max(T_q, RD(f - eps_r)), T_q the kk-th largest certified bound of the threshold
// candidates and f the kk-th largest FP32 score so far, has similarity below the kk-th largest
// similarity, so it is not in the answer.  Only the kept survivors are read in FP32; their
// scores go into the running top-kk (pass 1) and a per-warp cache of kTopkCache, from which
// pass 2 takes the band members (FP32 score >= f_k - 2 eps_r) without reading a row again.
// Every member of the exact top-kk is kept (its bound reaches its similarity >= the cut) and
// f_k <= the kk-th similarity + eps_r, so each of them is a band member, as in k_rescore_topk.
// A cache overflow makes pass 2 bound the survivors again against the final cut.
constexpr int kTopkCache = 128;

__global__ void __launch_bounds__(256) k_rescore_topk16(const float *__restrict__ rows,
                                                        const __half *__restrict__ rows16,
                                                        const float *__restrict__ q, int64_t nq,
                                                        const int32_t *__restrict__ bucket,
                                                        const int32_t *__restrict__ count, int cap,
                                                        const float *__restrict__ qnorm, float xnorm_max,
                                                        const float *__restrict__ tlow, int kk,
                                                        int64_t *__restrict__ out_idx, double *__restrict__ out_sim,
                                                        int32_t *__restrict__ status, long long *__restrict__ counters) {
    __shared__ float4 qsh[8][kD / 4];
    __shared__ int32_t cid[8][kTopkCache];
    __shared__ float csc[8][kTopkCache];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nq) return;
    const int cnt = count[j];
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_SURVIVORS), (unsigned long long)cnt);
        atomicMax(reinterpret_cast<unsigned long long *>(counters + CT_MAXSURV), (unsigned long long)cnt);
    }
    if (cnt > cap) {
        if (lane == 0) atomicExch(status + ST_OVERFLOW, 1);
        return;
    }
    const float4 qv = reinterpret_cast<const float4 *>(q + j * kD)[lane];
    qsh[wib][lane] = qv;
    __syncwarp();
    const float4 *qs = qsh[wib];
    const float eps = rescore_eps(qnorm[j], xnorm_max);
    const float e16 = rescore16_slack(qnorm[j], xnorm_max);
    const float band = __fmul_ru(2.f, eps);
    const int32_t *bk = bucket + j * (int64_t)cap;
    const float t0 = tlow[j];
    // the FP16-row bound of survivor s (one lane each)
    auto bound16 = [&](int s) {
        const uint4 *r = reinterpret_cast<const uint4 *>(rows16 + (int64_t)bk[s] * kD);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int i = 0; i < kD / 8; ++i) {
            const uint4 v = __ldg(r + i);
            const float4 qa = qs[2 * i], qb = qs[2 * i + 1];
            const float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
            const float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
            const float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&v.z));
            const float2 f3 = __half22float2(*reinterpret_cast<const __half2 *>(&v.w));
            a0 = fmaf(qa.x, f0.x, fmaf(qa.y, f0.y, a0));
            a1 = fmaf(qa.z, f1.x, fmaf(qa.w, f1.y, a1));
            a2 = fmaf(qb.x, f2.x, fmaf(qb.y, f2.y, a2));
            a3 = fmaf(qb.z, f3.x, fmaf(qb.w, f3.y, a3));
        }
        return __fadd_ru((a0 + a1) + (a2 + a3), e16);
    };
    // FP32 full score of the survivor whose id lane src holds (warp-cooperative row)
    auto full32 = [&](int32_t id) {
        const float4 xv = reinterpret_cast<const float4 *>(rows + (int64_t)id * kD)[lane];
        float v = fmaf(qv.x, xv.x, fmaf(qv.y, xv.y, fmaf(qv.z, xv.z, qv.w * xv.w)));
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    // pass 1: the kk largest FP32 scores of the kept survivors, descending over lanes 0 .. kk-1
    float top = -INFINITY;
    int filled = 0, ncache = 0;
    long long kept_total = 0;
    float cut = t0;
    for (int s0 = 0; s0 < cnt; s0 += 32) {
        const int s = s0 + lane;
        const int32_t my_id = s < cnt ? bk[s] : -1;
        const bool keep = my_id >= 0 && bound16(s) >= cut;
        unsigned mk = __ballot_sync(0xffffffffu, keep);
        kept_total += __popc(mk);
        while (mk) {
            const int src = __ffs(mk) - 1;
            mk &= mk - 1;
            const int32_t id = __shfl_sync(0xffffffffu, my_id, src);
            const float v = full32(id);
            if (ncache < kTopkCache && lane == 0) {
                cid[wib][ncache] = id;
                csc[wib][ncache] = v;
            }
            ++ncache;
            const float kth = __shfl_sync(0xffffffffu, top, kk - 1);
            if (filled < kk || v > kth) {
                const int p = __popc(__ballot_sync(0xffffffffu, lane < filled && top >= v));
                const float up = __shfl_up_sync(0xffffffffu, top, 1);
                if (lane > p && lane < kk) top = up;
                if (lane == p) top = v;
                filled = filled < kk ? filled + 1 : kk;
            }
        }
        if (filled >= kk) cut = fmaxf(cut, __fsub_rd(__shfl_sync(0xffffffffu, top, kk - 1), eps));
    }
    __syncwarp();
    const float fk = filled >= kk ? __shfl_sync(0xffffffffu, top, kk - 1) : -INFINITY;
    const float lo = fk == -INFINITY ? -INFINITY : __fsub_rd(fk, band);
    // pass 2: band members, member m at lane m % 32, slot m / 32
    int32_t m0 = -1, m1 = -1;
    int nm = 0;
    bool spill = false;
    auto add_member = [&](int32_t id) {
        if (nm < 64) {
            if (lane == (nm & 31)) {
                if (nm < 32) m0 = id; else m1 = id;
            }
            ++nm;
        } else {
            spill = true;
        }
    };
    if (ncache <= kTopkCache) {
        for (int c0 = 0; c0 < ncache; c0 += 32) {
            const int c = c0 + lane;
            const int32_t my_id = c < ncache ? cid[wib][c] : -1;
            unsigned mb = __ballot_sync(0xffffffffu, c < ncache && csc[wib][c] >= lo);
            while (mb) {
                const int src = __ffs(mb) - 1;
                mb &= mb - 1;
                add_member(__shfl_sync(0xffffffffu, my_id, src));
            }
        }
    } else {
        for (int s0 = 0; s0 < cnt; s0 += 32) {
            const int s = s0 + lane;
            const int32_t my_id = s < cnt ? bk[s] : -1;
            unsigned mk = __ballot_sync(0xffffffffu, my_id >= 0 && bound16(s) >= cut);
            while (mk) {
                const int src = __ffs(mk) - 1;
                mk &= mk - 1;
                const int32_t id = __shfl_sync(0xffffffffu, my_id, src);
                if (full32(id) >= lo) add_member(id);
            }
        }
    }
    if (lane == 0 && cnt > kept_total)
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + CT_SKIPPED), (unsigned long long)(cnt - kept_total));
    topk_finish(rows, q, j, bk, cnt, kk, lane, spill, nm, m0, m1, out_idx, out_sim, counters);
}

cudaError_t launch_rescore_topk(const Index &ix, const float *q, int64_t nq, int kk, int64_t *out_idx,
                                double *out_sim, cudaStream_t st, int mode) {
    const int64_t blocks = (nq * 32 + 255) / 256;
    if (mode == HN_RESCORE_FILTER16 && ix.rows16) {
        k_rescore_topk16<<<(unsigned)blocks, 256, 0, st>>>(ix.rows, ix.rows16, q, nq, ix.ws.bucket, ix.ws.count,
                                                           ix.ws.bucket_cap, ix.ws.qnorm, ix.host_max[4], ix.ws.tlow,
                                                           kk, out_idx, out_sim, ix.ws.status, ix.ws.counters);
        return cudaGetLastError();
    }
    k_rescore_topk<<<(unsigned)blocks, 256, 0, st>>>(ix.rows, q, nq, ix.ws.bucket, ix.ws.count, ix.ws.bucket_cap,
                                                     ix.ws.qnorm, ix.host_max[4], kk, out_idx, out_sim, ix.ws.status,
                                                     ix.ws.counters);
    return cudaGetLastError();
}

cudaError_t launch_rescore(const Index &ix, const float *q, int64_t nq, int64_t *out_idx, double *out_sim,
                           cudaStream_t st, int mode) {
    const int64_t blocks = (nq * 32 + 255) / 256;
    if (mode == HN_RESCORE_FILTER16 && ix.rows16) {
        k_rescore16<<<(unsigned)blocks, 256, 0, st>>>(ix.rows, ix.rows16, q, nq, ix.ws.bucket, ix.ws.count,
                                                      ix.ws.bucket_cap, ix.ws.qnorm, ix.host_max[4], ix.ws.tlow,
                                                      out_idx, out_sim, ix.ws.status, ix.ws.counters);
    } else if (mode == HN_RESCORE_BEST_FIRST)
        k_rescore_bf<<<(unsigned)blocks, 256, 0, st>>>(ix.rows, q, nq, ix.ws.bucket, ix.ws.count, ix.ws.bucket_cap,
                                                       ix.ws.qnorm, ix.host_max[4], ix.ws.qeps32, ix.ws.tlow, ix.k, out_idx,
                                                       out_sim, ix.ws.status, ix.ws.counters);
    else
        k_rescore<<<(unsigned)blocks, 256, 0, st>>>(ix.rows, q, nq, ix.ws.bucket, ix.ws.count, ix.ws.bucket_cap,
                                                    ix.ws.qnorm, ix.host_max[4], out_idx, out_sim, ix.ws.status,
                                                    ix.ws.counters);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ brute force
__global__ void k_brute_finish(const unsigned long long *__restrict__ key1, int64_t nq, int64_t *out_idx,
                               double *out_sim) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    out_idx[j] = (int64_t)best_idx(key1[j]);
    out_sim[j] = (double)best_score(key1[j]);
}

cudaError_t launch_bruteforce(const Index &ix, const float *q, int64_t nq, int64_t *out_idx, double *out_sim,
                              cudaStream_t st) {
    // rows are [n][128]; the last tile reads up to n_tiles*256 rows, so the
    // master copy is allocated with that padding (zeros).
    cudaError_t e = cudaMemsetAsync(ix.ws.key1, 0, sizeof(unsigned long long) * nq, st);
    if (e != cudaSuccess) return e;
    e = stream_scan_kt<128, FMT_F32>(ix.rows, nullptr, ix.n, ix.n_tiles, q, nq, 1, ix.ws, st);
    if (e != cudaSuccess) return e;
    k_brute_finish<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(ix.ws.key1, nq, out_idx, out_sim);
    return cudaGetLastError();
}

cudaError_t launch_bruteforce_keys(const Index &ix, const float *q, int64_t nq, unsigned long long *keys,
                                   int64_t *out_idx, double *out_sim, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * nq, st);
    if (e != cudaSuccess) return e;
    Workspace w = ix.ws;  // same scan, keys redirected to the caller's array
    w.key1 = keys;
    e = stream_scan_kt<128, FMT_F32>(ix.rows, nullptr, ix.n, ix.n_tiles, q, nq, 1, w, st);
    if (e != cudaSuccess) return e;
    k_brute_finish<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(keys, nq, out_idx, out_sim);
    return cudaGetLastError();
}

}  // namespace hn
