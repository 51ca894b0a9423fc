// Internal declarations shared by the CUDA translation units of libhn.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hn.h"

namespace hn {

constexpr int kD = 128;           // descriptor width (HardNet, §3.1)
constexpr int kTileE = 256;       // entries per scan tile (dense kernel N dimension)
constexpr int kTileQ = 128;       // queries per dense MMA (UMMA M)
constexpr int kQPad = 256;        // query padding: the dense scan takes queries 256 at a time

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
hn_status fail(hn_status st, const std::string &msg);
hn_status cuda_fail(cudaError_t e, const char *what);

#define HN_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::hn::cuda_fail(e_, #call);      \
    } while (0)

__host__ __device__ inline int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------- keys
// Order-preserving map of a binary32 value onto uint32: a < b  <=>  key(a) < key(b)
// for all non-NaN a, b (with -0 < +0).  Used for atomicMax across CTAs.
__host__ __device__ inline uint32_t f2key(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key2f(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    float f;
    memcpy(&f, &u, 4);
    return f;
}
// (score, index) packed so that a larger key means a larger score, then a lower index.
__host__ __device__ inline unsigned long long pack_best(float s, uint32_t idx) {
    return ((unsigned long long)f2key(s) << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
}
__host__ __device__ inline uint32_t best_idx(unsigned long long k) {
    return 0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull);
}
__host__ __device__ inline float best_score(unsigned long long k) { return key2f((uint32_t)(k >> 32)); }

// ---------------------------------------------------------------- index
struct Workspace {
    // per-query scratch, sized for `q_cap` queries and `bucket_cap` survivors each
    int64_t q_cap = 0;
    int32_t bucket_cap = 0;
    int32_t *bucket = nullptr;         // [q_cap][bucket_cap] survivor entry ids
    int32_t *count = nullptr;          // [q_cap] survivor counts (may exceed bucket_cap)
    unsigned long long *key1 = nullptr;// [q_cap] Phase-1 best (score, index) key (stream scan)
    unsigned long long *cand = nullptr;// [q_cap][cand_slots] Phase-1 per-chunk bests (dense scan)
    uint32_t *gbits = nullptr;         // dense scan group map: two-pass form, one bit per 32-entry group
                                       //   that reached tau_q; one-pass form, one 8-bit code of the group's
                                       //   largest score per 32-entry group
    int64_t gbits_cap = 0;             // allocated words of gbits
    int64_t gbits_limit = 0;           // words the current search may use (<= gbits_cap; 0 = all)
    uint64_t wait_ns = 0;              // main-loop wait limit of the dense scan for the current search (0 = 2 s)
    int32_t stall = 0;                 // failure-path test for the current search (hn_search_opts.test_stall)
    int32_t plain = 0;                 // the one-pass scan's unsplit form (hn_search_opts.test_plain_epilogue)
    int64_t cand_cap = 0;              // allocated length of cand
    int32_t cand_slots = 1;            // candidates per query written by the last Phase 1
    float *tau = nullptr;              // [q_cap] Phase-2 prefix threshold
    float *tlow = nullptr;             // [q_cap] T_q: certified lower bound on the best similarity
                                       //   (the best fully scored threshold candidate; -inf: none)
    float *qpre32 = nullptr;           // [q_cap][k_pad4] query prefix (FP32, or BF16 values)
    __nv_bfloat16 *qpre16 = nullptr;   // [q_cap rounded to 128][k_pad16] UMMA A tiles (FP8 index:
                                       //   the e4m3 hi/lo pairs of Phase 2, 2 * k_pad16 bytes a query)
    __half *qpre16h = nullptr;         // int8 index: read as float[q_cap], 1 / (t_q s) (hn_prep.cu);
                                       // qpre16 then holds k_pad16 int8 codes a query
    float *qeps = nullptr;             // [q_cap] per-query Phase-2 slack E_q (FP32, rounded up)
    float *qeps32 = nullptr;           // [q_cap] slack of the FP32 prefix score over the master rows
                                       //   (best-first rescore): gamma_K |q_maj| max|x_maj| + minor bound
    float *qnorm = nullptr;            // [q_cap] |q| rounded up
    int32_t *status = nullptr;         // [8] device status words
    long long *counters = nullptr;     // [8] device counters for stats
    int32_t *h_status = nullptr;       // pinned host mirror of status + counters
    int32_t last_max = 0;              // largest survivor count seen (sizing hint)
    cudaEvent_t ev[8] = {};            // step timers (created on first timed search)
    bool ev_ready = false;
    uint64_t gen = 0;                  // bumped whenever the buffers above are reallocated
};

struct Index {
    int64_t n = 0;
    int32_t d = kD, k = 0;
    double alpha = 0;
    int32_t prefix = HN_PREFIX_F32;
    int32_t k_pad4 = 0;    // FP32 prefix row width
    int32_t k_pad16 = 0;   // BF16 prefix width (multiple of 16, UMMA K step)
    int64_t n_tiles = 0;   // ceil(n / kTileE)
    float *rows = nullptr;           // [n][128] FP32 master copy (full rescore)
    __half *rows16 = nullptr;        // [n_pad][128] the rows rounded to FP16 (the rescore's bound)
    float *pre32 = nullptr;          // [n][k_pad4] FP32 prefix (HN_PREFIX_F32)
    __nv_bfloat16 *pre16 = nullptr;  // [n_tiles*256][k_pad16] BF16 prefix, UMMA core-matrix order
    uint8_t *pre8 = nullptr;         // HN_PREFIX_FP8_E4M3: [n_tiles * 2] tiles of kF8TileBytes(k_pad16)
    int8_t *prei8 = nullptr;         // HN_PREFIX_I8: [n_tiles * 256][k_pad16] int8 codes, row-major
    float qt = 0.f;                  // FP8: |q~_major| bound the per-entry error terms assume
    float *mx = nullptr;             // [n] |x_minor| rounded up
    float *dev_max = nullptr;        // [8] maxima (rounded up): |x_minor|, |x_major|, residual, |prefix|, |x|,
                                     //     max |x_major component| (int8 index: sets the code scale)
    float host_max[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // see dev_max
    uint64_t serial = 0;             // unique per built index (a freed index's address may be reused)
    int32_t dense_min_q = 1024;      // smallest batch the AUTO scan sends to the dense kernel (autotuned)
    int32_t units_per_cta = 256;     // dense work-unit granularity (autotuned); more, shorter entry
                                     // chunks give the threshold more candidate regions and the
                                     // extraction more blocks
    float code_inv = 1.f;            // one-pass dense scan: inv of the group code (127 / bound on |score|)
    int32_t n_blocks = 0;            // block partition for the learned proposal (0 = none)
    int32_t *block_ids = nullptr;    // [n] entry ids in block order
    int32_t *block_of = nullptr;     // [n] block of each entry
    int32_t *block_start = nullptr;  // [n_blocks + 1]
    int64_t bytes = 0;
    Workspace ws;
};

// status word slots
enum { ST_NOT_NORMALIZED = 0, ST_ZERO_NORM = 1, ST_OVERFLOW = 2, ST_TIMEOUT = 3, ST_BAD_ROW = 4 };
// counter slots
enum { CT_SURVIVORS = 0, CT_MAXSURV = 1, CT_FP64 = 2, CT_GROUPS = 3, CT_SKIPPED = 4 };

// byte offset of (entry e, prefix column c) in the BF16 UMMA-ordered prefix:
// groups of 8 entries; inside a group, 16-byte core-matrix rows per 8 columns.
__host__ __device__ inline int64_t pre16_offset(int64_t e, int c, int k_pad16) {
    const int64_t g = e >> 3;
    const int r = (int)(e & 7);
    return g * (int64_t)k_pad16 * 16 + (int64_t)(c >> 3) * 128 + r * 16 + (c & 7) * 2;
}

// ---------------------------------------------------------------- FP8 prefix
// An FP8 index stores the major prefix as e4m3 with a per-entry power-of-two scale
// s_i (dequantisation x~ = s_i * x^ is exact), in 128-entry tiles:
//   [128 x kp e4m3 values, UMMA core-matrix order: 8-entry groups of kp/16 core
//    matrices of 8 rows x 16 bytes]
//   [128 x float  s_i / kF8QScale]      (scale of the Phase-2 tensor-core product)
//   [128 x float  b_i = RU(qt * r_i)]   (r_i = |x_i,major - x~_i|: per-entry error term)
//   [4 x float4 (max_i s_i / kF8QScale, min_i s_i / kF8QScale, max_i b_i, 0)] over the
//    real entries (i < n) of each 32-entry group: the one-pass scan bounds a group's
//    largest score from its largest raw accumulator with them (zeros for a group
//    holding padding rows only)
constexpr int kF8Tile = 128;
constexpr float kF8QScale = 256.f;   // query prefix scale of the tensor-core product (hi + lo e4m3 parts)
__host__ __device__ constexpr int64_t kF8TileBytes(int kp) { return (int64_t)kF8Tile * (kp + 8) + 64; }
__host__ __device__ inline int64_t f8_scale_off(int kp) { return (int64_t)kF8Tile * kp; }
__host__ __device__ inline int64_t f8_group_off(int kp) { return (int64_t)kF8Tile * (kp + 8); }
// byte offset of (row r, byte column c) in a K-major UMMA tile whose rows hold `row_bytes` bytes
__host__ __device__ inline int64_t umma8_offset(int64_t r, int c, int row_bytes) {
    return (r >> 3) * (int64_t)row_bytes * 8 + (int64_t)(c >> 4) * 128 + (r & 7) * 16 + (c & 15);
}

// ---------------------------------------------------------------- group-map codes
// One-pass dense scan: the largest score g of every 32-entry group is kept as an
// 8-bit code, and the survivor extraction, once tau_q is known, looks only at the
// groups with code(g) >= code(tau_q).  Any non-decreasing code is exact for that
// test (g >= tau  =>  code(g) >= code(tau)); this one is
//   code(v) = clamp(RU(v * inv + base) - 2^23, 0, 255)
// with inv = 127 / B and base = 2^23 + 128 (B bounds |g| for unit HN prefixes, so
// scores map to 1..255 with a step of about B / 127).  The value RU(.) lies in
// [2^23, 2^24) where binary32 steps by 1, so its bits minus those of 2^23 are the
// integer code.  The scan side takes the cheaper clamp code_group: a score below
// the range wraps round to 255 instead of 0, which can only flag more groups.
constexpr uint32_t kCodeBits0 = 0x4B000000u;  // bits of 2^23
__host__ __device__ inline float code_base() { return 8388608.f + 128.f; }
// The scan's code of a group score, returned in the low byte of a binary32 bit pattern:
// RU(g * inv + base) clamped from above to 2^23 + 255.  Inside [2^23, 2^23 + 255] the low
// byte is the code.  A score below the range leaves a value under 2^23 whose low byte is
// arbitrary: harmless, because such a group matters only for a threshold below the range
// too, whose code is 0, which every byte reaches.
__device__ __forceinline__ uint32_t code_group_bits(float g, float inv, float base) {
    return __float_as_uint(fminf(__fmaf_ru(g, inv, base), 8388608.f + 255.f));
}
__device__ __forceinline__ uint32_t code_threshold(float tau, float inv, float base) {
    const float v = fminf(fmaxf(__fmaf_ru(tau, inv, base), 8388608.f), 8388608.f + 255.f);
    return __float_as_uint(v) - kCodeBits0;
}

// search pipeline pieces (hn_api.cu), shared with the multi-batch path
int pick_scan(const Index &ix, int64_t nq, int requested);
// nn: neighbours per query (1: the 1-NN; 2..32: exact top-nn, outputs [nq][nn])
// seeded: the proposal gives the threshold (a dense Phase 2 then takes the two-pass bit scan);
// scratch_limit: bytes of the dense group map this search may use (0 = the default cap)
hn_status prepare_search(Index &ix, int64_t nq, int scan, int32_t cap, int nn = 1, bool seeded = false,
                         int64_t scratch_limit = 0);
hn_status enqueue_search(Index &ix, const float *q, int64_t nq, int scan, const hn_proposal *seed, int topk,
                         int64_t *out_idx, double *out_sim, bool timing, cudaStream_t s, int nn = 1,
                         float minor_scale = 1.f, int rescore = HN_RESCORE_FILTER16);
hn_status check_search(Index &ix, int64_t nq, int32_t *want_cap);
int32_t default_cap(const Index &ix);
Index *index_state_mut(hn_index *h);

// launches (defined in the .cu files)
cudaError_t launch_normalize(const float *in, float *out, int64_t n, int k, double alpha,
                             int32_t *status, cudaStream_t s);
cudaError_t launch_check_hn(const float *x, int64_t n, int k, double alpha, int32_t *status,
                            cudaStream_t s);
cudaError_t launch_pack(Index &ix, const float *x, cudaStream_t s);
// minor_scale: 1 for the exact search; beta / alpha in the soft ANN mode
cudaError_t launch_query_prep(const Index &ix, const float *q, int64_t nq, float minor_scale, cudaStream_t s);
// cand != NULL (Phase 1): one best entry per entry range into cand[q][stream_cand_slots], else key1
cudaError_t launch_stream_scan(const Index &ix, int64_t nq, int phase, cudaStream_t s,
                               unsigned long long *cand = nullptr);
int64_t stream_cand_slots(const Index &ix, int64_t nq);
cudaError_t launch_dense_scan(const Index &ix, int64_t nq, int phase, cudaStream_t s);
// kk: the threshold certifies the kk-th best similarity (1 for the 1-NN)
// keep_best (soft ANN mode): the best scored candidate is put into survivor slot 0
cudaError_t launch_seed_threshold(const Index &ix, const float *q, int64_t nq, bool dense, int kk, bool keep_best,
                                  cudaStream_t s);
// The same for queries q0 .. q0 + nq - 1 of the batch, from S candidate keys per query naming
// seg_entries-entry segments (cand laid out [query][S] from query 0 of the batch).
cudaError_t launch_seed_threshold_at(const Index &ix, const float *q, int64_t q0, int64_t nq, int S, int seg_entries,
                                     int kk, bool keep_best, cudaStream_t s);
// One-pass dense search steps (scan, threshold, extraction per pass; hn_dense.cu)
cudaError_t launch_dense_onepass(const Index &ix, const float *q, int64_t nq, int kk, bool keep_best, cudaStream_t s,
                                 cudaEvent_t *ev);
// Verification: [nq][n] prefix scores of the prepared queries; path 0 tensor cores, 1 CUDA-core FMA chain
cudaError_t launch_prefix_scores(const Index &ix, int64_t nq, int path, float *out, cudaStream_t s);
// Exact top-kk of every query from its Phase-2 survivors (1 <= kk <= 32): out_idx/out_sim [nq][kk].
cudaError_t launch_rescore_topk(const Index &ix, const float *q, int64_t nq, int kk, int64_t *out_idx,
                                double *out_sim, cudaStream_t s, int mode = HN_RESCORE_FILTER16);
// mode (hn_rescore): the FP16-row filter (default), the best-first prefix bound (f4), or every
// survivor in FP32
cudaError_t launch_rescore(const Index &ix, const float *q, int64_t nq, int64_t *out_idx,
                           double *out_sim, cudaStream_t s, int mode = HN_RESCORE_FILTER16);
cudaError_t launch_bruteforce(const Index &ix, const float *q, int64_t nq, int64_t *out_idx,
                              double *out_sim, cudaStream_t s);
// Brute force with a caller-provided per-query key array (nq entries, cleared here).
cudaError_t launch_bruteforce_keys(const Index &ix, const float *q, int64_t nq, unsigned long long *keys,
                                   int64_t *out_idx, double *out_sim, cudaStream_t s);
// Device state of a built index (used by entry points outside hn_api.cu).
const Index *index_state(const hn_index *h);
bool dense_scan_supported(const Index &ix);
cudaError_t dense_init();
cudaError_t build_blocks(Index &ix, int n_blocks, int iters, cudaStream_t s);
cudaError_t launch_seed_blocks(const Index &ix, const float *q, int64_t nq, const int32_t *blocks, int topk,
                               bool keep_best, cudaStream_t s);
// proposal helpers (hn_mlp.cu)
// status: device word set to 1 if an inference layer's bounded wait gave up (may be NULL)
cudaError_t proposal_topk(hn_proposal *p, const float *q, int64_t nq, int topk, int32_t *out, int32_t *status,
                          cudaStream_t s);
// One fully connected layer on the tensor cores (BF16 operands, FP32 accumulation):
// out[r][j] = act(sum_k in[r][k] w[j][k] + b[j]), act 0 none / 1 gelu; row-major FP32 operands.
cudaError_t linear_bf16(int M, int N, int K, const float *in, int64_t ldi, const float *w, int64_t ldw,
                        const float *bias, int act, float *out, int64_t ldo, int32_t *status, cudaStream_t st);
cudaError_t proposal_scratch(hn_proposal *p, int64_t n, int32_t **out);
int32_t proposal_blocks(const hn_proposal *p);
int32_t proposal_k(const hn_proposal *p);
int64_t dense_cand_slots(const Index &ix, int64_t nq);
int64_t dense_phase1_slots(const Index &ix, int64_t nq);
// uint32 words of the dense group map the workspace holds for nq queries (onepass: codes, else
// the two-pass Phase-2 bits), at most limit_bytes when > 0, at least one query tile's
int64_t dense_gbits_words(const Index &ix, int64_t nq, bool onepass, int64_t limit_bytes);
// kernel launches of the dense steps after Phase 1 / the threshold (see hn_dense.cu)
int64_t dense_phase2_launches(const Index &ix, int64_t nq, bool onepass);
// Batched serving: one persistent one-pass dense scan over several (index, queries) groups
// that share the tile format (hn_dense.cu).  Create after prepare_search has sized every
// group's scratch; the scan needs every group's query prep done, and dense_multi_post then
// gives each group its threshold and survivors.
struct DenseMulti;
bool dense_multi_joinable(const Index &ix, int64_t nq, int kp, bool f8);
hn_status dense_multi_create(const std::vector<const Index *> &ixs, const std::vector<int64_t> &nqs, DenseMulti **out);
void dense_multi_destroy(DenseMulti *m);
cudaError_t dense_multi_scan(const DenseMulti *m, cudaStream_t s);
cudaError_t dense_multi_post(const DenseMulti *m, int gi, const float *q, cudaStream_t s);

}  // namespace hn
