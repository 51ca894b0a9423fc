// C-ABI entry points of libhn (declared in include/hn.h).
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>

#include <cmath>

#include "hn_internal.cuh"

namespace hn {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }
hn_status fail(hn_status st, const std::string &msg) {
    g_err = msg;
    return st;
}
hn_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? HN_ERR_OOM : HN_ERR_CUDA;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static int next_width(int k, int lo) {
    int w = lo;
    while (w < k) w *= 2;
    return w;
}

template <class T>
static cudaError_t dalloc(T **p, size_t count) {
    return cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(T));
}

static void free_ws(Workspace &ws) {
    cudaFree(ws.bucket);
    cudaFree(ws.count);
    cudaFree(ws.key1);
    cudaFree(ws.cand);
    ws.cand = nullptr;
    ws.cand_cap = 0;
    cudaFree(ws.gbits);
    ws.gbits = nullptr;
    ws.gbits_cap = 0;
    cudaFree(ws.tau);
    cudaFree(ws.tlow);
    ws.tlow = nullptr;
    cudaFree(ws.qpre32);
    cudaFree(ws.qpre16);
    cudaFree(ws.qpre16h);
    ws.qpre16h = nullptr;
    cudaFree(ws.qeps);
    cudaFree(ws.qeps32);
    ws.qeps32 = nullptr;
    cudaFree(ws.qnorm);
    ws.bucket = nullptr;
    ws.count = nullptr;
    ws.key1 = nullptr;
    ws.tau = nullptr;
    ws.qpre32 = nullptr;
    ws.qpre16 = nullptr;
    ws.qeps = nullptr;
    ws.qnorm = nullptr;
    ws.q_cap = 0;
    ws.bucket_cap = 0;
}

static void free_index(Index *ix) {
    if (!ix) return;
    free_ws(ix->ws);
    if (ix->ws.ev_ready)
        for (cudaEvent_t e : ix->ws.ev) cudaEventDestroy(e);
    cudaFree(ix->ws.status);
    cudaFree(ix->ws.counters);
    cudaFreeHost(ix->ws.h_status);
    cudaFree(ix->rows);
    cudaFree(ix->rows16);
    cudaFree(ix->pre32);
    cudaFree(ix->pre16);
    cudaFree(ix->pre8);
    cudaFree(ix->prei8);
    cudaFree(ix->mx);
    cudaFree(ix->dev_max);
    cudaFree(ix->block_ids);
    cudaFree(ix->block_of);
    cudaFree(ix->block_start);
    delete ix;
}

// Make the per-query scratch hold nq queries and `cap` survivor slots each.
static hn_status ensure_ws(Index &ix, int64_t nq, int32_t cap) {
    Workspace &ws = ix.ws;
    const int64_t nq_pad = (nq + kQPad - 1) / kQPad * kQPad;
    if (nq_pad <= ws.q_cap && cap <= ws.bucket_cap) return HN_OK;
    const int64_t qc = std::max(nq_pad, ws.q_cap);
    const int32_t bc = std::max(cap, ws.bucket_cap);
    free_ws(ws);
    HN_CUDA(dalloc(&ws.bucket, (size_t)qc * bc));
    HN_CUDA(dalloc(&ws.count, qc));
    HN_CUDA(dalloc(&ws.key1, qc));
    HN_CUDA(dalloc(&ws.tau, qc));
    HN_CUDA(dalloc(&ws.tlow, qc));
    HN_CUDA(dalloc(&ws.qpre32, (size_t)qc * ix.k_pad4));
    HN_CUDA(dalloc(&ws.qpre16, (size_t)qc * ix.k_pad16));
    HN_CUDA(dalloc(&ws.qpre16h, (size_t)qc * ix.k_pad16));
    HN_CUDA(dalloc(&ws.qeps, qc));
    HN_CUDA(dalloc(&ws.qeps32, qc));
    HN_CUDA(dalloc(&ws.qnorm, qc));
    ws.q_cap = qc;
    ws.bucket_cap = bc;
    ++ws.gen;
    return HN_OK;
}

static hn_status check_dims(int32_t d, int32_t k, double alpha, bool for_index) {
    if (d != kD) return fail(HN_ERR_UNSUPPORTED, "d must be 128");
    if (k < 1 || k >= d) return fail(HN_ERR_INVALID_ARG, "need 1 <= k < d");
    if (for_index && k > 64) return fail(HN_ERR_UNSUPPORTED, "an index needs k <= 64");
    if (!(alpha >= 0.0 && alpha < 1.0)) return fail(HN_ERR_INVALID_ARG, "need 0 <= alpha < 1");
    return HN_OK;
}

}  // namespace hn

using namespace hn;

struct hn_index {
    Index ix;
};

const Index *hn::index_state(const hn_index *h) { return h ? &h->ix : nullptr; }
Index *hn::index_state_mut(hn_index *h) { return h ? &h->ix : nullptr; }

extern "C" {

int32_t hn_version(void) { return (0 << 16) | 1; }

const char *hn_last_error(void) { return g_err.c_str(); }

hn_status hn_normalize(const float *in, float *out, int64_t n, int32_t d, int32_t k, double alpha, void *stream) {
    hn_status st = check_dims(d, k, alpha, false);
    if (st != HN_OK) return st;
    if (n < 0) return fail(HN_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return HN_OK;
    if (!in || !out || !aligned16(in) || !aligned16(out)) return fail(HN_ERR_INVALID_ARG, "null or unaligned pointer");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *dstat = nullptr;
    HN_CUDA(cudaMallocAsync((void **)&dstat, 8 * sizeof(int32_t), s));
    int32_t h[8];
    cudaError_t e = cudaMemsetAsync(dstat, 0, 8 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_normalize(in, out, n, k, alpha, dstat, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, dstat, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dstat, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "hn_normalize");
    if (h[ST_NOT_NORMALIZED]) return fail(HN_ERR_INVALID_ARG, "non-finite input row");
    if (h[ST_ZERO_NORM]) return fail(HN_ERR_ZERO_NORM, "zero major (or minor) norm");
    return HN_OK;
}

hn_status hn_normalize_async(const float *in, float *out, int64_t n, int32_t d, int32_t k, double alpha,
                             int32_t *status, void *stream) {
    hn_status st = check_dims(d, k, alpha, false);
    if (st != HN_OK) return st;
    if (n < 0) return fail(HN_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return HN_OK;
    if (!in || !out || !aligned16(in) || !aligned16(out)) return fail(HN_ERR_INVALID_ARG, "null or unaligned pointer");
    if (status && ((uintptr_t)status & 3u)) return fail(HN_ERR_INVALID_ARG, "unaligned status");
    static_assert(ST_NOT_NORMALIZED == 0 && ST_ZERO_NORM == 1, "status[0], status[1] of hn_normalize_async");
    const cudaError_t e = launch_normalize(in, out, n, k, alpha, status, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "hn_normalize_async");
    return HN_OK;
}

hn_status hn_index_build(const float *x, int64_t n, int32_t d, int32_t k, double alpha, const hn_index_opts *opts,
                         hn_index **out, void *stream) {
    if (!out) return fail(HN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    hn_status st = check_dims(d, k, alpha, true);
    if (st != HN_OK) return st;
    if (n < 1 || n > 0x7FFFFFFFll - kTileE) return fail(HN_ERR_INVALID_ARG, "need 1 <= n < 2^31 - 256");
    if (!x || !aligned16(x)) return fail(HN_ERR_INVALID_ARG, "null or unaligned x");
    hn_index_opts o{};
    if (opts) o = *opts;
    if (o.prefix != HN_PREFIX_F32 && o.prefix != HN_PREFIX_BF16 && o.prefix != HN_PREFIX_FP8_E4M3 &&
        o.prefix != HN_PREFIX_I8)
        return fail(HN_ERR_INVALID_ARG, "bad prefix type");
    for (int i = 0; i < 4; ++i)
        if (o.reserved[i]) return fail(HN_ERR_INVALID_ARG, "reserved option fields must be zero");
    if (o.n_blocks < 0 || o.n_blocks > n || o.n_blocks > (1 << 20))
        return fail(HN_ERR_INVALID_ARG, "need 0 <= n_blocks <= min(n, 2^20)");
    if (o.kmeans_iters < 0 || o.kmeans_iters > 1000) return fail(HN_ERR_INVALID_ARG, "need 0 <= kmeans_iters <= 1000");
    cudaStream_t s = (cudaStream_t)stream;
    hn_index *h = new hn_index();
    Index &ix = h->ix;
    static std::atomic<uint64_t> next_serial{1};
    ix.serial = next_serial++;
    ix.n = n;
    ix.k = k;
    ix.alpha = alpha;
    ix.prefix = o.prefix;
    ix.k_pad16 = next_width(k, 16);
    ix.k_pad4 = ix.prefix == HN_PREFIX_F32 ? next_width(k, 8) : ix.k_pad16;
    // FP8: |q~_major| of an HN query is sqrt(1 - alpha) up to rounding; the per-entry
    // error terms assume this bound (with margin) and the query slack covers any excess
    ix.qt = std::nextafter((float)(std::sqrt(1.0 - alpha) * (1.0 + 1.0 / 64)), INFINITY);
    ix.n_tiles = (n + kTileE - 1) / kTileE;
    const int64_t n_pad = ix.n_tiles * kTileE;
    cudaError_t e = cudaSuccess;
#define TRY(call)                       \
    do {                                \
        e = (call);                     \
        if (e != cudaSuccess) {         \
            hn_index_destroy(h);        \
            return cuda_fail(e, #call); \
        }                               \
    } while (0)
    TRY(dalloc(&ix.rows, (size_t)n_pad * kD));
    TRY(cudaMemsetAsync(ix.rows + n * kD, 0, (size_t)(n_pad - n) * kD * sizeof(float), s));
    TRY(dalloc(&ix.rows16, (size_t)n_pad * kD));
    if (ix.prefix == HN_PREFIX_F32) {
        TRY(dalloc(&ix.pre32, (size_t)n_pad * ix.k_pad4));
    } else if (ix.prefix == HN_PREFIX_FP8_E4M3) {
        TRY(dalloc(&ix.pre8, (size_t)(n_pad / kF8Tile) * kF8TileBytes(ix.k_pad16)));
    } else if (ix.prefix == HN_PREFIX_I8) {
        TRY(dalloc(&ix.prei8, (size_t)n_pad * ix.k_pad16));
    } else {
        TRY(dalloc(&ix.pre16, (size_t)n_pad * ix.k_pad16));
    }
    TRY(dalloc(&ix.mx, n));
    TRY(dalloc(&ix.dev_max, 8));
    TRY(dalloc(&ix.ws.status, 8));
    TRY(dalloc(&ix.ws.counters, 8));
    TRY(cudaMallocHost((void **)&ix.ws.h_status, 8 * sizeof(int32_t) + 8 * sizeof(long long)));
    TRY(cudaMemsetAsync(ix.dev_max, 0, 8 * sizeof(float), s));
    TRY(cudaMemsetAsync(ix.ws.status, 0, 8 * sizeof(int32_t), s));
    TRY(cudaMemsetAsync(ix.ws.status + ST_BAD_ROW, 0x7F, sizeof(int32_t), s));
    TRY(launch_pack(ix, x, s));
    int32_t hs[8];
    TRY(cudaMemcpyAsync(hs, ix.ws.status, sizeof(hs), cudaMemcpyDeviceToHost, s));
    TRY(cudaMemcpyAsync(ix.host_max, ix.dev_max, sizeof(ix.host_max), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
#undef TRY
    {
        // one-pass dense scan: group scores lie within about |q^| max|x^| (+ the FP8 error
        // term); the code maps [-B, B] onto 1..255 (any scale is exact, B sets the step)
        const double b = 1.05 * (std::sqrt(1.0 - alpha) * ix.host_max[3] + (double)ix.qt * ix.host_max[2]);
        ix.code_inv = b > 0 ? (float)(127.0 / b) : 1.f;
    }
    ix.bytes = (int64_t)n_pad * kD * (4 + 2) + (ix.pre32 ? n_pad * ix.k_pad4 * 4 : 0) +
               (ix.pre16 ? n_pad * ix.k_pad16 * 2 : 0) +
               (ix.pre8 ? (n_pad / kF8Tile) * kF8TileBytes(ix.k_pad16) : 0) +
               (ix.prei8 ? n_pad * ix.k_pad16 : 0) + n * 4;
    if (hs[ST_NOT_NORMALIZED]) {
        const int row = hs[ST_BAD_ROW];
        hn_index_destroy(h);
        return fail(HN_ERR_NOT_NORMALIZED, "entry " + std::to_string(row) + " violates the HN norm identities");
    }
    if (o.n_blocks > 0) {
        e = build_blocks(ix, o.n_blocks, o.kmeans_iters ? o.kmeans_iters : 8, s);
        if (e != cudaSuccess) {
            hn_index_destroy(h);
            return cuda_fail(e, "block partition");
        }
        ix.bytes += (int64_t)(2 * n + o.n_blocks + 1) * 4;
    }
    *out = h;
    return HN_OK;
}

hn_status hn_index_destroy(hn_index *index) {
    if (!index) return HN_OK;
    Index *ix = new Index(std::move(index->ix));
    delete index;
    free_index(ix);
    return HN_OK;
}

hn_status hn_index_get_info(const hn_index *index, hn_index_info *info) {
    if (!index || !info) return fail(HN_ERR_INVALID_ARG, "NULL argument");
    const Index &ix = index->ix;
    info->n = ix.n;
    info->d = ix.d;
    info->k = ix.k;
    info->alpha = ix.alpha;
    info->prefix = ix.prefix;
    info->k_pad = ix.prefix == HN_PREFIX_F32 ? ix.k_pad4 : ix.k_pad16;
    info->device_bytes = ix.bytes;
    info->minor_norm_max = ix.host_max[0];
    info->major_norm_max = ix.host_max[1];
    info->resid_norm_max = ix.host_max[2];
    info->prefix_norm_max = ix.host_max[3];
    info->n_blocks = ix.n_blocks;
    info->reserved = 0;
    return HN_OK;
}

hn_status hn_index_blocks(const hn_index *index, int32_t *block_start, int32_t *block_ids, int32_t *block_of,
                          void *stream) {
    if (!index) return fail(HN_ERR_INVALID_ARG, "index is NULL");
    const Index &ix = index->ix;
    if (ix.n_blocks <= 0) return fail(HN_ERR_INVALID_ARG, "the index has no block partition");
    cudaStream_t s = (cudaStream_t)stream;
    if (block_start)
        HN_CUDA(cudaMemcpyAsync(block_start, ix.block_start, sizeof(int32_t) * (ix.n_blocks + 1),
                                cudaMemcpyDeviceToDevice, s));
    if (block_ids) HN_CUDA(cudaMemcpyAsync(block_ids, ix.block_ids, sizeof(int32_t) * ix.n, cudaMemcpyDeviceToDevice, s));
    if (block_of) HN_CUDA(cudaMemcpyAsync(block_of, ix.block_of, sizeof(int32_t) * ix.n, cudaMemcpyDeviceToDevice, s));
    return HN_OK;
}

// One run of the search pipeline (Algorithm 1 on the GPU); 5 kernel launches.
// With `timing`, events ev[0..5] bracket the steps on stream s.
// With a proposal (`seed`), its top blocks give the threshold and Phase 1 is skipped.
static hn_status run_search(Index &ix, const float *q, int64_t nq, int scan, const hn_proposal *seed, int topk,
                            int64_t *out_idx, double *out_sim, bool timing, cudaStream_t s, int nn,
                            float minor_scale, int rescore) {
    Workspace &ws = ix.ws;
    auto mark = [&](int i) { return timing ? cudaEventRecord(ws.ev[i], s) : cudaSuccess; };
    HN_CUDA(cudaMemsetAsync(ws.key1, 0, sizeof(unsigned long long) * nq, s));
    HN_CUDA(mark(0));
    HN_CUDA(launch_query_prep(ix, q, nq, minor_scale, s));
    HN_CUDA(mark(1));
    if (seed) {
        int32_t *blocks = nullptr;
        hn_proposal *sp = const_cast<hn_proposal *>(seed);
        HN_CUDA(proposal_scratch(sp, nq * topk, &blocks));
        HN_CUDA(proposal_topk(sp, q, nq, topk, blocks, ws.status + ST_TIMEOUT, s));
        HN_CUDA(mark(2));
        HN_CUDA(launch_seed_blocks(ix, q, nq, blocks, topk, minor_scale < 1.f, s));
    } else if (scan == HN_SCAN_DENSE) {
        // one pass: the prefix product once, then the threshold and the survivors from the
        // group codes (ev[2], ev[3], ev[4] mark the scan, threshold and extraction)
        HN_CUDA(launch_dense_onepass(ix, q, nq, nn, minor_scale < 1.f, s, timing ? &ws.ev[2] : nullptr));
    } else {
        HN_CUDA(scan == HN_SCAN_DENSE_TWO_PASS ? launch_dense_scan(ix, nq, 1, s)
                                               : launch_stream_scan(ix, nq, 1, s, nn > 1 ? ws.cand : nullptr));
        HN_CUDA(mark(2));
        HN_CUDA(launch_seed_threshold(ix, q, nq, scan == HN_SCAN_DENSE_TWO_PASS, nn, minor_scale < 1.f, s));
    }
    if (seed || scan != HN_SCAN_DENSE) {
        // seeded: the proposal replaces Phase 1, and a dense Phase 2 takes the two-pass form's
        // bit scan against the known threshold
        HN_CUDA(mark(3));
        HN_CUDA(scan != HN_SCAN_STREAM ? launch_dense_scan(ix, nq, 2, s) : launch_stream_scan(ix, nq, 2, s));
        HN_CUDA(mark(4));
    }
    HN_CUDA(nn > 1 ? launch_rescore_topk(ix, q, nq, nn, out_idx, out_sim, s, rescore)
                   : launch_rescore(ix, q, nq, out_idx, out_sim, s, rescore));
    HN_CUDA(mark(5));
    return HN_OK;
}

}  // extern "C"

namespace hn {

int pick_scan(const Index &ix, int64_t nq, int requested) {
    if (requested != HN_SCAN_AUTO) return requested;
    return (dense_scan_supported(ix) && nq >= ix.dense_min_q) ? HN_SCAN_DENSE : HN_SCAN_STREAM;  // one-pass dense
}

// Size the index's scratch for nq queries and `cap` survivor slots (may allocate).
hn_status prepare_search(Index &ix, int64_t nq, int scan, int32_t cap, int nn, bool seeded, int64_t scratch_limit) {
    Workspace &ws = ix.ws;
    hn_status st = ensure_ws(ix, nq, cap);
    if (st != HN_OK) return st;
    const bool dense = scan == HN_SCAN_DENSE || scan == HN_SCAN_DENSE_TWO_PASS;
    if (dense || nn > 1) {
        // candidate keys: dense segments, or one entry per stream-scan entry range (top-k)
        const int64_t slots = dense ? dense_cand_slots(ix, nq) : stream_cand_slots(ix, nq);
        const int64_t need = ((nq + kQPad - 1) / kQPad * kQPad) * slots;
        if (need > ws.cand_cap) {
            cudaFree(ws.cand);
            ws.cand = nullptr;
            ws.cand_cap = 0;
            HN_CUDA(dalloc(&ws.cand, need));
            ws.cand_cap = need;
            ++ws.gen;
        }
        ws.cand_slots = (int32_t)slots;
    }
    if (dense) {
        // the one-pass form's code map, or the two-pass form's bitmap (seeded searches take the
        // latter), within the search's scratch limit; ws.gbits_limit keeps that limit for the launch
        const bool onepass = scan == HN_SCAN_DENSE && !seeded;
        const int64_t need = dense_gbits_words(ix, nq, onepass, scratch_limit);
        ws.gbits_limit = scratch_limit > 0 ? need : 0;
        if (need > ws.gbits_cap) {
            cudaFree(ws.gbits);
            ws.gbits = nullptr;
            ws.gbits_cap = 0;
            HN_CUDA(dalloc(&ws.gbits, need));
            ws.gbits_cap = need;
            ++ws.gen;
        }
    }
    return HN_OK;
}

// Enqueue one search on stream s: allocation-free, synchronisation-free, so it can
// be captured into a CUDA graph.  Status words and counters land in the pinned
// host mirror ws.h_status once the stream has run.
hn_status enqueue_search(Index &ix, const float *q, int64_t nq, int scan, const hn_proposal *seed, int topk,
                         int64_t *out_idx, double *out_sim, bool timing, cudaStream_t s, int nn, float minor_scale,
                         int rescore) {
    Workspace &ws = ix.ws;
    HN_CUDA(cudaMemsetAsync(ws.status, 0, 8 * sizeof(int32_t), s));
    HN_CUDA(cudaMemsetAsync(ws.counters, 0, 8 * sizeof(long long), s));
    hn_status st = run_search(ix, q, nq, scan, seed, topk, out_idx, out_sim, timing, s, nn, minor_scale, rescore);
    if (st != HN_OK) return st;
    HN_CUDA(cudaMemcpyAsync(ws.h_status, ws.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HN_CUDA(cudaMemcpyAsync(ws.h_status + 8, ws.counters, 8 * sizeof(long long), cudaMemcpyDeviceToHost, s));
    return HN_OK;
}

// After the stream has run: HN_OK, an error, or HN_ERR_OVERFLOW with *want_cap set.
hn_status check_search(Index &ix, int64_t nq, int32_t *want_cap) {
    Workspace &ws = ix.ws;
    const long long *hc = reinterpret_cast<const long long *>(ws.h_status + 8);
    ws.last_max = (int32_t)std::min<long long>(hc[CT_MAXSURV], 1 << 30);
    if (ws.h_status[ST_NOT_NORMALIZED]) return fail(HN_ERR_NOT_NORMALIZED, "a query violates the HN norm identities");
    if (ws.h_status[ST_TIMEOUT]) return fail(HN_ERR_TIMEOUT, "a device-side wait timed out");
    if (!ws.h_status[ST_OVERFLOW]) return HN_OK;
    if (hc[CT_MAXSURV] >= (1 << 30)) return fail(HN_ERR_OVERFLOW, "survivor storage overflow");
    const int64_t want = hc[CT_MAXSURV] + hc[CT_MAXSURV] / 8 + 32;
    if ((int64_t)nq * want * 4 > ((int64_t)96 << 30)) return fail(HN_ERR_OVERFLOW, "survivor storage would exceed 96 GiB");
    *want_cap = (int32_t)want;
    return HN_ERR_OVERFLOW;
}

int32_t default_cap(const Index &ix) {
    return std::max<int32_t>(std::max<int32_t>(256, ix.ws.bucket_cap), ix.ws.last_max + ix.ws.last_max / 4);
}

}  // namespace hn

// hn_search_batch (nn = 1) and hn_search_topk (nn = k): validation, scratch sizing,
// the search pipeline, overflow re-runs and statistics.
static hn_status search_impl(hn_index *index, const float *q, int64_t nq, int nn, const hn_search_opts *opts,
                             int64_t *out_idx, double *out_sim, hn_search_stats *stats, void *stream) {
    if (!index) return fail(HN_ERR_INVALID_ARG, "index is NULL");
    Index &ix = index->ix;
    if (nq < 0 || nq > (int64_t)1 << 30) return fail(HN_ERR_INVALID_ARG, "need 0 <= nq <= 2^30");
    if (nn < 1 || nn > 32 || nn > ix.n) return fail(HN_ERR_INVALID_ARG, "need 1 <= k <= min(32, n)");
    hn_search_opts o{};
    if (opts) o = *opts;
    if (o.soft != 0 && o.soft != 1) return fail(HN_ERR_INVALID_ARG, "soft must be 0 or 1");
    if (o.soft && !(o.beta >= 0.f && (double)o.beta <= ix.alpha * (1.0 + 1e-6)))
        return fail(HN_ERR_INVALID_ARG, "soft mode needs 0 <= beta <= alpha");
    if (o.soft && nn > 1) return fail(HN_ERR_UNSUPPORTED, "the soft mode serves the 1-NN search only");
    // soft ANN mode: the minor bound scaled by beta / alpha <= 1 (alpha = 0: no minor part at all)
    const float minor_scale = o.soft && ix.alpha > 0 ? (float)std::min(1.0, (double)o.beta / ix.alpha) : 1.f;
    if (o.bucket_cap < 0) return fail(HN_ERR_INVALID_ARG, "bucket_cap < 0");
    const int topk = o.seed_topk ? o.seed_topk : 4;
    if (o.seed) {
        if (proposal_blocks(o.seed) != ix.n_blocks || proposal_k(o.seed) != ix.k)
            return fail(HN_ERR_INVALID_ARG, "the proposal was not trained for this index's blocks");
        if (topk < 1 || topk > 64 || topk > ix.n_blocks) return fail(HN_ERR_INVALID_ARG, "need 1 <= seed_topk <= 64");
        if (nn > 1) return fail(HN_ERR_UNSUPPORTED, "the proposal seeds the 1-NN search only");
    }
    const int scan = pick_scan(ix, nq, o.scan);
    if (scan != HN_SCAN_STREAM && scan != HN_SCAN_DENSE && scan != HN_SCAN_DENSE_TWO_PASS)
        return fail(HN_ERR_INVALID_ARG, "bad scan kind");
    if (scan != HN_SCAN_STREAM && !dense_scan_supported(ix))
        return fail(HN_ERR_UNSUPPORTED, "dense scan needs a BF16 or FP8 prefix index");
    if (o.test_stall && (scan == HN_SCAN_STREAM || o.seed))
        return fail(HN_ERR_INVALID_ARG, "test_stall needs a dense scan without a proposal seed");
    if (o.scratch_limit < 0) return fail(HN_ERR_INVALID_ARG, "scratch_limit < 0");
    if (o.wait_limit_ns != 0 && (o.wait_limit_ns < 1000 || o.wait_limit_ns > 10000000000ull))
        return fail(HN_ERR_INVALID_ARG, "need wait_limit_ns = 0 or 1e3 <= wait_limit_ns <= 1e10");
    if (o.reserved[0]) return fail(HN_ERR_INVALID_ARG, "reserved option fields must be zero");
    if (o.test_stall != 0 && o.test_stall != 1) return fail(HN_ERR_INVALID_ARG, "test_stall must be 0 or 1");
    if (o.test_plain_epilogue != 0 && o.test_plain_epilogue != 1)
        return fail(HN_ERR_INVALID_ARG, "test_plain_epilogue must be 0 or 1");
    if (o.test_stall && (o.wait_limit_ns == 0 || o.wait_limit_ns > 10000000ull))
        return fail(HN_ERR_INVALID_ARG, "test_stall needs 1e3 <= wait_limit_ns <= 1e7");
    if (o.rescore < HN_RESCORE_FILTER16 || o.rescore > HN_RESCORE_FULL) return fail(HN_ERR_INVALID_ARG, "bad rescore mode");
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->n_queries = nq;
        stats->n_entries = ix.n;
        stats->scan = scan;
    }
    if (nq == 0) return HN_OK;
    if (!q || !out_idx || !out_sim || !aligned16(q)) return fail(HN_ERR_INVALID_ARG, "null or unaligned pointer");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t cap = o.bucket_cap ? o.bucket_cap : default_cap(ix);
    Workspace &ws = ix.ws;
    const bool timing = o.timing != 0;
    if (timing && !ws.ev_ready) {
        for (cudaEvent_t &e : ws.ev) HN_CUDA(cudaEventCreate(&e));
        ws.ev_ready = true;
    }
    int32_t reruns = 0, kernels = 0;
    for (;;) {
        hn_status st = prepare_search(ix, nq, scan, cap, nn, o.seed != nullptr, o.scratch_limit);
        if (st != HN_OK) return st;
        ws.wait_ns = o.wait_limit_ns;
        ws.stall = o.test_stall;
        ws.plain = o.test_plain_epilogue;
        st = enqueue_search(ix, q, nq, scan, o.seed, topk, out_idx, out_sim, timing, s, nn, minor_scale,
                            o.rescore);
        ws.wait_ns = 0;
        ws.stall = 0;
        ws.plain = 0;
        if (st != HN_OK) {
            ws.gbits_limit = 0;
            return st;
        }
        // query prep and rescore, plus Phase 1 and the threshold (or the seed's kernels), plus
        // the Phase-2 launches; the one-pass dense form counts its scan, threshold and extraction
        int32_t passes = 0;
        if (scan == HN_SCAN_DENSE && !o.seed) {
            const int32_t l = (int32_t)dense_phase2_launches(ix, nq, true);
            kernels += 2 + l;
            passes = l / 3;
        } else {
            const int32_t l = scan == HN_SCAN_STREAM ? 1 : (int32_t)dense_phase2_launches(ix, nq, false);
            kernels += (o.seed ? 3 + 5 * (int32_t)((nq + 8191) / 8192) : 4) + l;
            passes = scan == HN_SCAN_STREAM ? 0 : l / 2;
        }
        ws.gbits_limit = 0;  // the scratch limit holds for this search only
        HN_CUDA(cudaStreamSynchronize(s));
        int32_t want = 0;
        st = check_search(ix, nq, &want);
        if (st == HN_OK) {
            if (stats) {
                const long long *hc = reinterpret_cast<const long long *>(ws.h_status + 8);
                stats->survivors = hc[CT_SURVIVORS];
                stats->max_survivors = hc[CT_MAXSURV];
                stats->fp64_rescored = hc[CT_FP64];
                stats->groups_scored = hc[CT_GROUPS];
                stats->rescore_skipped = hc[CT_SKIPPED];
                stats->reruns = reruns;
                stats->kernels = kernels;
                stats->passes = passes;
                if (timing) {
                    float *ms[5] = {&stats->ms_prep, &stats->ms_phase1, &stats->ms_threshold, &stats->ms_phase2,
                                    &stats->ms_rescore};
                    for (int i = 0; i < 5; ++i) HN_CUDA(cudaEventElapsedTime(ms[i], ws.ev[i], ws.ev[i + 1]));
                    HN_CUDA(cudaEventElapsedTime(&stats->ms_total, ws.ev[0], ws.ev[5]));
                }
            }
            return HN_OK;
        }
        if (st != HN_ERR_OVERFLOW) return st;
        // survivors did not fit: grow the slots to the largest count seen and run again
        if (reruns >= 2) return fail(HN_ERR_OVERFLOW, "survivor storage overflow after re-runs");
        cap = want;
        ++reruns;
    }
}

extern "C" {

hn_status hn_search_batch(hn_index *index, const float *q, int64_t nq, const hn_search_opts *opts, int64_t *out_idx,
                          double *out_sim, hn_search_stats *stats, void *stream) {
    return search_impl(index, q, nq, 1, opts, out_idx, out_sim, stats, stream);
}

hn_status hn_search_topk(hn_index *index, const float *q, int64_t nq, int32_t k, const hn_search_opts *opts,
                         int64_t *out_idx, double *out_sim, hn_search_stats *stats, void *stream) {
    return search_impl(index, q, nq, k, opts, out_idx, out_sim, stats, stream);
}

hn_status hn_prefix_scores(hn_index *index, const float *q, int64_t nq, int32_t path, float *out_scores,
                           float *out_slack, void *stream) {
    if (!index) return fail(HN_ERR_INVALID_ARG, "index is NULL");
    Index &ix = index->ix;
    if (!dense_scan_supported(ix)) return fail(HN_ERR_UNSUPPORTED, "needs a BF16 or FP8 prefix index");
    if (path != 0 && path != 1) return fail(HN_ERR_INVALID_ARG, "path must be 0 or 1");
    if (nq < 1 || nq > ((int64_t)1 << 28) / ix.n) return fail(HN_ERR_INVALID_ARG, "need 1 <= nq and nq * n <= 2^28");
    if (!q || !out_scores || !out_slack || !aligned16(q)) return fail(HN_ERR_INVALID_ARG, "null or unaligned pointer");
    cudaStream_t s = (cudaStream_t)stream;
    hn_status st = ensure_ws(ix, nq, std::max<int32_t>(ix.ws.bucket_cap, 1));
    if (st != HN_OK) return st;
    Workspace &ws = ix.ws;
    HN_CUDA(cudaMemsetAsync(ws.status, 0, 8 * sizeof(int32_t), s));
    HN_CUDA(launch_query_prep(ix, q, nq, 1.f, s));
    HN_CUDA(launch_prefix_scores(ix, nq, path, out_scores, s));
    HN_CUDA(cudaMemcpyAsync(out_slack, ws.qeps, sizeof(float) * nq, cudaMemcpyDeviceToDevice, s));
    HN_CUDA(cudaMemcpyAsync(ws.h_status, ws.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HN_CUDA(cudaStreamSynchronize(s));
    if (ws.h_status[ST_NOT_NORMALIZED]) return fail(HN_ERR_NOT_NORMALIZED, "a query violates the HN norm identities");
    if (ws.h_status[ST_TIMEOUT]) return fail(HN_ERR_TIMEOUT, "a device-side wait timed out");
    return HN_OK;
}

hn_status hn_bruteforce(const hn_index *index, const float *q, int64_t nq, int64_t *out_idx, double *out_sim,
                        void *stream) {
    if (!index) return fail(HN_ERR_INVALID_ARG, "index is NULL");
    if (nq < 0 || nq > (int64_t)1 << 30) return fail(HN_ERR_INVALID_ARG, "need 0 <= nq <= 2^30");
    if (nq == 0) return HN_OK;
    if (!q || !out_idx || !out_sim || !aligned16(q)) return fail(HN_ERR_INVALID_ARG, "null or unaligned pointer");
    Index &ix = const_cast<hn_index *>(index)->ix;
    hn_status st = ensure_ws(ix, nq, std::max<int32_t>(ix.ws.bucket_cap, 1));
    if (st != HN_OK) return st;
    HN_CUDA(launch_bruteforce(ix, q, nq, out_idx, out_sim, (cudaStream_t)stream));
    return HN_OK;
}

}  // extern "C"
