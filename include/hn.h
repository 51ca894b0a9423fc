/*
 * hn.h -- C ABI of the B300 (sm_103a) exact 1-NN search library for
 * Hierarchical-Normalization (HN) descriptors.
 *
 * The method (§3): a 128-dim descriptor is split into a K-dim major prefix of
 * norm sqrt(1-alpha) and a (128-K)-dim minor part of norm sqrt(alpha) (Eq. 1).
 * Because <q_minor, x_minor> <= alpha (Cauchy-Schwarz, Eq. 3), dot_K + alpha
 * bounds the full inner product (Eq. 2 and Eq. 3), so a scan of the major
 * prefixes prunes every entry whose bound cannot beat the best fully scored
 * entry, and only survivors are scored at 128 dims (Algorithm 1, §3.3).  The
 * result equals exhaustive search (Theorem 1) and is deterministic with ties
 * resolved by index (Theorem 2).
 *
 * Conventions shared by every entry point:
 *  - Every array argument is a DEVICE pointer on the current CUDA device,
 *    owned by the caller, row-major and densely packed.  Float arrays need
 *    16-byte alignment.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; calls that must report device-detected errors
 *    (normalisation, invariant checks, survivor overflow) synchronise that
 *    stream once before returning, as documented per call.
 *  - Argument errors are detected on the host before any work is enqueued and
 *    leave outputs untouched.
 *  - Handles (hn_index) are owned by the library and released by their
 *    destroy call.  A handle may be used by one host thread at a time.
 *  - hn_last_error() returns a message for the most recent failure on the
 *    calling host thread.
 *  - D (the descriptor dimension) must be 128 (HardNet's width, §1, §3.1).
 */
#ifndef HN_H
#define HN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hn_status {
    HN_OK = 0,
    HN_ERR_INVALID_ARG = 1,    /* bad size, pointer, alignment or parameter */
    HN_ERR_NOT_NORMALIZED = 2, /* input violates the norm identities below Eq. 1 */
    HN_ERR_ZERO_NORM = 3,      /* Eq. 1 undefined: zero major (or zero minor with alpha > 0) */
    HN_ERR_OOM = 4,            /* device allocation failed */
    HN_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    HN_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
    HN_ERR_OVERFLOW = 7,       /* survivor storage still too small after re-running */
    HN_ERR_UNSUPPORTED = 8     /* valid request this build does not serve (e.g. D != 128) */
} hn_status;

/* Storage precision of the major prefix that the scan reads. */
typedef enum hn_prefix {
    HN_PREFIX_F32 = 0,  /* binary32 prefix, scanned with FP32 FMA */
    HN_PREFIX_BF16 = 1, /* bfloat16 prefix, scanned on the tensor cores (FP32 accumulation) */
    HN_PREFIX_FP8_E4M3 = 2, /* FP8 e4m3 prefix with a per-entry binary32 scale (a power of two, so
                              that dequantisation is exact) and a per-entry rounding-error term;
                              scanned on the tensor cores (FP32 accumulation) or dequantised on the
                              CUDA cores.  K <= 64. */
    HN_PREFIX_I8 = 3       /* 8-bit fixed-point prefix (§7, "Power-of-two alpha"; the remark after
                              Theorem 2 on quantised descriptors): x^ = RN(x / s) in [-127, 127]
                              with ONE power-of-two scale s for the whole index, and queries coded
                              the same way with a power-of-two scale per query.  The CUDA-core
                              scan forms the prefix dot product in integers (dp4a), so it is
                              exact; the only error terms are the two quantisation residuals.
                              Stream scan only (HN_SCAN_DENSE returns HN_ERR_UNSUPPORTED).
                              K <= 64. */
} hn_prefix;

/* Which prefix-scan kernel runs (Phase 1 and Phase 2 of Algorithm 1). */
typedef enum hn_scan {
    HN_SCAN_AUTO = 0,   /* pick by query count and prefix type (HN_SCAN_DENSE from the autotuned
                           batch size on a BF16 or FP8 index, else HN_SCAN_STREAM) */
    HN_SCAN_STREAM = 1, /* CUDA-core FMA scan streaming the prefix (any prefix type), two passes */
    HN_SCAN_DENSE = 2,  /* tcgen05 tensor-core scan (HN_PREFIX_BF16 and HN_PREFIX_FP8_E4M3), ONE pass
                           over the prefix product: it keeps an 8-bit code of the largest score of
                           every (query, 32-entry group) and the best group per (query, entry chunk);
                           the threshold comes from those candidates, and the survivors from the
                           groups whose code reaches the threshold's code.  Same result as the two
                           passes of Algorithm 1; the scratch holds nq * n / 32 bytes of codes */
    HN_SCAN_DENSE_TWO_PASS = 3 /* tcgen05 tensor-core scan in Algorithm 1's two passes: Phase 1 for
                           the threshold candidates, Phase 2 against the threshold (one bit per
                           (query, 32-entry group), nq * n / 256 bytes) */
} hn_scan;

/* How the 1-NN Phase 2 scores its survivors (hn_search_opts.rescore); every mode returns the
 * oracle's answer.  The index keeps an FP16 copy of every row (256 B per entry) for the first. */
typedef enum hn_rescore {
    HN_RESCORE_FILTER16 = 0,    /* certified FP16-row bound first, FP32 row only where it can win */
    HN_RESCORE_BEST_FIRST = 1,  /* the sorted-Phase-2 early exit with the FP32 prefix bound */
    HN_RESCORE_FULL = 2         /* every survivor scored in FP32 (Algorithm 1's Phase 2) */
} hn_rescore;

typedef struct hn_index_opts {
    int32_t prefix;       /* hn_prefix; default HN_PREFIX_F32 */
    int32_t n_blocks;     /* > 0: partition the entries into this many blocks for the learned
                             proposal (1 <= n_blocks <= min(n, 2^20)); 0: no blocks */
    int32_t kmeans_iters; /* Lloyd iterations of the block partition; 0 = 8 */
    uint32_t seed;        /* reserved for partition seeding; currently unused, may be 0 */
    int32_t reserved[4];  /* must be zero */
} hn_index_opts;

typedef struct hn_proposal hn_proposal;

typedef struct hn_search_opts {
    int32_t scan;         /* hn_scan; default HN_SCAN_AUTO */
    int32_t bucket_cap;   /* survivor slots per query; 0 = library default (grown on overflow) */
    int32_t timing;       /* non-zero: time each step with CUDA events on `stream` (fills stats->ms_*) */
    int32_t seed_topk;    /* blocks the proposal contributes per query (with `seed`); 0 = 4 */
    const hn_proposal *seed; /* NULL: plain search.  Otherwise the proposal's top blocks give the
                                threshold and the Phase-1 scan is skipped (result unchanged) */
    int32_t soft;         /* 0: exact search.  1: soft ANN mode (the threshold relaxation of §7): the
                             admissible minor bound alpha of the skip test becomes beta, i.e. the
                             stored-norm minor bound is scaled by beta / alpha; beta = alpha is the
                             exact search, smaller beta prunes more and may miss the true neighbour;
                             the best fully scored threshold candidate always stays a candidate (as
                             Algorithm 1 keeps its Phase-1 winner).  1-NN only (hn_search_batch) */
    float beta;           /* with soft = 1: 0 <= beta <= alpha (else HN_ERR_INVALID_ARG) */
    int64_t scratch_limit; /* > 0: bytes the dense scan's group map (codes or bits) may take; a larger
                              batch runs in passes over 256-query tiles (at least one tile a pass,
                              whatever the limit).  0: up to 16 GiB of codes (one-pass) or 4 GiB of
                              bits (two-pass) */
    uint64_t wait_limit_ns; /* device-side wait limit of the dense scan's main loop in nanoseconds of
                              GPU global time; 0 = 2 s, else 1e3 .. 1e10 (HN_ERR_INVALID_ARG
                              otherwise).  A wait that runs out ends the kernel early (its copies and
                              MMAs still drain with the 2 s limit) and the call returns
                              HN_ERR_TIMEOUT.  Limits of a few microseconds make the waits of a
                              normally loaded scan run out: used to exercise that path */
    int32_t rescore;      /* hn_rescore: how the 1-NN Phase 2 scores its survivors (same result in
                             every mode).  HN_RESCORE_FILTER16 (0, default): each survivor first gets
                             a certified upper bound from its FP16 row (256 B: the FP32 dot of the
                             query with the row rounded to FP16, plus the rounding and summation
                             slack); only survivors whose bound reaches the best certified full
                             score so far (starting from the threshold candidates') are read and
                             scored in FP32.  HN_RESCORE_BEST_FIRST (1): the early exit the remark
                             after Algorithm 1 describes for a sorted Phase 2, with the FP32 prefix
                             score as the bound.  HN_RESCORE_FULL (2): every survivor scored in
                             FP32 in slot order (Algorithm 1's Phase 2 in index order).
                             hn_search_topk: HN_RESCORE_FILTER16 bounds against the k-th best
                             certified score; the other two score every survivor in FP32 */
    int32_t test_stall;   /* failure-path test hook, 0 in normal use.  1: in every dense-scan launch
                             of this call, each CTA's copy producer stops after the CTA's first work
                             unit, so the MMA warps wait for a query copy that never comes; that
                             wait runs out after wait_limit_ns, the CTA raises its abort flag, the
                             copies and MMAs in flight drain, tensor memory is freed and the call
                             returns HN_ERR_TIMEOUT.  Needs a dense scan, no seed and
                             1e3 <= wait_limit_ns <= 1e7 (HN_ERR_INVALID_ARG otherwise) */
    int32_t test_plain_epilogue; /* test hook, 0 in normal use.  1: the one-pass dense scans of this
                             call run their unsplit form (no register split between the warp
                             groups: one reducing tensor-memory load in flight per epilogue warp),
                             the form a build whose scan kernel does not get exactly 96 registers a
                             thread falls back to.  Same result.  0 or 1 (HN_ERR_INVALID_ARG
                             otherwise) */
    int32_t reserved[1];  /* must be zero */
} hn_search_opts;

/* Counters of one hn_search_batch call (filled when the stats pointer is non-NULL). */
typedef struct hn_search_stats {
    int64_t n_queries;
    int64_t n_entries;
    int64_t survivors;      /* (query, entry) pairs passing the Phase-2 bound test */
    int64_t max_survivors;  /* largest survivor count of a single query */
    int64_t fp64_rescored;  /* near-tie candidates re-scored in binary64 */
    int32_t reruns;         /* Phase-2 re-runs after survivor-slot overflow */
    int32_t scan;           /* hn_scan that ran */
    int32_t kernels;        /* kernel launches made by this call (all runs) */
    int32_t passes;         /* dense scan: passes over query tiles of the last run (its group map
                               held that many parts of the batch; see scratch_limit); 0 otherwise */
    /* device time of each step of the last run, milliseconds (with opts->timing) */
    float ms_prep;          /* query prefix packing and slack computation */
    float ms_phase1;        /* Phase-1 prefix scan, or the proposal's inference when seeded;
                               HN_SCAN_DENSE: its one tensor-core scan (first pass) */
    float ms_threshold;     /* full score of the Phase-1 (or proposed) candidates -> threshold */
    float ms_phase2;        /* Phase-2 prefix scan with the bound test; HN_SCAN_DENSE: the
                               extraction of the survivors from the group codes (plus any
                               further passes over query tiles) */
    float ms_rescore;       /* survivor rescore, binary64 near-ties, argmax */
    float ms_total;         /* whole search */
    int64_t groups_scored;  /* dense scan: 32-entry groups the survivor extraction scored on the
                               CUDA cores (the group map's pass count of the bound test) */
    int64_t rescore_skipped; /* best-first rescore: survivors dropped by the prefix bound before
                               their full score */
} hn_search_stats;

typedef struct hn_index_info {
    int64_t n;              /* entries */
    int32_t d, k;           /* dimension (128) and major width K */
    double alpha;           /* energy split */
    int32_t prefix;         /* hn_prefix */
    int32_t k_pad;          /* stored prefix width (K rounded up for the scan) */
    int64_t device_bytes;   /* device memory held by the index */
    float minor_norm_max;   /* max_i |x_i,minor| of the stored values, rounded up */
    float major_norm_max;   /* max_i |x_i,major|, rounded up */
    float resid_norm_max;   /* max_i |x_i,major - prefix_i| (0 for HN_PREFIX_F32), rounded up;
                               prefix_i = the dequantised stored prefix */
    float prefix_norm_max;  /* max_i |prefix_i|, rounded up */
    int32_t n_blocks;       /* block partition size (0: none) */
    int32_t reserved;
} hn_index_info;

/* Options of hn_proposal_train (zero fields take the defaults in brackets). */
typedef struct hn_train_opts {
    int32_t hidden1, hidden2;   /* hidden widths [256, 256] */
    int32_t epochs;             /* passes over the pairs [4] */
    int32_t batch;              /* mini-batch rows [4096] */
    float lr;                   /* Adam learning rate [1e-3]; beta1 0.9, beta2 0.999, eps 1e-8 */
    uint32_t seed;              /* initial weights and shuffling [0] */
    const hn_proposal *init;    /* non-NULL: continue training this network (weights, Adam state) */
    int32_t precision;          /* the training GEMMs: 0 = on the tensor cores with BF16 operands and
                                   FP32 accumulation (default); 1 = FP32 CUDA-core GEMMs (the
                                   arithmetic hn_mlp_loss_grad checks against binary64).  The master
                                   weights and the Adam state are FP32 either way */
    int32_t reserved[1];        /* must be zero */
} hn_train_opts;

typedef struct hn_proposal_info {
    int32_t k, hidden1, hidden2, n_blocks;
    int64_t n_params;
    int64_t steps;              /* Adam steps taken so far */
    int32_t epochs;             /* epochs trained so far */
    float last_loss;            /* mean cross-entropy of the last training batch */
} hn_proposal_info;

typedef struct hn_index hn_index;

/* Library version, (major << 16) | minor. */
int32_t hn_version(void);

/* Message describing the last failure on this host thread ("" if none). */
const char *hn_last_error(void);

/*
 * HN normalisation (Eq. 1, §3.1), row by row:
 *   out[:k] = sqrt(1-alpha) * in[:k] / |in[:k]|,  out[k:] = sqrt(alpha) * in[k:] / |in[k:]|
 * Arithmetic: binary64 sums of squares in dimension order, sqrt and division
 * correctly rounded, each output rounded once to binary32; alpha == 0 sets the
 * minor to zero.  in, out: n x d float32 (may be the same buffer).
 * Requirements: d == 128, 1 <= k < d, 0 <= alpha < 1, n >= 0.
 * Errors: HN_ERR_ZERO_NORM if some row has a zero major part (or a zero minor
 * part with alpha > 0); out is then unspecified.  Synchronises `stream`.
 */
hn_status hn_normalize(const float *in, float *out, int64_t n, int32_t d, int32_t k, double alpha,
                       void *stream);

/*
 * The same normalisation, enqueued on `stream` without synchronising it (for serving
 * loops that normalise each batch just before searching it).  Same arithmetic and
 * requirements as hn_normalize; the arguments are checked on the host before the launch
 * (HN_ERR_INVALID_ARG, nothing enqueued).  A row with a non-finite value or a zero major
 * (or, with alpha > 0, minor) part is copied to `out` unchanged, and hn_search_batch /
 * hn_search_topk / hn_search_multi then report HN_ERR_NOT_NORMALIZED for the batch.
 * status: NULL, or device memory int32_t[2] that this call does not clear (the caller
 * zeroes it once and may read it after any number of calls): the kernel sets status[0]
 * to 1 when a row held a non-finite value and status[1] to 1 when a row had a zero norm.
 */
hn_status hn_normalize_async(const float *in, float *out, int64_t n, int32_t d, int32_t k, double alpha,
                             int32_t *status, void *stream);

/*
 * Build a search index over n HN-normalised entries x (n x d float32, device).
 * The index copies x (the caller may free it once this call returns) and packs
 * the major prefixes into a separate contiguous array in the chosen precision
 * (the Structure-of-Arrays layout of §6.1), plus per-entry minor norms.
 * Checks the norm identities below Eq. 1 on every row:
 *   | |x_major|^2 - (1-alpha) | <= (d+4) 2^-24 (1-alpha), same for the minor with alpha;
 * otherwise HN_ERR_NOT_NORMALIZED.  Synchronises `stream`.
 * Requirements: d == 128, 1 <= k <= 64 (else HN_ERR_UNSUPPORTED), 0 <= alpha < 1,
 * 1 <= n < 2^31 - 256.  opts may be NULL (defaults).  On success *out owns
 * device memory until hn_index_destroy.
 */
hn_status hn_index_build(const float *x, int64_t n, int32_t d, int32_t k, double alpha,
                         const hn_index_opts *opts, hn_index **out, void *stream);

hn_status hn_index_destroy(hn_index *index);

hn_status hn_index_get_info(const hn_index *index, hn_index_info *info);

/*
 * Exact 1-NN search of nq HN-normalised queries q (nq x d float32, device):
 *   out_idx[j] = min{ i : <q_j, x_i> = max_i' <q_j, x_i'> },  out_sim[j] = that maximum,
 * where <.,.> is the binary64 sum of the d products in dimension order -- the
 * result of exhaustive full-vector search (Theorem 1) with ties resolved by
 * the lowest index (Theorem 2).  out_idx: nq int64, out_sim: nq double.
 *
 * Steps (Algorithm 1 on the GPU): Phase 1 scans every prefix and takes each
 * query's best prefix score; that entry is scored in full, giving a certified
 * threshold; Phase 2 rescans the prefixes and keeps entry i only if
 *   prefix_score + scan_error + |q_minor| |x_minor| >= threshold;
 * survivors are scored in FP32, and the ones within the FP32 error band of
 * the best are scored again in binary64 to pick the exact winner.
 * The index's scratch storage is reused and grown on demand (device
 * allocation on first use and after an overflow).  Besides the per-query
 * survivor slots it holds, for the tensor-core scan, one bit per (query,
 * 32-entry group): nq * n / 256 bytes (1 GB for 65,536 queries over 4M
 * entries), at most 4 GiB (larger batches take Phase 2 in passes).  Calls on
 * one index must not overlap.  Checks the query norm identities (HN_ERR_NOT_NORMALIZED).
 * Synchronises `stream` once at the end.  opts and stats may be NULL.
 */
hn_status hn_search_batch(hn_index *index, const float *q, int64_t nq, const hn_search_opts *opts,
                          int64_t *out_idx, double *out_sim, hn_search_stats *stats, void *stream);

/*
 * Exact top-k search (an extension of the problem statement of §3.3, which asks
 * for the single nearest neighbour): for every query the k entries of largest
 * binary64 inner product <q_j, x_i> (as defined for hn_search_batch), in the order
 * (similarity descending, index ascending), so that rank 0 is hn_search_batch's
 * answer.  out_idx[j * k + r] and out_sim[j * k + r] (nq * k int64 / double) give
 * rank r of query j.  Requires 1 <= k <= min(32, n).
 * Steps: Algorithm 1 with the threshold T_q certified for the k-th best (the k-th
 * largest of the lower bounds of k distinct fully scored Phase-1 candidates; an
 * entry whose bound is below T_q cannot be among the k best), the same Phase-2
 * bound test, FP32 rescore of the survivors, and binary64 scores for every survivor
 * within the FP32 error band of the k-th FP32 score.  opts as for hn_search_batch;
 * opts->seed (the proposal) and opts->soft are not supported for k > 1 (HN_ERR_UNSUPPORTED).
 * Errors, scratch storage and synchronisation as for hn_search_batch.
 */
hn_status hn_search_topk(hn_index *index, const float *q, int64_t nq, int32_t k, const hn_search_opts *opts,
                         int64_t *out_idx, double *out_sim, hn_search_stats *stats, void *stream);

/*
 * Merge step of the entry-range sharded search.  Theorem 1's exact maximum is
 * associative: cut the database into contiguous entry ranges (one per GPU), search
 * each range exactly (hn_search_batch, k = 1, or hn_search_topk), gather every
 * range's results, and the k best of the union in the order (similarity
 * descending, global index ascending) -- Theorem 2's tie rule -- are the answer
 * over the whole database.
 *   idx, sim     [n_shards][nq][k] int64 / double: shard r's answers in that order,
 *                with indices local to the shard (idx < 0: no entry, e.g. a shard
 *                holding fewer than k entries);
 *   id_offset    [n_shards] int64: the global index of each shard's entry 0;
 *   out_idx, out_sim  [nq][k]: the merged answers (global indices; -1 and -inf
 *                where fewer than k entries exist in all).
 * Requires 1 <= n_shards <= 64, 1 <= k <= 32, nq >= 0.
 * hn_merge_topk: every array a DEVICE pointer; one thread per query on `stream`,
 * does not synchronise.  hn_merge_topk_host: the same on HOST arrays, on the
 * calling thread (for results gathered through host memory).
 */
hn_status hn_merge_topk(const int64_t *idx, const double *sim, const int64_t *id_offset, int32_t n_shards,
                        int64_t nq, int32_t k, int64_t *out_idx, double *out_sim, void *stream);
hn_status hn_merge_topk_host(const int64_t *idx, const double *sim, const int64_t *id_offset, int32_t n_shards,
                             int64_t nq, int32_t k, int64_t *out_idx, double *out_sim);

/*
 * Batched serving (an extension of the method; the paper searches one query
 * at a time).  One call answers nb batches of queries, each against its own
 * index; every batch's result is the same as hn_search_batch would give.
 * Batches are grouped by index and each group's queries concatenated, so that
 * small batches share the dense scan's work units.  The groups that take the
 * one-pass dense scan on indexes of one tile format (prefix type and padded K)
 * run their scans as ONE persistent launch whose work units cover every such
 * group; each group's query preparation, threshold, survivor extraction and
 * rescore run on a stream of its own, as does the whole pipeline of any other
 * group.  With opts->use_graph (default 1) the whole set is
 * captured once into a CUDA graph and the graph is replayed as long as the
 * same batches come back (same indexes, query and output pointers and sizes,
 * and no reallocation of the indexes' scratch in between).  Synchronises
 * `stream` once (plus re-runs after a survivor overflow).  The call holds a
 * process-wide lock; the indexes must not be used concurrently elsewhere.
 */
typedef struct hn_batch {
    hn_index *index;      /* index to search */
    const float *q;       /* nq x 128 HN-normalised float32 queries (device) */
    int64_t nq;
    int64_t *out_idx;     /* nq int64 (device) */
    double *out_sim;      /* nq double (device) */
} hn_batch;

typedef struct hn_multi_opts {
    int32_t use_graph;    /* capture and replay a CUDA graph [1] */
    int32_t reserved[7];  /* must be zero */
} hn_multi_opts;

typedef struct hn_multi_stats {
    int64_t n_queries;
    int32_t n_batches, n_groups;
    int32_t graph_replayed;  /* 1: an instantiated graph was replayed */
    int32_t reruns;          /* re-runs after survivor-slot overflow */
    float ms_total;          /* device time from the start of the set to its last batch */
    float batch_ms_p50, batch_ms_p99, batch_ms_max;  /* time from the start to each batch's completion */
    int32_t joined;          /* groups whose dense scans ran as one shared persistent launch (0: none) */
    int64_t survivors;       /* Phase-2 survivors over all batches */
} hn_multi_stats;

hn_status hn_search_multi(const hn_batch *batches, int32_t nb, const hn_multi_opts *opts, hn_multi_stats *stats,
                          void *stream);

/*
 * Autotuner: times the streaming and dense scans of `index` on n_sizes batch
 * sizes (the index's own first rows as queries) and stores in the index the
 * smallest batch from which hn_search_batch's automatic choice takes the dense
 * scan, and the dense work-unit granularity (units per SM: 32, 64, 128 or 256)
 * that is fastest at the largest size.  Synchronises `stream`.
 */
#define HN_TUNE_MAX 16
typedef struct hn_tune_result {
    int32_t n_sizes;
    int32_t dense_min_q;      /* chosen crossover (INT32_MAX: the dense scan never won) */
    int32_t units_per_cta;    /* chosen dense work-unit granularity */
    int32_t reserved;
    int64_t sizes[HN_TUNE_MAX];
    float ms_stream[HN_TUNE_MAX];
    float ms_dense[HN_TUNE_MAX];   /* -1 when the index has no tensor-core (BF16 or FP8) prefix */
    float ms_units[4];             /* dense time at the largest size for 32, 64, 128, 256 units per SM */
} hn_tune_result;

hn_status hn_autotune(hn_index *index, const int64_t *sizes, int32_t n_sizes, hn_tune_result *out, void *stream);

/*
 * Block partition of an index built with opts.n_blocks > 0 (device arrays, may be NULL):
 * block_start[n_blocks + 1] (block b = sorted positions [start[b], start[b+1])),
 * block_ids[n] (entry ids in block order), block_of[n] (block of each entry).
 * Entries are sorted by nearest centre of a spherical k-means over the major
 * prefixes, then cut into equal contiguous blocks.  Does not synchronise.
 */
hn_status hn_index_blocks(const hn_index *index, int32_t *block_start, int32_t *block_ids, int32_t *block_of,
                          void *stream);

/*
 * Learned block proposal (an extension that seeds the threshold of Algorithm 1;
 * the paper has no network).  An MLP  K -> hidden1 -> hidden2 -> n_blocks with
 * exact GELU maps a query's major prefix to block scores; it is trained with
 * softmax cross-entropy and Adam by this library's kernels on pairs
 * (train_q[j], block of its nearest neighbour).  nn_block (npairs int32, device)
 * gives the labels; NULL labels them with hn_search_batch (exact).
 * train_q: npairs x 128 HN-normalised float32 (device).  Synchronises `stream`.
 * Training runs in FP32 with FP32 master weights; inference uses the weights
 * rounded to BF16 with FP32 accumulation.
 */
hn_status hn_proposal_train(const hn_index *index, const float *train_q, const int32_t *nn_block, int64_t npairs,
                            const hn_train_opts *opts, hn_proposal **out, void *stream);

/* Top-k blocks per query (out_blocks: nq x topk int32, device), by (score desc, block asc).
 * Inference runs the three layers on the tensor cores (hn_linear_bf16's arithmetic). */
hn_status hn_proposal_infer(const hn_proposal *proposal, const float *q, int64_t nq, int32_t topk,
                            int32_t *out_blocks, void *stream);

hn_status hn_proposal_get_info(const hn_proposal *proposal, hn_proposal_info *info);

/* Checkpoint: weights and Adam state in a flat binary file with a header. Synchronous. */
hn_status hn_proposal_save(const hn_proposal *proposal, const char *path);
hn_status hn_proposal_load(const char *path, hn_proposal **out);
hn_status hn_proposal_destroy(hn_proposal *proposal);

/*
 * Verification entry point of the proposal's training kernels: mean softmax
 * cross-entropy of a batch and its gradient w.r.t. all parameters, computed by
 * the same forward and backward kernels hn_proposal_train uses with precision 1
 * (FP32 CUDA-core GEMMs).  params and grads: [W1 (h1 x k), b1, W2 (h2 x h1), b2,
 * W3 (c x h2), b3] float32 (device); x: batch x k, y: batch int32 labels in
 * [0, c).  *loss is written on the host.  Synchronises `stream`.
 * hn_mlp_loss_grad_bf16: the same with the tensor-core GEMMs of precision 0 (every
 * GEMM operand rounded to BF16, products summed in FP32); HN_ERR_TIMEOUT if a
 * device-side wait gave up.
 */
hn_status hn_mlp_loss_grad(const float *params, int32_t k, int32_t h1, int32_t h2, int32_t c, const float *x,
                           const int32_t *y, int32_t batch, float *loss, float *grads, void *stream);
hn_status hn_mlp_loss_grad_bf16(const float *params, int32_t k, int32_t h1, int32_t h2, int32_t c, const float *x,
                                const int32_t *y, int32_t batch, float *loss, float *grads, void *stream);

/*
 * The tensor-core GEMM of the proposal's training (an extension; the paper has no
 * network), with strided operands so that every training product -- activations
 * against weights, error signals against weights, transposed error signals against
 * activations -- is one call:
 *   c[i * ldc + j] = sum_{t<k} bf16(a[i * sai + t * sak]) * bf16(b[t * sbk + j * sbj])
 * for i < m, j < n: operands rounded to BF16 (round to nearest even), products exact
 * in FP32 and summed in FP32 by tcgen05.mma.  a, b, c: float32 (device,
 * caller-owned).  Requires m, n >= 0, 1 <= k <= 65536, non-negative strides and
 * ldc >= n (HN_ERR_INVALID_ARG otherwise).  Synchronises `stream`; HN_ERR_TIMEOUT
 * if a device-side wait gave up.
 */
hn_status hn_gemm_bf16(int32_t m, int32_t n, int32_t k, const float *a, int64_t sai, int64_t sak, const float *b,
                       int64_t sbk, int64_t sbj, float *c, int64_t ldc, void *stream);

/*
 * One fully connected layer exactly as the proposal's inference runs it (an
 * extension; the paper has no network): on the tensor cores (tcgen05.mma,
 * kind::f16), operands rounded to BF16 (round to nearest even), products exact
 * and summed in FP32:
 *   out[r][j] = act( sum_{i<k} bf16(in[r][i]) * bf16(w[j][i]) + bias[j] ),
 * act 0: none, 1: GELU 0.5 x (1 + erf(x / sqrt 2)).  in: m x k, w: n x k, out:
 * m x n, all row-major float32 (device, caller-owned); bias: n float32 or NULL.
 * Requires 1 <= k <= 65536, m, n >= 0, act 0 or 1 (HN_ERR_INVALID_ARG
 * otherwise).  Synchronises `stream`; HN_ERR_TIMEOUT if a device-side wait gave
 * up (its output is then unset).
 */
hn_status hn_linear_bf16(const float *in, int32_t m, int32_t k, const float *w, int32_t n, const float *bias,
                         int32_t act, float *out, void *stream);

/*
 * Block scores of the proposal for nq queries (nq x 128 HN-normalised float32,
 * device): out_z[j * n_blocks + b] = z_b of query j, the network output
 * hn_proposal_infer ranks (three hn_linear_bf16 layers on the BF16-rounded
 * weights).  out_z: nq x n_blocks float32 (device, caller-owned).  Asynchronous
 * on `stream`.
 */
hn_status hn_proposal_logits(const hn_proposal *proposal, const float *q, int64_t nq, float *out_z, void *stream);

/*
 * Verification entry point of the scan arithmetic of the reduced-precision
 * prefixes (ext. 1; the paper scans FP32 prefixes and has no counterpart).  For
 * nq HN-normalised queries q (nq x 128 float32, device) and an index with a BF16
 * or FP8 prefix, writes
 *   out_scores[j * n + i]  the prefix score of query j and entry i exactly as the
 *                          search computes it: path 0 the tensor-core scan (the
 *                          FP32 accumulator of q^ . x^; FP8: RN(acc s_i/256 + b_i)),
 *                          path 1 the CUDA-core FMA chain of the survivor extraction
 *                          and of the stream scan;
 *   out_slack[j]           E_q, what the search adds to a prefix score in its bound
 *                          test: the scan's rounding error, |q_minor| max|x_minor|
 *                          and 1e-12 for the binary64 rounding, rounded up.
 * The search is exact because  <q_j, x_i> <= out_scores[j*n+i] + out_slack[j]
 * for every pair (Eq. 2 and Eq. 3 with rounding terms).  out_scores: nq * n
 * float32, out_slack: nq float32 (device, caller-owned).  Requires
 * 1 <= nq, nq * n <= 2^28 and path 0 or 1.  Synchronises `stream`.
 */
hn_status hn_prefix_scores(hn_index *index, const float *q, int64_t nq, int32_t path, float *out_scores,
                           float *out_slack, void *stream);

/*
 * Brute-force baseline (the denominator of the paper's speed-ups, §6.2): the
 * full 128-dim FP32 inner product of every (query, entry) pair on CUDA cores,
 * argmax by (FP32 score, lowest index).  NOT exact in the sense of
 * hn_search_batch: it ranks by FP32 scores.  out_sim receives the FP32 score
 * widened to double.  Does not synchronise.
 */
hn_status hn_bruteforce(const hn_index *index, const float *q, int64_t nq, int64_t *out_idx,
                        double *out_sim, void *stream);

/*
 * Allocation-free variant of hn_bruteforce (the paper has no counterpart; this
 * is a deployment aid).  Same kernels and same results as hn_bruteforce, but
 * its per-query scratch is a fixed array inside the library instead of memory
 * allocated on demand, so the call itself allocates nothing.  It is meant for
 * callers that must not allocate device memory while answering queries: a
 * latency-critical thread (cudaMalloc may block and synchronise the device),
 * a process whose device memory is owned by another allocator or capped by a
 * fixed budget, or a deployment that forbids allocation after start-up.
 *  - index, q, out_idx, out_sim: as for hn_bruteforce (built index, caller-owned
 *    device buffers).  nq <= HN_STATIC_MAX_QUERIES, else HN_ERR_INVALID_ARG.
 *  - The scratch holds HN_STATIC_MAX_QUERIES 8-byte keys (512 KiB) on every GPU
 *    that loads the library, kept until the process exits.
 *  - The first call on each device looks the scratch address up
 *    (cudaGetSymbolAddress) with that device current and keeps it with the
 *    CUDA context's unique id; after a device reset (cudaDeviceReset makes a new
 *    context) the next call looks it up again.  Make the first call on a device,
 *    and the first after a reset, before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents; each
 *    call clears the keys it uses before scanning.  Calls that overlap on the
 *    GPU (e.g. on unordered streams) race and can return wrong answers: order them.
 *  - Does not synchronise.
 */
#define HN_STATIC_MAX_QUERIES 65536
hn_status hn_bruteforce_static(const hn_index *index, const float *q, int64_t nq, int64_t *out_idx,
                               double *out_sim, void *stream);

/*
 * Self-test of failure detection (the paper has no counterpart).  Launches one
 * warp that waits on a device barrier nothing arrives on, through the same bounded
 * wait every mbarrier wait of the dense scan uses.  The wait gives up after
 * limit_ns nanoseconds of GPU global time (1e3 <= limit_ns <= 1e10, else
 * HN_ERR_INVALID_ARG), the kernel returns normally, and the call reports
 * HN_ERR_TIMEOUT -- the expected outcome.  HN_OK would mean the wait did not fire.
 * The CUDA context stays usable.  Synchronises `stream`.
 */
hn_status hn_selftest_wait_timeout(uint64_t limit_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HN_H */
