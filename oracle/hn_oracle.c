/*
 * CPU oracle for exact 1-NN search over Hierarchical-Normalization (HN)
 * descriptors.  TEST INFRASTRUCTURE ONLY: this file is compiled into
 * liboracle and used by tests/, by __graft_entry__.smoke() and by bench.py's
 * CPU-baseline leg.  The CUDA library never links, loads or calls it, and it
 * shares no code, header or constant with the CUDA library.
 *
 * Plain, slow, obviously correct.  All arithmetic is IEEE-754 binary64 with
 * round-to-nearest, summed sequentially in dimension order d = 0, 1, ..., D-1.
 * A product of two binary32 values is exact in binary64 (24 + 24 < 53 bits),
 * so fused and unfused multiply-add give the same bits; only the summation
 * order matters, and it is fixed here.  Build without -ffast-math.
 *
 * Functions and the passages they follow:
 *   hno_normalize   Eq. 1 (§3.1): major = sqrt(1-a) f[:K]/|f[:K]|,
 *                   minor = sqrt(a) f[K:]/|f[K:]|.
 *   hno_dot         Eq. 2 (§3.2): <q, x> as a plain sum of D products.
 *   hno_search      the result the method must reach: exhaustive full-vector
 *                   search (Theorem 1, §3.3) with ties resolved by index
 *                   (Theorem 2 and the remark after it): the lowest index
 *                   among the maximal binary64 similarities.
 *   hno_two_phase   the branch-and-bound that Eq. 3 licenses and Theorem 1
 *                   proves exact (the search of §3.3), with the readings listed
 *                   at its definition.
 *   hno_search_topk exhaustive top-k by (similarity desc, index asc).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { HNO_OK = 0, HNO_BAD_ARG = 1, HNO_ZERO_NORM = 3 };

/* ---------------------------------------------------------------- Eq. 1 */
/* Row-wise HN normalisation.  For each row f (length d):
 *   s_maj = sum_{t<k} f_t^2,  s_min = sum_{t>=k} f_t^2   (binary64, in order)
 *   c_maj = sqrt(1 - alpha) / sqrt(s_maj),  out_t = (float)(f_t * c_maj), t < k
 *   c_min = sqrt(alpha)     / sqrt(s_min),  out_t = (float)(f_t * c_min), t >= k
 * alpha == 0: the minor is set to zero (the paper's alpha = 0 case, §6.2).
 * Returns HNO_ZERO_NORM (first offending row in *bad_row) when s_maj == 0, or
 * s_min == 0 with alpha > 0; HNO_BAD_ARG for a non-finite sum or bad sizes. */
int hno_normalize(const float *in, float *out, int64_t n, int d, int k, double alpha,
                  int64_t *bad_row)
{
    if (n < 0 || d < 2 || k < 1 || k >= d || !(alpha >= 0.0 && alpha < 1.0)) return HNO_BAD_ARG;
    const double r_maj = sqrt(1.0 - alpha);
    const double r_min = sqrt(alpha);
    for (int64_t i = 0; i < n; ++i) {
        const float *f = in + i * d;
        float *o = out + i * d;
        double s_maj = 0.0, s_min = 0.0;
        for (int t = 0; t < k; ++t) s_maj += (double)f[t] * (double)f[t];
        for (int t = k; t < d; ++t) s_min += (double)f[t] * (double)f[t];
        if (!isfinite(s_maj) || !isfinite(s_min)) { if (bad_row) *bad_row = i; return HNO_BAD_ARG; }
        if (s_maj == 0.0 || (alpha > 0.0 && s_min == 0.0)) { if (bad_row) *bad_row = i; return HNO_ZERO_NORM; }
        const double c_maj = r_maj / sqrt(s_maj);
        for (int t = 0; t < k; ++t) o[t] = (float)((double)f[t] * c_maj);
        if (alpha == 0.0) {
            for (int t = k; t < d; ++t) o[t] = 0.0f;
        } else {
            const double c_min = r_min / sqrt(s_min);
            for (int t = k; t < d; ++t) o[t] = (float)((double)f[t] * c_min);
        }
    }
    return HNO_OK;
}

/* Squared norms of the major and minor parts, binary64 in order. */
void hno_part_norms2(const float *x, int64_t n, int d, int k, double *maj2, double *min2)
{
    for (int64_t i = 0; i < n; ++i) {
        const float *f = x + i * d;
        double a = 0.0, b = 0.0;
        for (int t = 0; t < k; ++t) a += (double)f[t] * (double)f[t];
        for (int t = k; t < d; ++t) b += (double)f[t] * (double)f[t];
        maj2[i] = a;
        min2[i] = b;
    }
}

/* ---------------------------------------------------------------- Eq. 2 */
/* <a, b> over dimensions [lo, hi), sequential binary64, starting from acc. */
static double dot_range(const float *a, const float *b, int lo, int hi, double acc)
{
    for (int t = lo; t < hi; ++t) acc += (double)a[t] * (double)b[t];
    return acc;
}

double hno_dot(const float *a, const float *b, int d) { return dot_range(a, b, 0, d, 0.0); }

/* All n similarities of one query (used by tests on small inputs). */
void hno_sims(const float *db, int64_t n, const float *q, int d, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = hno_dot(q, db + i * d, d);
}

/* ------------------------------------------------- exhaustive 1-NN search */
/* Entries are visited in blocks of EB consecutive indices.  Inside a block the
 * EB sums run side by side (one per entry, each still summed in dimension
 * order), so a compiler can vectorise across entries without reordering any
 * single sum.  Within a block, and across blocks, entries are compared in
 * increasing index with a strict '>', so the lowest index among equal maxima
 * is kept. */
#define EB 8

typedef struct { double sim; int64_t idx; } best_t;

static void search_range(const float *db, int64_t lo, int64_t hi, const float *q, int d,
                         best_t *best)
{
    float xt[512 * EB];          /* d <= 512: transposed block, xt[t*EB + e] */
    double acc[EB];
    double bs = -INFINITY;
    int64_t bi = -1;
    for (int64_t base = lo; base < hi; base += EB) {
        int m = (int)((hi - base) < EB ? (hi - base) : EB);
        for (int e = 0; e < EB; ++e)
            for (int t = 0; t < d; ++t)
                xt[t * EB + e] = e < m ? db[(base + e) * d + t] : 0.0f;
        for (int e = 0; e < EB; ++e) acc[e] = 0.0;
        for (int t = 0; t < d; ++t) {
            const double qt = (double)q[t];
            for (int e = 0; e < EB; ++e) acc[e] += qt * (double)xt[t * EB + e];
        }
        for (int e = 0; e < m; ++e)
            if (acc[e] > bs) { bs = acc[e]; bi = base + e; }
    }
    best->sim = bs;
    best->idx = bi;
}

/* Exhaustive search: out_idx[j] = min{ i : sim(j,i) = max_i' sim(j,i') },
 * out_sim[j] = that maximum.  Parallel over (query, entry range) work items;
 * the per-range winners are merged in range order with a strict '>'.
 * nthreads <= 0 uses the OpenMP default. */
int hno_search(const float *db, int64_t n, const float *q, int64_t nq, int d,
               int64_t *out_idx, double *out_sim, int nthreads)
{
    if (n < 1 || nq < 0 || d < 1 || d > 512) return HNO_BAD_ARG;
    if (nq == 0) return HNO_OK;
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    /* enough entry ranges that nq * nr work items keep every thread busy */
    int64_t nr = 1;
    while (nq * nr < 4 * (int64_t)nt && n / (nr * 2) >= 4096) nr *= 2;
    best_t *part = (best_t *)malloc(sizeof(best_t) * (size_t)(nq * nr));
    if (!part) return HNO_BAD_ARG;
    const int64_t items = nq * nr;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t w = 0; w < items; ++w) {
        int64_t j = w / nr, r = w % nr;
        int64_t lo = n * r / nr, hi = n * (r + 1) / nr;
        search_range(db, lo, hi, q + j * d, d, &part[w]);
    }
    for (int64_t j = 0; j < nq; ++j) {
        double bs = -INFINITY;
        int64_t bi = -1;
        for (int64_t r = 0; r < nr; ++r)
            if (part[j * nr + r].sim > bs) { bs = part[j * nr + r].sim; bi = part[j * nr + r].idx; }
        out_idx[j] = bi;
        out_sim[j] = bs;
    }
    free(part);
    return HNO_OK;
}

/* Exhaustive top-k per query: the k pairs (sim, idx) largest in the order
 * sim descending, idx ascending.  Insertion into a sorted list of length k. */
int hno_search_topk(const float *db, int64_t n, const float *q, int64_t nq, int d, int topk,
                    int64_t *out_idx, double *out_sim, int nthreads)
{
    if (n < 1 || nq < 0 || d < 1 || topk < 1 || topk > n) return HNO_BAD_ARG;
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t j = 0; j < nq; ++j) {
        double *s = out_sim + j * topk;
        int64_t *ix = out_idx + j * topk;
        int filled = 0;
        for (int64_t i = 0; i < n; ++i) {
            double v = hno_dot(q + j * d, db + i * d, d);
            if (filled == topk && !(v > s[topk - 1])) continue;   /* equal: larger index loses */
            int p = filled < topk ? filled++ : topk - 1;
            while (p > 0 && v > s[p - 1]) { s[p] = s[p - 1]; ix[p] = ix[p - 1]; --p; }
            s[p] = v;
            ix[p] = i;
        }
    }
    return HNO_OK;
}

/* --------------------------------------------------- bound-based search (§3.3) */
/* Per query, from Eq. 2 and Eq. 3: <q, x_i> = s_i + <q_minor, x_i,minor> with
 * s_i = dot_K(q, x_i), and <q_minor, x_i,minor> <= bound_i, so an entry whose
 * s_i + bound_i lies below the full score of an entry already evaluated cannot be
 * the nearest neighbour, and evaluating every other entry in full gives the
 * exhaustive answer (Theorem 1).  The first full score is taken from the entry of
 * largest s_i (lowest index on ties), the natural choice the search of §3.3 makes;
 * every other entry is then tested against the best full score so far, in index
 * order, and evaluated only when its bound reaches it.
 * Readings (the paper is silent or literal-but-different on these):
 *   - bound_i: with literal_bound != 0 it is alpha, as printed in Eq. 3; otherwise
 *     it is |q_minor| |x_i,minor| (binary64 norms of the stored values) + 1e-12,
 *     Cauchy-Schwarz on the stored values plus a margin for binary64 rounding,
 *     because binary32 storage moves the norms off sqrt(alpha) by O(2^-24).
 *   - the skip is strict ('<' instead of the printed '<=') and equal full scores
 *     go to the lower index, so the result is the lowest index among the maxima
 *     (the printed '<=' with a strict-'>' update returns the first evaluated entry
 *     on an exact tie instead).
 * Because the full score continues the prefix sum in dimension order, it equals
 * hno_dot(q, x_i) bit for bit.  *n_full counts the full evaluations after the
 * first (the paper's Phase2%). */
int hno_two_phase(const float *db, int64_t n, const float *q, int64_t nq, int d, int k,
                  double alpha, int literal_bound, int64_t *out_idx, double *out_sim,
                  int64_t *n_full)
{
    if (n < 1 || nq < 0 || d < 2 || k < 1 || k >= d) return HNO_BAD_ARG;
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    double *xmin = (double *)malloc(sizeof(double) * (size_t)n);
    if (!s || !xmin) { free(s); free(xmin); return HNO_BAD_ARG; }
    for (int64_t i = 0; i < n; ++i) xmin[i] = sqrt(dot_range(db + i * d, db + i * d, k, d, 0.0));
    int64_t total_full = 0;
    for (int64_t j = 0; j < nq; ++j) {
        const float *qq = q + j * d;
        const double qmin = sqrt(dot_range(qq, qq, k, d, 0.0));
        /* Phase 1 */
        int64_t b = 0;
        for (int64_t i = 0; i < n; ++i) {
            s[i] = dot_range(qq, db + i * d, 0, k, 0.0);
            if (s[i] > s[b]) b = i;
        }
        double s_best = dot_range(qq, db + b * d, k, d, s[b]);
        int64_t best_idx = b;
        /* Phase 2 */
        for (int64_t i = 0; i < n; ++i) {
            if (i == b) continue;
            const double bound = literal_bound ? alpha : qmin * xmin[i] + 1e-12;
            if (literal_bound ? (s[i] + bound <= s_best) : (s[i] + bound < s_best)) continue;
            ++total_full;
            const double c = dot_range(qq, db + i * d, k, d, s[i]);
            if (literal_bound ? (c > s_best) : (c > s_best || (c == s_best && i < best_idx))) {
                s_best = c;
                best_idx = i;
            }
        }
        out_idx[j] = best_idx;
        out_sim[j] = s_best;
    }
    if (n_full) *n_full = total_full;
    free(s);
    free(xmin);
    return HNO_OK;
}
