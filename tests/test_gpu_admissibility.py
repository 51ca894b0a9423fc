"""Admissibility of the reduced-precision prefix bound on the GPU (ext. 1).

The search drops entry i for query q only when  s~_qi + E_q < T_q, where s~ is the
prefix score as the kernels compute it (BF16 or FP8 operands, tensor-core or CUDA-core
FP32 accumulation) and E_q the query's slack.  Exactness needs

    <q, x_i>  <=  s~_qi + E_q          for every pair (Eq. 2 and Eq. 3),

with <.,.> the oracle's binary64 similarity.  hn_prefix_scores returns s~ from the
search's own arithmetic (path 0: the tcgen05 scan, path 1: the FMA chain of the
survivor extraction and the stream scan) and E_q, and these tests check the
inequality pair by pair on inputs built to make the rounding as bad as it gets:

* alpha = 0, so the minor part is zero and E_q is the scan's rounding term alone;
* components placed on BF16 and on e4m3 rounding midpoints (largest rounding error,
  with the errors of a vector all of one sign, so they add up);
* all components of one magnitude (the largest |x|_inf / |x| an HN prefix allows
  bounds the accumulation error from above);
* sign-alternating columns: partial sums far larger than the result;
* BF16-exact components spread over 13 binades: no rounding residual, so the
  accumulation term is all of E_q.

Besides the pass/fail check, each case reports the largest observed error as a
fraction of the rounding term (printed; run pytest with -s to see it).
"""
import numpy as np
import pytest

import hn_synth
import oracle
from tests._gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


def _midpoint_rows(rng, n, k, fmt):
    """Rows with k - 1 components on rounding midpoints of `fmt` and one filler column
    that brings the norm to 1 (alpha = 0: no minor part).

    bf16: midpoints (m + 1/2) 2^e of 8-bit significands m in [128, 256), scaled by one
    power of two per row (which keeps them midpoints) so that they carry between 1/4
    and all of the energy.  e4m3: midpoints of the e4m3 grid relative to the row's own
    power-of-two scale s, with component 0 at 448 s (so s is the scale the FP8 index
    picks) and the filler no larger than 448 s.  Random signs.  Rows whose float32
    norm misses 1 by more than the index's tolerance are dropped."""
    out = []
    while sum(len(o) for o in out) < n:
        m = n * 2
        if fmt == "bf16":
            v = (rng.integers(128, 256, size=(m, k - 1)) + 0.5) * np.exp2(rng.integers(-3, 1, size=(m, k - 1)))
            s2 = np.sum(v ** 2, axis=1)
            sc = np.exp2(-np.ceil(np.log2(s2) / 2))                 # s2 * sc^2 in (1/4, 1]
            ok = np.ones(m, bool)
        else:
            e = rng.integers(3, 6, size=(m, k - 1))                 # binades 64.., 128.., 256..
            mant = rng.integers(8, 16, size=(m, k - 1)) + 0.5
            mant = np.where(e == 5, np.minimum(mant, 13.5), mant)   # 448 is the largest e4m3 value
            v = mant * np.exp2(e.astype(np.float64))
            v[:, 0] = 448.0
            s2 = np.sum(v ** 2, axis=1)
            sc = np.exp2(-np.ceil(np.log2(s2) / 2))
            ok = (1.0 - s2 * sc ** 2) <= (448.0 * sc) ** 2          # filler no larger than 448 s
        v = v * sc[:, None] * rng.choice([-1.0, 1.0], size=v.shape)
        x = np.zeros((m, 128), np.float32)
        x[:, :k - 1] = v.astype(np.float32)                         # exact: few significant bits
        rest = 1.0 - np.sum(x[:, :k - 1].astype(np.float64) ** 2, axis=1)
        x[:, k - 1] = np.sqrt(np.maximum(rest, 0.0)).astype(np.float32)
        n2 = np.sum(x.astype(np.float64) ** 2, axis=1)
        out.append(x[ok & (np.abs(n2 - 1.0) <= 100 * 2.0 ** -24)])
    return np.concatenate(out)[:n]


def _bf16(v):
    """Round float64 values to the nearest BF16 (8 significant bits), ties to even."""
    m, e = np.frexp(v)
    return np.ldexp(np.round(m * 256.0), e - 8)


def _bf16_exact_rows(rng, n, k):
    """Rows whose k components are BF16 numbers spread over the binades 2^-1 .. 2^-13
    (products of two such numbers span ~2^-26 .. 2^-2, so an FP32 sum of them rounds),
    with squared norm 1 within the index's tolerance: k - 2 random components, one
    BF16 component close to the remaining energy less 1e-3, and a last small BF16
    component (~0.03, where BF16 rounding moves the square by < 4e-6) for the rest.
    Their BF16 rounding residuals are zero, so the slack is the accumulation term alone."""
    out = []
    while sum(len(o) for o in out) < n:
        m = 4 * n
        v = _bf16(rng.uniform(0.5, 1.0, size=(m, k - 2)) * np.exp2(-rng.integers(1, 14, size=(m, k - 2))))
        s2 = np.sum(v ** 2, axis=1)
        v = v * np.exp2(-np.ceil(np.log2(s2 / 0.9) / 2))[:, None]     # sum of squares in (0.225, 0.9]
        s2 = np.sum(v ** 2, axis=1)
        a = _bf16(np.sqrt(np.maximum(1.0 - s2 - 1e-3, 0.0)))
        c = _bf16(np.sqrt(np.maximum(1.0 - s2 - a ** 2, 0.0)))
        x = np.zeros((m, 128), np.float32)
        x[:, :k - 2], x[:, k - 2], x[:, k - 1] = v, a, c
        x[:, :k] *= rng.choice([-1.0, 1.0], size=(m, k))
        n2 = np.sum(x.astype(np.float64) ** 2, axis=1)
        assert np.array_equal(_bf16(x[:, :k].astype(np.float64)), x[:, :k].astype(np.float64))
        out.append(x[np.abs(n2 - 1.0) <= 100 * 2.0 ** -24])
    return np.concatenate(out)[:n]


def _adversarial(seed, n, k, kind):
    rng = np.random.default_rng(seed)
    if kind in ("bf16_mid", "e4m3_mid"):
        return _midpoint_rows(rng, n, k, kind[:4])
    if kind == "bf16_exact":
        return _bf16_exact_rows(rng, n, k)
    if kind == "flat":
        # every component +-1/sqrt(k): the largest accumulation error an HN prefix allows
        rows = np.zeros((n, 128), np.float32)
        rows[:, :k] = (rng.choice([-1.0, 1.0], size=(n, k)) / np.sqrt(k)).astype(np.float32)
        n2 = np.sum(rows.astype(np.float64) ** 2, axis=1)
        return rows[np.abs(n2 - 1.0) <= 100 * 2.0 ** -24]
    if kind == "alternate":
        # BF16-midpoint magnitudes, signs alternating by column (entries) or constant
        # (queries, via the caller): partial sums far above the result
        rows = np.abs(_midpoint_rows(rng, n, k, "bf16"))
        rows[:, :k] *= np.where(np.arange(k) % 2 == 0, 1.0, -1.0).astype(np.float32)
        return rows
    raise ValueError(kind)


def _check(hn, db, q, k, alpha, prefix, path, label):
    with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
        s, eps = ix.prefix_scores(to_dev(q), path)
    s = s.cpu().numpy().astype(np.float64)
    eps = eps.cpu().numpy().astype(np.float64)
    exact = np.stack([oracle.sims(db, qq) for qq in q])          # binary64, the oracle's order
    gap = exact - s                                              # must be <= eps row-wise
    assert np.all(np.isfinite(s))
    worst = np.max(gap / eps[:, None])
    bad = np.argwhere(gap > eps[:, None])
    assert bad.size == 0, f"{label}: bound violated at {bad[:5]} (gap {gap[tuple(bad[0])]}, eps {eps[bad[0][0]]})"
    print(f"\n{label}: largest (exact - prefix score) / E_q = {worst:.4f} over {gap.size} pairs")
    return worst


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("prefix", [1, 2])
@pytest.mark.parametrize("kind", ["bf16_mid", "e4m3_mid", "flat", "alternate"])
@pytest.mark.parametrize("k", [16, 64, 9])
def test_scan_error_term_is_admissible(hn, path, prefix, kind, k):
    db = _adversarial(1000 + k, 3000, k, kind)
    q = _adversarial(2000 + k, 300, k, kind)
    if kind == "alternate":
        q = np.abs(q)   # same-sign queries against sign-alternating entries
    # queries that equal entries and their negations: largest |s| and exact ties
    q = np.concatenate([q, db[:40], -db[40:80]])
    worst = _check(hn, db, q, k, 0.0, prefix, path, f"K={k} {kind} prefix={prefix} path={path}")
    assert worst <= 1.0


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("k", [16, 64, 9])
def test_accumulation_term_alone(hn, path, k):
    """BF16-exact inputs (no rounding residual): E_q is the accumulation term
    (kp + 2) 2^-20 |q^| max|x^| plus 1e-12, and every pair's error stays below it."""
    db = _adversarial(3000 + k, 3000, k, "bf16_exact")
    q = np.concatenate([_adversarial(4000 + k, 300, k, "bf16_exact"), db[:40], -db[40:80]])
    worst = _check(hn, db, q, k, 0.0, 1, path, f"K={k} bf16_exact prefix=1 path={path}")
    assert worst <= 1.0


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("prefix", [1, 2])
def test_full_bound_on_clustered_data(hn, path, prefix):
    """The whole inequality, minor bound included, on the clustered workload (K = 16,
    alpha = 1/8): the prefix score plus E_q bounds the full similarity of every pair."""
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(6000, 200, 600, seed=91)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    worst = _check(hn, db, q, k, alpha, prefix, path, f"clustered K=16 alpha=1/8 prefix={prefix} path={path}")
    assert worst <= 1.0


def test_prefix_scores_rejects_bad_args(hn):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(300, 4, 30, seed=92)
    db = oracle.normalize(w.db_raw, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=0) as ix:   # FP32 prefix: no tensor-core scan
        with pytest.raises(hn.HNError):
            ix.prefix_scores(to_dev(db[:4]), 0)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        with pytest.raises(hn.HNError):
            ix.prefix_scores(to_dev(db[:4]), 2)
