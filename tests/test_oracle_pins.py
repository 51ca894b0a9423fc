"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: closed-form
values computed at 60 significant digits (mpmath), exact integer arithmetic,
an independent float64 matrix product, the identities under Eq. 1, the bound
of Eq. 3, Theorem 1 (two-phase search = exhaustive search), the tie rule of
Theorem 2, and the alpha = 0 case of §6.2.
"""
import fractions
import itertools

import mpmath
import numpy as np
import pytest

import hn_synth
import oracle

mpmath.mp.dps = 60
U32 = 2.0 ** -24


def _exact_hn_row(f, k, alpha):
    """Eq. 1 in 60-digit arithmetic, rounded once to float32 via the nearest double."""
    alpha = mpmath.mpf(fractions.Fraction(alpha).numerator) / fractions.Fraction(alpha).denominator
    maj = mpmath.sqrt(mpmath.fsum(mpmath.mpf(float(v)) ** 2 for v in f[:k]))
    mnr = mpmath.sqrt(mpmath.fsum(mpmath.mpf(float(v)) ** 2 for v in f[k:]))
    out = []
    for t, v in enumerate(f):
        if t < k:
            out.append(mpmath.sqrt(1 - alpha) * mpmath.mpf(float(v)) / maj)
        else:
            out.append(mpmath.mpf(0) if alpha == 0 else mpmath.sqrt(alpha) * mpmath.mpf(float(v)) / mnr)
    return out


# ---------------------------------------------------------------- Eq. 1
@pytest.mark.parametrize("k,alpha", [(8, 1 / 32), (16, 1 / 8), (16, 0.25), (1, 0.5), (127, 1 / 3)])
def test_normalize_unit_basis(k, alpha):
    """f = e_0 + e_K: major = sqrt(1-a) e_0, minor = sqrt(a) e_K exactly (Eq. 1)."""
    f = np.zeros((1, 128), np.float32)
    f[0, 0] = 1.0
    f[0, k] = 1.0
    out = oracle.normalize(f, k, alpha)[0]
    want = np.zeros(128, np.float32)
    want[0] = np.float32(np.sqrt(1.0 - alpha))
    want[k] = np.float32(np.sqrt(alpha))
    assert np.array_equal(out, want)


@pytest.mark.parametrize("k,alpha", [(8, 1 / 32), (16, 1 / 8), (16, 0.0), (16, 0.25), (3, 0.9)])
def test_normalize_matches_60_digit_definition(k, alpha):
    """Every output is within one float32 ulp of Eq. 1 evaluated at 60 digits."""
    raw = hn_synth.make_workload(6, 0, 3, seed=11).db_raw
    raw[1, :k] *= 1e-30          # tiny major, still representable
    raw[2, k:] *= 3e30           # huge minor
    out = oracle.normalize(raw, k, alpha)
    for r in range(raw.shape[0]):
        ex = _exact_hn_row(raw[r], k, alpha)
        for t in range(128):
            e = ex[t]
            got = mpmath.mpf(float(out[r, t]))
            ulp = np.spacing(np.float32(abs(float(e)))) if e != 0 else 0.0
            assert abs(got - e) <= mpmath.mpf(float(ulp)), (r, t, got, e)


def test_normalize_pythagorean_closed_form():
    """|(3,4)| = 5 and |(5,12)| = 13: outputs are sqrt(1-a)*(0.6,0.8), sqrt(a)*(5,12)/13."""
    k, alpha = 2, 0.25
    f = np.zeros((1, 128), np.float32)
    f[0, :2] = [3, 4]
    f[0, 2] = 5
    f[0, 3] = 12
    out = oracle.normalize(f, k, alpha)[0]
    ra, rb = np.sqrt(0.75), np.sqrt(0.25)
    assert out[0] == np.float32(3 * (ra / 5.0)) and out[1] == np.float32(4 * (ra / 5.0))
    assert out[2] == np.float32(5 * (rb / 13.0)) and out[3] == np.float32(12 * (rb / 13.0))
    assert abs(float(out[0]) - 0.6 * np.sqrt(0.75)) < 1e-7
    assert np.all(out[4:] == 0)


def test_normalize_power_of_two_scale_invariance():
    """Scaling a part by 2^p changes neither the real result nor its rounding."""
    raw = hn_synth.make_workload(64, 0, 8, seed=5).db_raw
    a = oracle.normalize(raw, 16, 1 / 8)
    s = raw.copy()
    s[:, :16] *= np.float32(2.0 ** 37)
    s[:, 16:] *= np.float32(2.0 ** -41)
    b = oracle.normalize(s, 16, 1 / 8)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("k,alpha", [(8, 1 / 32), (16, 1 / 8), (16, 0.25), (64, 0.5)])
def test_normalize_norm_identities(k, alpha):
    """|major|^2 = 1-a, |minor|^2 = a, total 1 (below Eq. 1), up to float32 rounding."""
    raw = hn_synth.make_workload(2000, 0, 100, seed=3).db_raw
    x = oracle.normalize(raw, k, alpha)
    maj2, min2 = oracle.part_norms2(x, k)
    # each stored coordinate carries a relative error <= 2^-24 (one rounding of an exact-ish
    # binary64 value), so a squared norm moves by at most about 2*2^-24 relative
    assert np.max(np.abs(maj2 - (1 - alpha))) <= 3 * U32 * (1 - alpha)
    assert np.max(np.abs(min2 - alpha)) <= 3 * U32 * alpha + 1e-300
    assert np.max(np.abs(maj2 + min2 - 1)) <= 3 * U32


def test_normalize_alpha_zero_minor_is_zero():
    raw = hn_synth.make_workload(50, 0, 5, seed=2).db_raw
    x = oracle.normalize(raw, 16, 0.0)
    assert np.all(x[:, 16:] == 0)
    raw[:, 16:] = 0  # a zero minor is fine when alpha = 0
    oracle.normalize(raw, 16, 0.0)


def test_normalize_zero_norm_rejected():
    raw = hn_synth.make_workload(4, 0, 2, seed=2).db_raw
    raw[2, :8] = 0
    with pytest.raises(oracle.OracleError) as e:
        oracle.normalize(raw, 8, 1 / 32)
    assert e.value.status == oracle.ZERO_NORM and e.value.row == 2
    raw = hn_synth.make_workload(4, 0, 2, seed=2).db_raw
    raw[1, 8:] = 0
    with pytest.raises(oracle.OracleError) as e:
        oracle.normalize(raw, 8, 1 / 32)
    assert e.value.row == 1


# ---------------------------------------------------------------- Eq. 2 / dot
def test_dot_exact_small_integers():
    rng = np.random.default_rng(0)
    for _ in range(200):
        a = rng.integers(-1000, 1000, 128)
        b = rng.integers(-1000, 1000, 128)
        assert oracle.dot(a.astype(np.float32), b.astype(np.float32)) == float(int(np.dot(a, b)))


def test_dot_sequential_order():
    """(2^60 + 1) - 2^60 is 0 in sequential binary64, 1 in exact arithmetic."""
    a = np.ones(128, np.float32)
    b = np.zeros(128, np.float32)
    b[0], b[1], b[2] = 2.0 ** 60, 1.0, -(2.0 ** 60)
    assert oracle.dot(a, b) == 0.0
    b[0], b[1], b[2] = 2.0 ** 60, -(2.0 ** 60), 1.0
    assert oracle.dot(a, b) == 1.0


def test_sims_match_float64_matmul():
    w = hn_synth.make_workload(500, 3, 50, seed=9)
    db = oracle.normalize(w.db_raw, 16, 1 / 8)
    q = oracle.normalize(w.q_raw, 16, 1 / 8)
    ref = db.astype(np.float64) @ q.astype(np.float64).T
    for j in range(3):
        assert np.max(np.abs(oracle.sims(db, q[j]) - ref[:, j])) < 1e-13


# ---------------------------------------------------------------- exhaustive search
def _rational_argmax(db_int, q_int):
    best, bi = None, -1
    for i, row in enumerate(db_int):
        s = sum(int(a) * int(b) for a, b in zip(row, q_int))
        if best is None or s > best:
            best, bi = s, i
    return bi, best


def test_search_exact_integers_with_ties():
    """Small-integer vectors: binary64 sums are exact, ties are common; lowest index wins."""
    rng = np.random.default_rng(1)
    db = rng.integers(-2, 3, (300, 128))
    db[200] = db[17]            # planted duplicates: 17 must win over 200
    db[250] = db[17]
    q = rng.integers(-2, 3, (40, 128))
    q[0] = db[17]
    idx, sim = oracle.search(db.astype(np.float32), q.astype(np.float32))
    for j in range(len(q)):
        bi, bs = _rational_argmax(db, q[j])
        assert idx[j] == bi and sim[j] == float(bs)
    assert idx[0] == 17


def test_search_matches_float64_matmul_on_hn_data():
    w = hn_synth.make_workload(3000, 200, 400, seed=4)
    db = oracle.normalize(w.db_raw, 8, 1 / 32)
    q = oracle.normalize(w.q_raw, 8, 1 / 32)
    idx, sim = oracle.search(db, q)
    ref = q.astype(np.float64) @ db.astype(np.float64).T
    top2 = np.sort(ref, axis=1)[:, -2:]
    am = np.argmax(ref, axis=1)
    assert np.max(np.abs(sim - ref.max(axis=1))) < 1e-12
    clear = (top2[:, 1] - top2[:, 0]) > 1e-12
    assert clear.sum() > 190
    assert np.array_equal(idx[clear], am[clear])


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_search_thread_count_invariant(threads):
    w = hn_synth.make_workload(20000, 7, 500, seed=6)
    db = oracle.normalize(w.db_raw, 16, 1 / 8)
    q = oracle.normalize(w.q_raw, 16, 1 / 8)
    i1, s1 = oracle.search(db, q, nthreads=1)
    i2, s2 = oracle.search(db, q, nthreads=threads)
    assert np.array_equal(i1, i2) and np.array_equal(s1, s2)


def test_search_edge_sizes():
    db = np.eye(128, dtype=np.float32)[:1]
    idx, sim = oracle.search(db, -db)
    assert idx[0] == 0 and sim[0] == -1.0
    db2 = np.stack([np.eye(128, dtype=np.float32)[0]] * 2)
    idx, _ = oracle.search(db2, db2[:1])
    assert idx[0] == 0
    idx, sim = oracle.search(db2, np.zeros((0, 128), np.float32))
    assert idx.shape == (0,)


def test_search_topk_matches_sorted_sims():
    w = hn_synth.make_workload(700, 5, 50, seed=8)
    db = oracle.normalize(w.db_raw, 16, 1 / 8)
    db[300] = db[12]
    q = oracle.normalize(w.q_raw, 16, 1 / 8)
    q[0] = db[12]
    ti, ts = oracle.search_topk(db, q, 5)
    for j in range(5):
        s = oracle.sims(db, q[j])
        order = sorted(range(len(s)), key=lambda i: (-s[i], i))[:5]
        assert list(ti[j]) == order
        assert np.array_equal(ts[j], s[order])
    assert ti[0, 0] == 12 and ti[0, 1] == 300
    i1, s1 = oracle.search(db, q)
    assert np.array_equal(ti[:, 0], i1) and np.array_equal(ts[:, 0], s1)


# ---------------------------------------------------------------- Eq. 3
@pytest.mark.parametrize("k,alpha", [(8, 1 / 32), (16, 1 / 8)])
def test_bound_eq3_every_pair(k, alpha):
    """<q,x> <= dot_K + |q_min||x_min| <= dot_K + a (1 + 3*2^-24) on every pair."""
    w = hn_synth.make_workload(2000, 300, 200, seed=12)
    db = oracle.normalize(w.db_raw, k, alpha).astype(np.float64)
    q = oracle.normalize(w.q_raw, k, alpha).astype(np.float64)
    full = q @ db.T
    dk = q[:, :k] @ db[:, :k].T
    mq = np.linalg.norm(q[:, k:], axis=1)
    mx = np.linalg.norm(db[:, k:], axis=1)
    assert np.all(full <= dk + np.outer(mq, mx) + 1e-13)
    assert np.all(np.outer(mq, mx) <= alpha * (1 + 3 * U32))
    assert np.all(full <= dk + alpha * (1 + 3 * U32) + 1e-13)


def test_bound_tight_when_minors_equal():
    """Eq. 3 is attained when the two minor parts are identical."""
    w = hn_synth.make_workload(2, 0, 2, seed=1)
    x = oracle.normalize(w.db_raw, 16, 1 / 8)
    y = x.copy()
    y[1, 16:] = y[0, 16:]
    full = oracle.dot(y[0], y[1])
    dk = oracle.dot(y[0, :16], y[1, :16])
    assert abs(full - (dk + 1 / 8)) < 4 * U32


# ---------------------------------------------------------------- Theorem 1 / 2
@pytest.mark.parametrize("k,alpha,seed", [(8, 1 / 32, 0), (16, 1 / 8, 1), (16, 0.25, 2), (4, 0.5, 3),
                                          (16, 0.0, 4)])
def test_two_phase_equals_exhaustive(k, alpha, seed):
    w = hn_synth.make_workload(4000, 300, 300, seed=seed)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    db[1000] = db[10]
    db[3000] = db[10]
    q[0] = db[10]
    i_bf, s_bf = oracle.search(db, q)
    i_tp, s_tp, nfull = oracle.two_phase(db, q, k, alpha)
    assert np.array_equal(i_bf, i_tp) and np.array_equal(s_bf, s_tp)
    assert i_bf[0] == 10
    if k >= 8 and alpha <= 1 / 8:
        assert nfull < 0.2 * 4000 * 300   # the paper's operating points prune most entries
    if alpha == 0:
        # §6.2: at alpha = 0 Phase 2 needs no dot product, except for the two planted exact
        # duplicates of entry 10 under query 0, which tie and must be compared by index
        assert nfull == 2
    il, sl, _ = oracle.two_phase(db, q, k, alpha, literal_bound=True)
    assert np.array_equal(sl, s_bf)  # the printed bound reaches the same maximum here


def test_two_phase_tie_reading():
    """Exact tie between entry 0 and a later entry b with a larger prefix score:
    the printed rule returns b, the lowest-index reading returns 0."""
    k = 2
    db = np.zeros((3, 8), np.float32)
    q = np.zeros((1, 8), np.float32)
    q[0, :4] = [1, 1, 1, 1]
    db[0, :4] = [1, 0, 1, 0]   # prefix 1, full 2
    db[1, :4] = [0, 0, 0, 1]   # prefix 0, full 1
    db[2, :4] = [1, 1, 0, 0]   # prefix 2, full 2  -> Phase-1 argmax b = 2
    i_bf, s_bf = oracle.search(db, q)
    assert i_bf[0] == 0 and s_bf[0] == 2.0
    i_tp, s_tp, _ = oracle.two_phase(db, q, k, alpha=2.0 / 3.0)
    assert i_tp[0] == 0
    il, sl, _ = oracle.two_phase(db, q, k, alpha=2.0 / 3.0, literal_bound=True)
    assert il[0] == 2 and sl[0] == 2.0


def test_alpha_zero_reduces_to_prefix_search():
    """alpha = 0: minors vanish, so exact 1-NN = argmax of the K-dim prefix product."""
    w = hn_synth.make_workload(5000, 100, 500, seed=21)
    db = oracle.normalize(w.db_raw, 16, 0.0)
    q = oracle.normalize(w.q_raw, 16, 0.0)
    idx, sim = oracle.search(db, q)
    ref = q[:, :16].astype(np.float64) @ db[:, :16].astype(np.float64).T
    assert np.array_equal(idx, np.argmax(ref, axis=1))
    assert np.max(np.abs(sim - ref.max(axis=1))) < 1e-13


def test_generator_deterministic_and_thread_free():
    a = hn_synth.make_workload(70000, 10, 100, seed=3)
    b = hn_synth.make_workload(70000, 10, 100, seed=3)
    assert np.array_equal(a.db_raw, b.db_raw) and np.array_equal(a.q_raw, b.q_raw)
    c = hn_synth.make_workload(70000, 10, 100, seed=4)
    assert not np.array_equal(a.db_raw[:10], c.db_raw[:10])
    # queries are drawn near their source entries
    d = np.linalg.norm(a.q_raw - a.db_raw[a.source_of], axis=1)
    assert np.all(d < 0.1 * np.sqrt(128) * 2)
