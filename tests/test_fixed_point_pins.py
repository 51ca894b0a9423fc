"""CPU pins of the arithmetic behind the int8 fixed-point prefix (§7, power-of-two
alpha and fixed-point HN).  They check facts of binary32/binary64 arithmetic and the
quantisation bound on their own, in numpy, independently of the CUDA code:

* accumulator encoding: the int32 bits 0x4B400000 + D read as the binary32 value
  1.5 * 2^23 + D exactly for |D| < 2^22, so comparing those floats compares D;
* integer threshold: with t, s powers of two, D >= ceil(tau / (t s)) holds exactly when
  t s D >= tau (real arithmetic), tau any binary32;
* quantisation bound: with codes RN(v / scale) on power-of-two scales,
  q.x <= t s (q^ . x^) + r(q) |x| + |q~| r(x) for HN-normalised vectors.
"""
import math

import numpy as np

import hn_synth
import oracle

BIAS = 0x4B400000  # bits of 1.5 * 2^23


def enc(d):
    return (np.int64(BIAS) + np.asarray(d, np.int64)).astype(np.int32).view(np.float32)


def test_accumulator_encoding_is_exact_and_monotone():
    d = np.concatenate([np.arange(-2000, 2001), np.array([-(1 << 22) + 1, (1 << 22) - 1, -258064, 258064,
                                                          -1032256, 1032256])])
    f = enc(d).astype(np.float64)
    assert np.array_equal(f, 1.5 * 2.0 ** 23 + d)            # exact value
    order = np.argsort(d, kind="stable")
    assert np.all(np.diff(f[order]) > 0)                      # strictly increasing in D
    assert np.all(f > 0)                                      # positive: float order = bit order
    # the largest |D| of a kp <= 64 int8 dot product fits: 64 * 127 * 127 < 2^22
    assert 64 * 127 * 127 < (1 << 22)


def i8_threshold(tau, inv):
    """Threshold on the encoded accumulator: 1.5 * 2^23 + ceil(tau * inv), clamped to |.| < 2^22."""
    if tau == -math.inf:
        return -math.inf
    v = min(max(math.ceil(float(tau) * float(inv)), -4194303), 4194303)
    return np.float32(12582912.0 + v)


def test_integer_threshold_matches_the_real_test():
    rng = np.random.default_rng(7)
    for _ in range(4000):
        t = 2.0 ** int(rng.integers(-12, 2))
        s = 2.0 ** int(rng.integers(-9, -5))
        inv = 1.0 / (t * s)                       # a power of two
        tau = np.float32(rng.uniform(-1.2, 1.2))
        th = i8_threshold(tau, inv)
        for d in rng.integers(-300000, 300000, size=8):
            keep_int = enc(d) >= th
            keep_real = t * s * int(d) >= float(tau)   # products of powers of two: exact in binary64
            assert keep_int == keep_real, (t, s, tau, d)
    # tau = -inf keeps everything; a tau above every reachable score keeps nothing
    assert enc(-1032256) >= i8_threshold(-math.inf, 1.0)
    assert not enc(1032256) >= i8_threshold(np.float32(1e30), 2.0 ** 20)


def pow2_scale(amax):
    """Smallest power of two s (>= 2^-100) with amax / s <= 127, as frexp gives it; 1 for amax = 0."""
    if amax <= 0:
        return 1.0
    _, ex = math.frexp(amax / 127.0)
    return math.ldexp(1.0, max(ex, -100))


def codes(v, scale):
    c = np.rint(v.astype(np.float64) / scale)
    assert np.all(np.abs(c) <= 127)
    return c


def test_quantisation_bound_holds_on_hn_vectors():
    for k, alpha in [(8, 1 / 32), (16, 1 / 8), (16, 0.0), (32, 1 / 8), (64, 1 / 16)]:
        w = hn_synth.make_workload(3000, 300, 600, seed=61 + k, entry_noise=0.3, query_noise=0.2)
        db = oracle.normalize(w.db_raw, k, alpha)
        q = oracle.normalize(w.q_raw, k, alpha)
        xm = db[:, :k].astype(np.float64)
        qm = q[:, :k].astype(np.float64)
        s = pow2_scale(float(np.max(np.abs(db[:, :k]))))
        xc = codes(db[:, :k], s)
        xt = xc * s
        assert np.array_equal(xt.astype(np.float32).astype(np.float64), xt)      # dequantisation exact
        rx = np.sqrt(np.sum((xm - xt) ** 2, axis=1))
        xmaj = np.sqrt(np.sum(xm ** 2, axis=1))
        for j in range(q.shape[0]):
            t = pow2_scale(float(np.max(np.abs(q[j, :k]))))
            qc = codes(q[j, :k], t)
            qt = qc * t
            rq = math.sqrt(float(np.sum((qm[j] - qt) ** 2)))
            d = xc @ qc                                        # exact: integers below 2^53
            assert np.all(d == np.round(d)) and np.max(np.abs(d)) < (1 << 22)
            scan = t * s * d                                   # exact (powers of two)
            exact = xm @ qm[j]
            bound = scan + rq * np.max(xmaj) + math.sqrt(float(qt @ qt)) * np.max(rx)
            assert np.all(exact <= bound + 1e-12), (k, alpha, j)
            # and the bound is not vacuous: within a few code steps of the prefix dot product
            assert np.max(bound - exact) < 0.05


def test_quantisation_bound_is_tight_for_a_single_coordinate():
    # one coordinate carries the whole major norm: the code error is at most half a step
    v = np.zeros(16, np.float32)
    v[3] = np.float32(math.sqrt(1 - 1 / 8))
    s = pow2_scale(float(v[3]))
    c = codes(v, s)
    assert abs(float(v[3]) - c[3] * s) <= s / 2
    assert s <= 2 * float(v[3]) / 127
