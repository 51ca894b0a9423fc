"""The slack of the FP16-row rescore filter, checked on the CPU in numpy against binary64.

The filter bounds a survivor's similarity by RU(dot + e16), where dot is the FP32 sum of
q_d * fp16(x_d) and e16 = RU(|q| RU(RU(|x|max c1) + c2)), c1 = 4.96e-4, c2 = 3.4e-7.  This
test simulates the kernel's arithmetic (the rows rounded to FP16 with ties to even, FP32
products and sums in the lane-private order, four partial sums, and in the warp order,
4 products a lane then a butterfly) and checks that the result plus the slack never falls
below the binary64 dot of the unrounded row, on random, adversarial (all coordinates near the
FP16 subnormal range, alternating signs, one dominant coordinate) and aligned (q = x) cases.
It also checks that the slack is not loose by orders of magnitude, which would make the
filter useless (the observed error reaches a sizable fraction of it)."""
import numpy as np

C1 = np.float32(4.96e-4)
C2 = np.float32(3.4e-7)


def ru(x):
    """Round a float64 value up to float32."""
    f = np.float32(x)
    return f if np.float64(f) >= x else np.nextafter(f, np.float32(np.inf))


def slack(qn, xn_max):
    return ru(np.float64(qn) * np.float64(ru(np.float64(ru(np.float64(xn_max) * np.float64(C1))) + np.float64(C2))))


def dot_lane_private(q, x16):
    """Four FP32 partial sums over 16 groups of 8 coordinates, as in the one-per-lane path."""
    a = [np.float32(0)] * 4
    xf = x16.astype(np.float32)
    for i in range(16):
        b = 8 * i
        for t in range(4):
            c = b + 2 * t
            # fmaf(q[c], x[c], fmaf(q[c+1], x[c+1], a)): exact products (at most 35 bits), one
            # rounding per fused multiply-add
            inner = np.float32(np.float64(q[c + 1]) * np.float64(xf[c + 1]) + np.float64(a[t]))
            a[t] = np.float32(np.float64(q[c]) * np.float64(xf[c]) + np.float64(inner))
    return np.float32(np.float32(a[0] + a[1]) + np.float32(a[2] + a[3]))


def dot_warp(q, x16):
    """Lane l: q[4l..4l+3] . x[4l..4l+3] nested as fma(q0,x0, fma(q1,x1, fma(q2,x2, q3*x3))), then
    the xor butterfly over 32 lanes (every lane ends with the same sum)."""
    xf = x16.astype(np.float32)
    p = np.empty(32, np.float32)
    for l in range(32):
        c = 4 * l
        v = np.float32(q[c + 3] * xf[c + 3])
        v = np.float32(np.float64(q[c + 2]) * np.float64(xf[c + 2]) + np.float64(v))
        v = np.float32(np.float64(q[c + 1]) * np.float64(xf[c + 1]) + np.float64(v))
        v = np.float32(np.float64(q[c]) * np.float64(xf[c]) + np.float64(v))
        p[l] = v
    for o in (16, 8, 4, 2, 1):
        p = (p + p[np.arange(32) ^ o]).astype(np.float32)
    return p[0]


def cases(rng):
    for _ in range(300):
        q = rng.standard_normal(128)
        x = rng.standard_normal(128)
        yield q / np.linalg.norm(q), x / np.linalg.norm(x)
    # coordinates near and below the FP16 normal range (2^-14), alternating signs
    for s in (2.0 ** -13, 2.0 ** -15, 2.0 ** -20):
        q = np.full(128, 1 / np.sqrt(128))
        x = np.where(np.arange(128) % 2 == 0, 1.0, -1.0) * s * (1 + rng.random(128))
        x[0] = np.sqrt(max(0.0, 1 - np.sum(x[1:] ** 2)))
        yield q, x
    # one dominant coordinate, the rest tiny
    x = np.full(128, 1e-5)
    x[7] = 1.0
    x /= np.linalg.norm(x)
    yield x.copy(), x
    # aligned: the largest similarities, where the filter decides ties
    for _ in range(50):
        x = rng.standard_normal(128)
        x /= np.linalg.norm(x)
        yield x.copy(), x


def test_fp16_row_bound_holds():
    rng = np.random.default_rng(2026)
    worst = 0.0
    for q, x in cases(rng):
        q = q.astype(np.float32)
        x = x.astype(np.float32)
        exact = float(np.dot(q.astype(np.float64), x.astype(np.float64)))
        x16 = x.astype(np.float16)
        qn = ru(np.sqrt(np.sum(q.astype(np.float64) ** 2)))
        xn = ru(np.sqrt(np.sum(x.astype(np.float64) ** 2)))
        e = slack(qn, xn)
        for d in (dot_lane_private(q, x16), dot_warp(q, x16)):
            ub = ru(np.float64(d) + np.float64(e))
            assert np.float64(ub) >= exact, (exact, float(d), float(e))
            worst = max(worst, abs(float(d) - exact) / float(e))
    # the slack is tight enough to matter: observed error is a real fraction of it
    assert 0.05 < worst <= 1.0, worst


def test_slack_constants_cover_their_terms():
    """c1 >= 2^-11 + gamma_128 (1 + 2^-11) + 1e-12 and c2 >= 2^-25 sqrt(128), in binary64."""
    u = 2.0 ** -24
    gamma = 128 * u / (1 - 128 * u)
    assert float(C1) >= 2.0 ** -11 + gamma * (1 + 2.0 ** -11) + 1e-12
    assert float(C2) >= 2.0 ** -25 * np.sqrt(128)
