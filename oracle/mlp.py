"""Binary64 oracle of the learned block proposal -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module; the CUDA library never calls it.

The proposal is the extension that seeds the threshold of Algorithm 1 (§3.3):
an MLP maps a query's major prefix (the K-dim part of Eq. 1) to scores over
database blocks; the blocks it ranks highest are scored first to obtain a good
threshold.  The paper has no such network; this oracle fixes the arithmetic
the GPU kernels must reproduce:

    a1 = W1 x + b1,  h1 = gelu(a1)          W1: (H1, K)
    a2 = W2 h1 + b2, h2 = gelu(a2)          W2: (H2, H1)
    z  = W3 h2 + b3                         W3: (C, H2)
    loss = mean_j [ logsumexp(z_j) - z_j[y_j] ]
    gelu(a) = a * Phi(a) = 0.5 a (1 + erf(a / sqrt 2))     (exact GELU)

with the analytic gradients of that loss, and one Adam step
    m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
    p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
Parameters are kept as a dict of float64 arrays.  Inference runs each layer on
BF16-rounded operands (round to nearest even) with the products summed exactly
here (binary64) and in FP32 on the GPU: `linear_bf16`.  Tensor-core training does
the same to every operand of its contractions: `loss_and_grads_bf16`.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

_SQRT2 = math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)

PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / _SQRT2))


def gelu_grad(a):
    """d/da [a Phi(a)] = Phi(a) + a phi(a)."""
    return 0.5 * (1.0 + erf(a / _SQRT2)) + a * _INV_SQRT_2PI * np.exp(-0.5 * a * a)


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 value, ties to even (the binary32 value's upper 16 bits
    after adding half of the dropped 16 bits' weight, plus one more when the kept low bit is
    odd), returned as float64.  Finite inputs only."""
    u = np.asarray(a, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def linear_bf16(x, w, b=None, act: int = 0) -> np.ndarray:
    """One layer of the proposal's inference as its definition reads, in binary64:
    act(bf16(x) @ bf16(w).T + b), act 0 none, 1 the exact GELU.  x (m, k), w (n, k)."""
    z = bf16_round(x) @ bf16_round(w).T
    if b is not None:
        z = z + np.asarray(b, np.float64)
    return gelu(z) if act == 1 else z


def init_params(dims, seed: int) -> dict:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    k, h1, h2, c = dims
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((h1, k)) * math.sqrt(2.0 / k), "b1": np.zeros(h1),
        "W2": rng.standard_normal((h2, h1)) * math.sqrt(2.0 / h1), "b2": np.zeros(h2),
        "W3": rng.standard_normal((c, h2)) * math.sqrt(2.0 / h2), "b3": np.zeros(c),
    }


def forward(p: dict, x: np.ndarray):
    x = np.asarray(x, np.float64)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(a2)
    z = h2 @ p["W3"].T + p["b3"]
    return z, (x, a1, h1, a2, h2)


def loss_and_grads(p: dict, x: np.ndarray, y: np.ndarray):
    """Mean softmax cross-entropy over the batch and its gradient for every parameter."""
    z, (x, a1, h1, a2, h2) = forward(p, x)
    b = z.shape[0]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    s = e.sum(axis=1, keepdims=True)
    lse = zmax[:, 0] + np.log(s[:, 0])
    loss = float(np.mean(lse - z[np.arange(b), y]))
    dz = e / s
    dz[np.arange(b), y] -= 1.0
    dz /= b
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = dz @ p["W3"]
    da2 = dh2 * gelu_grad(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * gelu_grad(a1)
    g["W1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    return loss, g


def loss_and_grads_bf16(p: dict, x: np.ndarray, y: np.ndarray, rnd=bf16_round):
    """`loss_and_grads` as the tensor-core training computes it: every operand of the six
    training contractions (the three layer products, the two back-propagated activations and
    the three weight gradients) rounded to BF16 by `rnd`, the products then summed exactly
    (binary64) and every other step (bias, GELU, softmax, bias gradients) exact.  With `rnd`
    the identity this is `loss_and_grads` term for term."""
    x = np.asarray(x, np.float64)
    w1, w2, w3 = rnd(p["W1"]), rnd(p["W2"]), rnd(p["W3"])
    xr = rnd(x)
    a1 = xr @ w1.T + p["b1"]
    h1 = gelu(a1)
    h1r = rnd(h1)
    a2 = h1r @ w2.T + p["b2"]
    h2 = gelu(a2)
    h2r = rnd(h2)
    z = h2r @ w3.T + p["b3"]
    b = z.shape[0]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    s = e.sum(axis=1, keepdims=True)
    lse = zmax[:, 0] + np.log(s[:, 0])
    loss = float(np.mean(lse - z[np.arange(b), y]))
    dz = e / s
    dz[np.arange(b), y] -= 1.0
    dz /= b
    dzr = rnd(dz)
    g = {"W3": dzr.T @ h2r, "b3": dz.sum(axis=0)}
    da2 = (dzr @ w3) * gelu_grad(a2)
    da2r = rnd(da2)
    g["W2"] = da2r.T @ h1r
    g["b2"] = da2.sum(axis=0)
    da1 = (da2r @ w2) * gelu_grad(a1)
    g["W1"] = rnd(da1).T @ xr
    g["b1"] = da1.sum(axis=0)
    return loss, g


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8) -> None:
    for k in PARAM_ORDER:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def topk(z: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k largest scores per row, by (score desc, index asc)."""
    order = np.lexsort((np.broadcast_to(np.arange(z.shape[1]), z.shape), -z), axis=1)
    return order[:, :k]


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([p[k].ravel() for k in PARAM_ORDER])


def unflatten(flat: np.ndarray, dims) -> dict:
    k, h1, h2, c = dims
    shapes = {"W1": (h1, k), "b1": (h1,), "W2": (h2, h1), "b2": (h2,), "W3": (c, h2), "b3": (c,)}
    out, o = {}, 0
    for name in PARAM_ORDER:
        n = int(np.prod(shapes[name]))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shapes[name])
        o += n
    return out


def n_params(dims) -> int:
    k, h1, h2, c = dims
    return h1 * k + h1 + h2 * h1 + h2 + c * h2 + c
