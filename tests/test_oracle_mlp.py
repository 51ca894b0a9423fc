"""Pins of the binary64 MLP oracle (the learned block proposal).

The analytic gradient is checked against central finite differences of the
loss (independent of the backward formulas), the loss against closed forms,
GELU against its definition via math.erf, and Adam's first step against its
closed form (lr * sign(g))."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_definition_and_derivative():
    a = np.linspace(-6, 6, 121)
    want = np.array([0.5 * t * (1 + math.erf(t / math.sqrt(2))) for t in a])
    assert np.max(np.abs(mlp.gelu(a) - want)) < 1e-15
    h = 1e-6
    fd = (mlp.gelu(a + h) - mlp.gelu(a - h)) / (2 * h)
    assert np.max(np.abs(mlp.gelu_grad(a) - fd)) < 1e-8
    assert mlp.gelu(np.array([0.0]))[0] == 0.0 and abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


def test_loss_uniform_logits_is_log_classes():
    dims = (4, 6, 5, 7)
    p = mlp.init_params(dims, 0)
    for k in ("W3", "b3"):
        p[k][:] = 0.0
    x = np.random.default_rng(1).standard_normal((9, 4))
    y = np.arange(9) % 7
    loss, g = mlp.loss_and_grads(p, x, y)
    assert abs(loss - math.log(7)) < 1e-14
    # with W3 = 0 no gradient reaches the hidden layers
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_finite_differences(seed):
    dims = (5, 7, 6, 9)
    rng = np.random.default_rng(seed)
    p = mlp.init_params(dims, seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.3
    x = rng.standard_normal((6, 5))
    y = rng.integers(0, 9, 6)
    _, g = mlp.loss_and_grads(p, x, y)
    flat = mlp.flatten(p)
    gflat = mlp.flatten(g)
    h = 1e-6
    idx = rng.choice(flat.size, 60, replace=False)
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = mlp.loss_and_grads(mlp.unflatten(fp, dims), x, y)
        lm, _ = mlp.loss_and_grads(mlp.unflatten(fm, dims), x, y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_adam_first_step_is_lr_sign():
    dims = (3, 4, 4, 5)
    p = mlp.init_params(dims, 3)
    rng = np.random.default_rng(4)
    g = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    p0 = {k: v.copy() for k, v in p.items()}
    mlp.adam_step(p, g, m, v, t=1, lr=1e-3, eps=0.0)
    for k in p:
        assert np.allclose(p[k] - p0[k], -1e-3 * np.sign(g[k]), rtol=0, atol=1e-15)


def test_topk_ties_by_index():
    z = np.array([[1.0, 3.0, 3.0, 2.0, 3.0]])
    assert list(mlp.topk(z, 3)[0]) == [1, 2, 4]


def test_training_reduces_loss_on_separable_toy():
    dims = (2, 16, 16, 4)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((256, 2))
    y = (x[:, 0] > 0).astype(int) * 2 + (x[:, 1] > 0).astype(int)
    p = mlp.init_params(dims, 6)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    l0, _ = mlp.loss_and_grads(p, x, y)
    for t in range(1, 301):
        _, g = mlp.loss_and_grads(p, x, y)
        mlp.adam_step(p, g, m, v, t, lr=1e-2)
    l1, _ = mlp.loss_and_grads(p, x, y)
    z, _ = mlp.forward(p, x)
    assert l1 < 0.2 * l0 and np.mean(np.argmax(z, 1) == y) > 0.95


def test_bf16_round_ties_to_even_and_library_routine():
    """Round to nearest bfloat16, ties to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 and
    goes to 1 (even mantissa); 1 + 3 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6 and goes up;
    representable values stay; and the whole map equals torch's own float32 -> bfloat16 conversion."""
    import torch
    x = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-8, -(1 + 2**-8), 1 + 2**-8 + 2**-20, 0.0, -0.0, 2.0**-130, 3.0e38])
    want = np.array([1.0, 1.0, 1 + 2**-6, -1.0, 1 + 2**-7, 0.0, -0.0, 2.0**-130, None], dtype=object)
    got = mlp.bf16_round(x)
    for g, w in zip(got[:-1], want[:-1]):
        assert g == w
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(50000) * 10.0 ** rng.integers(-30, 30, 50000),
                        rng.standard_normal(1000).astype(np.float32).astype(np.float64)])
    lib = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(v), lib)


def test_linear_bf16_is_the_plain_layer_on_rounded_operands():
    """A hand case, then: on BF16-representable operands the layer is the exact binary64 matmul
    plus bias (and GELU of it); otherwise it is that of the rounded operands."""
    z = mlp.linear_bf16(np.array([[1.0, 2.0]]), np.array([[3.0, 4.0], [5.0, 6.0]]), np.array([0.5, -1.0]))
    assert np.array_equal(z, np.array([[11.5, 16.0]]))
    rng = np.random.default_rng(6)
    x = mlp.bf16_round(rng.standard_normal((7, 40)))
    w = mlp.bf16_round(rng.standard_normal((9, 40)))
    b = rng.standard_normal(9)
    exact = x @ w.T + b
    assert np.array_equal(mlp.linear_bf16(x, w, b), exact)
    assert np.array_equal(mlp.linear_bf16(x, w, b, act=1), mlp.gelu(exact))
    xr, wr = rng.standard_normal((5, 33)), rng.standard_normal((4, 33))
    assert np.array_equal(mlp.linear_bf16(xr, wr), mlp.bf16_round(xr) @ mlp.bf16_round(wr).T)
    assert not np.array_equal(mlp.linear_bf16(xr, wr), xr @ wr.T)


def _case(dims, batch, seed):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(dims, seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.3
    return p, rng.standard_normal((batch, dims[0])), rng.integers(0, dims[3], batch)


def test_bf16_gradient_without_rounding_is_the_exact_gradient():
    """With the rounding taken out, the BF16-operand loss and gradients are the exact ones
    (which the finite differences above pin), for every parameter."""
    p, x, y = _case((5, 7, 6, 9), 11, 7)
    l0, g0 = mlp.loss_and_grads(p, x, y)
    l1, g1 = mlp.loss_and_grads_bf16(p, x, y, rnd=lambda a: a)
    assert abs(l0 - l1) <= 1e-15 * abs(l0)
    for k in mlp.PARAM_ORDER:
        assert np.allclose(g1[k], g0[k], rtol=1e-14, atol=1e-17), k


def test_bf16_gradient_rounds_every_contraction_operand():
    """The rounding reaches each operand of the training contractions once: the three weight
    matrices, the input, both hidden activations and the three back-propagated signals (dz
    and the two GELU-scaled hidden gradients), identified by shape and, for the forward
    activations, by value against the exact forward pass."""
    dims, batch = (5, 7, 6, 9), 11
    p, x, y = _case(dims, batch, 8)
    seen = []
    mlp.loss_and_grads_bf16(p, x, y, rnd=lambda a: (seen.append(np.array(a, np.float64)), a)[1])
    k, h1, h2, c = dims
    shapes = sorted(a.shape for a in seen)
    assert shapes == sorted([(h1, k), (h2, h1), (c, h2), (batch, k), (batch, h1), (batch, h2), (batch, c),
                             (batch, h2), (batch, h1)])
    _, (x64, a1, h1v, a2, h2v) = mlp.forward(p, x)
    assert any(a.shape == h1v.shape and np.array_equal(a, h1v) for a in seen)
    assert any(a.shape == h2v.shape and np.array_equal(a, h2v) for a in seen)
    assert any(a.shape == x64.shape and np.array_equal(a, x64) for a in seen)
    for name in ("W1", "W2", "W3"):
        assert any(a.shape == p[name].shape and np.array_equal(a, p[name]) for a in seen)


def test_bf16_gradient_is_within_the_operand_rounding_of_the_exact_one():
    """Rounding the operands moves the weight gradients by about the BF16 unit (2^-8 relative,
    2^-9 on average per operand): normwise between 1e-4 and 2e-2 of the exact gradient."""
    p, x, y = _case((16, 64, 48, 40), 96, 9)
    _, g0 = mlp.loss_and_grads(p, x, y)
    _, g1 = mlp.loss_and_grads_bf16(p, x, y)
    for k in ("W1", "W2", "W3"):
        rel = np.linalg.norm(g1[k] - g0[k]) / np.linalg.norm(g0[k])
        assert 1e-4 < rel < 2e-2, (k, rel)
