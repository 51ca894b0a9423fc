"""GPU tests of the proposal's tensor-core inference: one layer (tcgen05.mma, BF16 operands,
FP32 accumulation) against its binary64 definition on the same rounded operands, with the
accumulation bound of FP32 sums; the network's block scores against the oracle evaluated
layer by layer, with that bound carried through the BF16 roundings of the hidden layers; and
the top-k blocks against the scores they rank."""
import os

import numpy as np
import pytest
import torch

import hn_synth
import oracle
from oracle import mlp
from tests._gpu_util import assert_parity, to_dev

pytestmark = pytest.mark.gpu

U = 2.0 ** -24          # unit roundoff of binary32
GELU_SLOPE = 1.13       # max |gelu'| (1.1289 at a = 2.42)


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


def layer_bound(xb, wb, b, act, pre_ref):
    """Largest |GPU - binary64| of one layer on BF16 operands xb, wb: the FP32 sum of k exact
    products in any order is within gamma_k sum|x w|; the bias add and the store round once
    more; GELU (evaluated in FP32 with erff) carries the pre-activation error with slope <= 1.13
    and adds a few ulps of its own."""
    k = xb.shape[1]
    gamma = k * U / (1 - k * U)
    s = np.abs(xb) @ np.abs(wb).T
    e = gamma * s + 2 * U * (np.abs(pre_ref) + (np.abs(b) if b is not None else 0.0)) + 1e-30
    if act == 1:
        e = GELU_SLOPE * e + 8 * U * np.abs(mlp.gelu(pre_ref)) + 1e-30
    return e


@pytest.mark.parametrize("m,k,n,act,bias,seed", [
    (1, 16, 256, 1, True, 0),       # one row, one tile
    (300, 16, 256, 1, True, 1),     # ragged rows
    (129, 256, 256, 1, True, 2),    # four K slices
    (257, 256, 4096, 0, True, 3),   # the block layer: 16 column tiles
    (200, 8, 40, 1, True, 4),       # K below one MMA step, ragged columns
    (1000, 200, 300, 0, False, 5),  # ragged K slice, no bias
    (64, 1, 17, 0, True, 6),        # K = 1
])
def test_linear_bf16_matches_definition(hn, m, k, n, act, bias, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((m, k)).astype(np.float32)
    w = (rng.standard_normal((n, k)) * np.sqrt(2.0 / k)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32) if bias else None
    got = hn.linear_bf16(to_dev(x), to_dev(w), to_dev(b) if bias else None, act=act).cpu().numpy().astype(np.float64)
    pre = mlp.linear_bf16(x, w, b, act=0)
    want = mlp.gelu(pre) if act == 1 else pre
    bound = layer_bound(mlp.bf16_round(x), mlp.bf16_round(w), b, act, pre)
    err = np.abs(got - want)
    # the bound (about k 2^-24 relative) is far below the operand rounding (2^-9), so a kernel
    # that skipped or misplaced the BF16 rounding would fail here
    assert np.all(err <= bound), (float(np.max(err / bound)), float(np.max(err)))


def test_linear_bf16_edges(hn):
    from paper_2606_27280_b300 import hn as binding
    x = to_dev(np.ones((0, 16), np.float32))
    w = to_dev(np.ones((5, 16), np.float32))
    assert hn.linear_bf16(x, w).shape == (0, 5)
    with pytest.raises(hn.HNError) as e:
        hn.linear_bf16(to_dev(np.ones((3, 16), np.float32)), w, act=2)
    assert e.value.status == binding.ERR_INVALID_ARG


def read_saved_params(path, dims):
    k, h1, h2, c = dims
    raw = np.fromfile(path, dtype=np.uint8)
    assert bytes(raw[:8]) == b"HNPROP01"
    hdr = raw[8:24].view(np.int32)
    assert tuple(hdr) == (k, h1, h2, c)
    w = raw[40:].view(np.float32)
    sizes = [h1 * k, h1, h2 * h1, h2, c * h2, c]
    out, o = [], 0
    for s in sizes:
        out.append(w[o:o + s].astype(np.float64))
        o += s
    W1, b1, W2, b2, W3, b3 = out
    return W1.reshape(h1, k), b1, W2.reshape(h2, h1), b2, W3.reshape(c, h2), b3


def test_proposal_logits_and_topk(hn, tmp_path):
    """Block scores of a trained proposal against the binary64 network on BF16-rounded weights,
    each layer's input rounded to BF16 as the kernels do.  The GPU rounds its own FP32 hidden
    values, which may sit one BF16 step away from the oracle's; the bound carries that step
    (2^-7 relative) through the next layer.  The top-k blocks are the scores' top-k (score
    desc, block asc)."""
    k, alpha = 16, 1 / 8
    wl = hn_synth.make_workload(40000, 700, 8000, seed=61)
    db = oracle.normalize(wl.db_raw, k, alpha)
    q = oracle.normalize(wl.q_raw, k, alpha)
    tq_raw, _ = hn_synth.queries_from(wl.db_raw, 8000, seed=62)
    with hn.Index(to_dev(db), k, alpha, prefix=1, n_blocks=300) as ix:
        with hn.Proposal.train(ix, to_dev(oracle.normalize(tq_raw, k, alpha)), hidden1=96, hidden2=80, epochs=2,
                               batch=1024, seed=3) as prop:
            path = os.path.join(str(tmp_path), "p.bin")
            prop.save(path)
            W1, b1, W2, b2, W3, b3 = read_saved_params(path, (k, 96, 80, 300))
            z = prop.logits(to_dev(q)).cpu().numpy().astype(np.float64)
            top = prop.infer(to_dev(q), 4).cpu().numpy()
    Wb = [mlp.bf16_round(W) for W in (W1, W2, W3)]
    x = q[:, :k].astype(np.float64)
    # layer 1 (input: the query prefix)
    pre1 = mlp.linear_bf16(x, Wb[0], b1)
    h1 = mlp.gelu(pre1)
    e1 = layer_bound(mlp.bf16_round(x), Wb[0], b1, 1, pre1)
    # layer 2: the GPU's rounded h1 is within e1 + one BF16 step of the oracle's rounded h1
    d1 = e1 + 2.0 ** -7 * (np.abs(h1) + e1)
    pre2 = mlp.linear_bf16(h1, Wb[1], b2)
    h2 = mlp.gelu(pre2)
    e2 = GELU_SLOPE * (d1 @ np.abs(Wb[1]).T) + layer_bound(mlp.bf16_round(h1), Wb[1], b2, 1, pre2)
    d2 = e2 + 2.0 ** -7 * (np.abs(h2) + e2)
    zr = mlp.linear_bf16(h2, Wb[2], b3)
    ez = d2 @ np.abs(Wb[2]).T + layer_bound(mlp.bf16_round(h2), Wb[2], b3, 0, zr)
    err = np.abs(z - zr)
    assert np.all(err <= ez), float(np.max(err / ez))
    assert float(np.median(err / np.maximum(np.abs(zr), 1e-3))) < 1e-2
    # the ranking is that of the scores: score descending, block ascending
    order = np.lexsort((np.arange(z.shape[1])[None, :].repeat(z.shape[0], 0), -z), axis=1)[:, :4]
    assert np.array_equal(top, order)


def _strided(rng, rows, cols, row_major):
    """A (rows, cols) matrix held row-major or column-major: (flat storage, row stride, col stride)."""
    a = rng.standard_normal((rows, cols)).astype(np.float32)
    if row_major:
        return a, a.ravel(), cols, 1
    return a, np.ascontiguousarray(a.T).ravel(), 1, rows


@pytest.mark.parametrize("a_rows,b_rows", [(True, False), (False, True), (True, True), (False, False)])
@pytest.mark.parametrize("m,n,k", [(300, 256, 16), (17, 40, 8), (256, 256, 1000), (129, 300, 200), (5, 3, 1),
                                   (512, 16, 4096), (130, 70, 3001)])
def test_gemm_bf16_strides_match_definition(hn, a_rows, b_rows, m, n, k):
    """The training GEMM C = bf16(A) bf16(B) for every operand layout training uses (an
    activation read by rows or, for a weight gradient, by columns; a weight read by rows or
    transposed), at ragged sizes and K up to 1000 (a batch-sized weight-gradient contraction),
    element by element against the binary64 definition with the FP32 sum's bound.  The long
    contractions (K of 1000 and more on few output tiles) run split across CTAs, the last split
    ragged at K = 3001."""
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    a, af, sai, sak = _strided(rng, m, k, a_rows)
    b, bf, sbk, sbj = _strided(rng, k, n, b_rows)
    got = hn.gemm_bf16(to_dev(af), to_dev(bf), m, n, k, sai, sak, sbk, sbj).cpu().numpy().astype(np.float64)
    ab, bb = mlp.bf16_round(a), mlp.bf16_round(b)
    want = ab @ bb
    gamma = k * U / (1 - k * U)
    bound = gamma * (np.abs(ab) @ np.abs(bb)) + U * np.abs(want) + 1e-30
    err = np.abs(got - want)
    assert np.all(err <= bound), (float(np.max(err / bound)), float(np.max(err)))


def test_gemm_bf16_edges(hn):
    from paper_2606_27280_b300 import hn as binding
    a = to_dev(np.ones(64, np.float32))
    assert hn.gemm_bf16(a, a, 0, 4, 4, 4, 1, 4, 1).shape == (0, 4)
    # the last elements read: a 3*16 + 15 = 63, b 15*4 + 3 = 63; both fit
    assert torch.all(hn.gemm_bf16(a, a, 4, 4, 16, 16, 1, 4, 1) == 16.0)
    # a split contraction sums its partials in a fixed order: repeated calls agree bit for bit
    rng = np.random.default_rng(5)
    x = to_dev(rng.standard_normal(4096 * 300).astype(np.float32))
    y = to_dev(rng.standard_normal(4096 * 200).astype(np.float32))
    r1 = hn.gemm_bf16(x, y, 300, 200, 4096, 1, 300, 200, 1)
    r2 = hn.gemm_bf16(x, y, 300, 200, 4096, 1, 300, 200, 1)
    assert torch.equal(r1, r2)
    with pytest.raises(ValueError):          # one more row of a would read element 79
        hn.gemm_bf16(a, a, 5, 4, 16, 16, 1, 4, 1)
    with pytest.raises(hn.HNError) as e:     # K = 0 is not a contraction
        hn.gemm_bf16(a, a, 4, 4, 0, 4, 1, 4, 1)
    assert e.value.status == binding.ERR_INVALID_ARG


@pytest.mark.parametrize("dims,batch,seed", [((16, 32, 24, 50), 64, 0), ((8, 20, 12, 7), 5, 1),
                                             ((16, 256, 256, 300), 130, 2), ((16, 256, 256, 4096), 1024, 3)])
def test_mlp_gradients_bf16_match_oracle(hn, dims, batch, seed):
    """Tensor-core training gradients against the binary64 oracle that rounds every contraction
    operand to BF16.  Where they differ: the FP32 sums (gamma_K relative) and the GPU's own FP32
    hidden values and back-propagated signals, which may round to the neighbouring BF16 value
    (probability about |FP32 error| / BF16 step per element, each such step 2^-8 relative); a
    CPU simulation of that arithmetic stays below 2e-4 normwise per tensor.  The bound, 1e-3,
    is under half of what leaving the operands unrounded moves the weight gradients (2e-3 to
    5e-3), which the test checks on the oracle side."""
    rng = np.random.default_rng(seed)
    p = mlp.init_params(dims, seed)
    for key in ("b1", "b2", "b3"):
        p[key] = rng.standard_normal(p[key].shape) * 0.2
    flat32 = mlp.flatten(p).astype(np.float32)
    x = rng.standard_normal((batch, dims[0])).astype(np.float32)
    y = rng.integers(0, dims[3], batch).astype(np.int32)
    p64 = mlp.unflatten(flat32.astype(np.float64), dims)
    loss_ref, g_ref = mlp.loss_and_grads_bf16(p64, x.astype(np.float64), y)
    _, g_exact = mlp.loss_and_grads(p64, x.astype(np.float64), y)
    loss, g = hn.mlp_loss_grad(to_dev(flat32), dims, to_dev(x), to_dev(y), bf16=True)
    g = mlp.unflatten(g.cpu().numpy().astype(np.float64), dims)
    assert abs(loss - loss_ref) <= 1e-4 * max(1.0, abs(loss_ref)), (loss, loss_ref)
    tol = 1e-3
    for name in mlp.PARAM_ORDER:
        ref = np.linalg.norm(g_ref[name])
        rel = np.linalg.norm(g[name] - g_ref[name]) / max(ref, 1e-30)
        assert rel <= tol, (name, rel)
        if name.startswith("W"):   # the bound tells rounded from unrounded operands apart
            assert np.linalg.norm(g_exact[name] - g_ref[name]) / ref > 2 * tol, name


@pytest.mark.parametrize("precision", [0, 1])
def test_training_precisions_train_and_seed_exactly(hn, precision):
    """Both training precisions bring the loss below that of a uniform guess over the blocks
    and seed an exact search, as does the untrained network."""
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(30000, 300, 6000, seed=71)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    tq_raw, _ = hn_synth.queries_from(w.db_raw, 16000, seed=72)
    tq = to_dev(oracle.normalize(tq_raw, k, alpha))
    o_idx, o_sim = oracle.search(db, q)
    with hn.Index(to_dev(db), k, alpha, prefix=1, n_blocks=128) as ix:
        with hn.Proposal.train(ix, tq, hidden1=64, hidden2=64, epochs=0, seed=9, precision=precision) as p0, \
             hn.Proposal.train(ix, tq, hidden1=64, hidden2=64, epochs=4, batch=1024, lr=2e-3, seed=9,
                               precision=precision) as p4:
            assert p4.info()["steps"] == 4 * 16
            assert np.isfinite(p4.info()["last_loss"]) and p4.info()["last_loss"] < np.log(128)
            r = ix.search(to_dev(q), proposal=p4, seed_topk=4)
            assert_parity(r.idx, r.sim, o_idx, o_sim)
            r0 = ix.search(to_dev(q), proposal=p0, seed_topk=4)
            assert_parity(r0.idx, r0.sim, o_idx, o_sim)


def test_training_rejects_bad_precision(hn):
    from paper_2606_27280_b300 import hn as binding
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 0, 500, seed=73)
    db = to_dev(oracle.normalize(w.db_raw, k, alpha))
    with hn.Index(db, k, alpha, prefix=1, n_blocks=16) as ix:
        with pytest.raises(hn.HNError) as e:
            hn.Proposal.train(ix, db[:256], epochs=1, precision=2)
        assert e.value.status == binding.ERR_INVALID_ARG
