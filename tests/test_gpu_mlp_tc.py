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
from tests._gpu_util import to_dev

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
