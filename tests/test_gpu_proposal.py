"""GPU tests of the learned block proposal: training kernels against the
binary64 MLP oracle, the block partition, and the seeded search (exact either
way, Phase 1 skipped when seeded)."""
import numpy as np
import pytest
import torch

import hn_synth
import oracle
from oracle import mlp
from tests._gpu_util import assert_parity, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@pytest.mark.parametrize("dims,batch,seed", [((16, 32, 24, 50), 64, 0), ((8, 20, 12, 7), 5, 1),
                                             ((16, 256, 256, 300), 130, 2)])
def test_mlp_gradients_match_oracle(hn, dims, batch, seed):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(dims, seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.2
    flat32 = mlp.flatten(p).astype(np.float32)
    x = rng.standard_normal((batch, dims[0])).astype(np.float32)
    y = rng.integers(0, dims[3], batch).astype(np.int32)
    # the oracle sees exactly the float32 values the GPU sees
    p64 = mlp.unflatten(flat32.astype(np.float64), dims)
    loss_ref, g_ref = mlp.loss_and_grads(p64, x.astype(np.float64), y)
    g_ref = mlp.flatten(g_ref)
    loss, g = hn.mlp_loss_grad(to_dev(flat32), dims, to_dev(x), to_dev(y))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - loss_ref) <= 2e-5 * max(1.0, abs(loss_ref))
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * scale, np.max(np.abs(g - g_ref)) / scale
    # per-tensor relative error too
    o = 0
    for name in mlp.PARAM_ORDER:
        n = p64[name].size
        gr, gg = g_ref[o:o + n], g[o:o + n]
        o += n
        assert np.linalg.norm(gg - gr) <= 1e-4 * max(np.linalg.norm(gr), 1e-12), name


def test_block_partition(hn):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(20011, 0, 2000, seed=51)
    x = to_dev(oracle.normalize(w.db_raw, k, alpha))
    outs = []
    for _ in range(2):
        with hn.Index(x, k, alpha, n_blocks=97, kmeans_iters=4) as ix:
            assert ix.info()["n_blocks"] == 97
            start, ids, of = (t.cpu().numpy() for t in ix.blocks())
            outs.append((start, ids, of))
    start, ids, of = outs[0]
    n = 20011
    assert start[0] == 0 and start[-1] == n
    assert np.array_equal(start, (np.arange(98) * n) // 97)       # equal contiguous blocks
    assert np.array_equal(np.sort(ids), np.arange(n))            # a permutation
    for b in range(97):
        assert np.all(of[ids[start[b]:start[b + 1]]] == b)
    for a, b in zip(outs[0], outs[1]):                           # deterministic build
        assert np.array_equal(a, b)
    # blocks are coherent in prefix space: members are closer to their block mean than to a random block's
    pre = oracle.normalize(w.db_raw, k, alpha)[:, :k].astype(np.float64)
    means = np.stack([pre[ids[start[b]:start[b + 1]]].mean(0) for b in range(97)])
    own = np.einsum("ij,ij->i", pre, means[of])
    other = np.einsum("ij,ij->i", pre, means[(of + 31) % 97])
    assert np.mean(own) > np.mean(other) + 0.1


@pytest.fixture(scope="module")
def trained(hn):
    k, alpha = 16, 1 / 8
    n = 60000
    w = hn_synth.make_workload(n, 600, 12000, seed=52)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    tq_raw, _ = hn_synth.queries_from(w.db_raw, 40000, seed=53)
    tq = to_dev(oracle.normalize(tq_raw, k, alpha))
    ix = hn.Index(to_dev(db), k, alpha, prefix=1, n_blocks=256)
    prop = hn.Proposal.train(ix, tq, hidden1=128, hidden2=128, epochs=6, batch=1024, lr=2e-3, seed=7)
    o_idx, o_sim = oracle.search(db, q)
    yield hn, ix, prop, db, q, o_idx, o_sim
    prop.close()
    ix.close()


def test_proposal_trains_and_ranks_nn_block(trained):
    hn, ix, prop, db, q, o_idx, o_sim = trained
    info = prop.info()
    assert info["epochs"] == 6 and info["steps"] == 6 * 40 and info["n_blocks"] == 256
    assert np.isfinite(info["last_loss"]) and info["last_loss"] < np.log(256)
    top = prop.infer(to_dev(q), 4).cpu().numpy()
    _, _, of = (t.cpu().numpy() for t in ix.blocks())
    hit = np.mean([of[o_idx[j]] in top[j] for j in range(len(q))])
    assert hit > 0.3, hit   # chance level is 4/256; the query noise moves many prefixes across blocks


@pytest.mark.parametrize("topk,scan", [(1, 2), (4, 2), (4, 1), (16, 2), (64, 2)])
def test_seeded_search_is_exact(trained, topk, scan):
    hn, ix, prop, db, q, o_idx, o_sim = trained
    r = ix.search(to_dev(q), scan=scan, proposal=prop, seed_topk=topk, stats=True)
    assert_parity(r.idx, r.sim, o_idx, o_sim)
    plain = ix.search(to_dev(q), scan=scan, stats=True)
    assert_parity(plain.idx, plain.sim, o_idx, o_sim)
    if topk >= 16:   # enough blocks: the seed prunes within a small factor of the plain search,
        # whose threshold takes the best of up to 32 candidates found across its whole scan
        assert r.stats["survivors"] < 6 * plain.stats["survivors"], (r.stats["survivors"], plain.stats["survivors"])


def test_training_gain_over_untrained_network(trained):
    """What training buys: the same network untrained ranks blocks at chance level, so its
    threshold is weak and far more entries survive the bound test (exact either way)."""
    hn, ix, prop, db, q, o_idx, o_sim = trained
    tq = to_dev(q[:64])
    with hn.Proposal.train(ix, tq, hidden1=128, hidden2=128, epochs=0, seed=7) as raw:
        qd = to_dev(q)
        r_raw = ix.search(qd, proposal=raw, seed_topk=4, stats=True)
        r_tr = ix.search(qd, proposal=prop, seed_topk=4, stats=True)
        assert_parity(r_raw.idx, r_raw.sim, o_idx, o_sim)
        assert_parity(r_tr.idx, r_tr.sim, o_idx, o_sim)
        assert r_tr.stats["survivors"] < 0.5 * r_raw.stats["survivors"], (r_tr.stats, r_raw.stats)


def test_save_load_roundtrip_and_continue(trained, tmp_path):
    hn, ix, prop, db, q, o_idx, o_sim = trained
    path = tmp_path / "prop.bin"
    prop.save(path)
    with hn.Proposal.load(path) as p2:
        assert p2.info()["steps"] == prop.info()["steps"]
        qd = to_dev(q)
        assert torch.equal(p2.infer(qd, 4), prop.infer(qd, 4))
        tq_raw, _ = hn_synth.queries_from(np.ascontiguousarray(db), 2048, seed=54)
        tq = to_dev(tq_raw)   # already HN rows: db rows plus small noise are renormalised below
        tq = hn.normalize(tq, 16, 1 / 8)
        with hn.Proposal.train(ix, tq, epochs=1, batch=512, init=p2) as p3:
            assert p3.info()["steps"] == p2.info()["steps"] + 4
            assert p3.info()["epochs"] == p2.info()["epochs"] + 1


def test_seeded_search_rejects_foreign_proposal(trained):
    hn, ix, prop, db, q, o_idx, o_sim = trained
    with hn.Index(to_dev(db[:5000]), 16, 1 / 8, n_blocks=64) as other:
        with pytest.raises(hn.HNError):
            other.search(to_dev(q[:10]), proposal=prop)
