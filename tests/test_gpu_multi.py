"""GPU tests of batched serving (hn_search_multi, CUDA-graph replay) and the autotuner."""
import numpy as np
import pytest
import torch

import hn_synth
import oracle
from tests._gpu_util import assert_parity, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@pytest.fixture(scope="module")
def setup(hn):
    """Three indexes (different K, alpha, prefix) and 24 uneven batches over them."""
    specs = [(20000, 8, 1 / 32, 1, 31), (12000, 16, 1 / 8, 1, 32), (9000, 16, 1 / 8, 0, 33)]
    indexes, data = [], []
    for n, k, a, prefix, seed in specs:
        w = hn_synth.make_workload(n, 0, n // 5, seed=seed)
        db = oracle.normalize(w.db_raw, k, a)
        indexes.append(hn.Index(to_dev(db), k, a, prefix=prefix))
        data.append((w, db, k, a))
    sizes = [int(x) for x in hn_synth.log_uniform_sizes(5, 24, 1, 600)]
    sizes[3] = 0  # an empty batch
    rng = np.random.default_rng(6)
    batches, expected = [], []
    for b, nq in enumerate(sizes):
        g = int(rng.integers(0, 3))
        w, db, k, a = data[g]
        qr, _ = hn_synth.queries_from(w.db_raw, max(nq, 1), seed=100 + b)
        q = oracle.normalize(qr, k, a)[:nq]
        o = oracle.search(db, q) if nq else (np.zeros(0, np.int64), np.zeros(0))
        qd = to_dev(q) if nq else torch.zeros((0, 128), dtype=torch.float32, device="cuda")
        batches.append((indexes[g], qd, torch.empty(nq, dtype=torch.int64, device="cuda"),
                        torch.empty(nq, dtype=torch.float64, device="cuda")))
        expected.append(o)
    yield hn, indexes, batches, expected
    for ix in indexes:
        ix.close()


def _check_all(batches, expected):
    for (ix, q, oi, os_), (e_idx, e_sim) in zip(batches, expected):
        if q.shape[0]:
            assert_parity(oi, os_, e_idx, e_sim)


def test_multi_graph_then_replay(setup):
    hn, indexes, batches, expected = setup
    st = hn.search_multi(batches, use_graph=True)
    assert st["n_groups"] == 3 and st["n_batches"] == 24 and st["graph_replayed"] == 0
    assert st["ms_total"] > 0 and 0 < st["batch_ms_p50"] <= st["batch_ms_p99"] <= st["batch_ms_max"]
    _check_all(batches, expected)
    for _, _, oi, os_ in batches:
        oi.fill_(-1)
        os_.fill_(0)
    st2 = hn.search_multi(batches, use_graph=True)
    assert st2["graph_replayed"] == 1
    _check_all(batches, expected)


def test_multi_without_graph_and_after_workspace_change(setup):
    hn, indexes, batches, expected = setup
    st = hn.search_multi(batches, use_graph=False)
    assert st["graph_replayed"] == 0
    _check_all(batches, expected)
    # a large single search reallocates an index's scratch: the graph must be rebuilt, not replayed
    ix, q, _, _ = batches[0]
    big = q.repeat(40, 1)
    ix.search(big)
    st = hn.search_multi(batches, use_graph=True)
    assert st["graph_replayed"] == 0
    _check_all(batches, expected)


def test_autotune_keeps_results_exact(hn):
    k, a = 16, 1 / 8
    w = hn_synth.make_workload(30000, 1500, 6000, seed=34)
    db = oracle.normalize(w.db_raw, k, a)
    q = oracle.normalize(w.q_raw, k, a)
    o_idx, o_sim = oracle.search(db, q)
    with hn.Index(to_dev(db), k, a, prefix=1) as ix:
        r = ix.autotune([64, 512, 2048])
        assert r["units_per_cta"] in (32, 64, 128, 256)
        assert len(r["ms_stream"]) == 3 and all(t > 0 for t in r["ms_stream"] + r["ms_dense"])
        res = ix.search(to_dev(q), stats=True)
        assert_parity(res.idx, res.sim, o_idx, o_sim)
        assert res.stats["scan"] == (2 if 1500 >= r["dense_min_q"] else 1)


def test_shared_one_pass_scan_across_indexes(hn):
    """Four BF16 indexes (K 8 and 16 share the padded width 16; two alphas) take one shared
    persistent one-pass scan; an FP32 index (stream scan) and an FP8 index (another tile
    format) keep their own pipelines.  Every batch equals the oracle, with and without the
    graph, and on replay."""
    specs = [(40000, 8, 1 / 32, 1, 41), (25000, 16, 1 / 8, 1, 42), (30011, 16, 1 / 32, 1, 43),
             (18000, 8, 1 / 8, 1, 44), (15000, 16, 1 / 8, 0, 45), (20000, 16, 1 / 8, 2, 46)]
    indexes, data = [], []
    for n, k, a, prefix, seed in specs:
        w = hn_synth.make_workload(n, 0, n // 5, seed=seed)
        db = oracle.normalize(w.db_raw, k, a)
        indexes.append(hn.Index(to_dev(db), k, a, prefix=prefix))
        data.append((w, db, k, a))
    try:
        rng = np.random.default_rng(47)
        batches, expected = [], []
        for b in range(30):
            g = b % len(specs)
            nq = int(rng.integers(300, 700)) if g != 4 else int(rng.integers(1, 40))   # FP32 group: stream scan
            w, db, k, a = data[g]
            qr, _ = hn_synth.queries_from(w.db_raw, nq, seed=200 + b)
            q = oracle.normalize(qr, k, a)
            batches.append((indexes[g], to_dev(q), torch.empty(nq, dtype=torch.int64, device="cuda"),
                            torch.empty(nq, dtype=torch.float64, device="cuda")))
            expected.append(oracle.search(db, q))
        for use_graph in (True, True, False):
            for _, _, oi, os_ in batches:
                oi.fill_(-1)
                os_.fill_(0)
            st = hn.search_multi(batches, use_graph=use_graph)
            assert st["n_groups"] == 6 and st["joined"] == 4, st
            _check_all(batches, expected)
        assert st["survivors"] > 0
    finally:
        for ix in indexes:
            ix.close()
