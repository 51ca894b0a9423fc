"""GPU parity of the tcgen05 dense prefix scan (BF16 prefix) against the oracle."""
import numpy as np
import pytest
import torch

import hn_synth
import oracle
from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu

DENSE, STREAM = 2, 1


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


def test_dense_one_tile(hn):
    """One query tile, one entry tile: the smallest launch."""
    w, db, q, o_idx, o_sim = oracle_case(256, 128, 40, 21, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=DENSE, stats=True)
        assert r.stats["scan"] == DENSE
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("n,nq", [(1, 1), (2, 3), (255, 1), (257, 129), (1000, 200), (4097, 300), (20011, 1000)])
def test_dense_ragged_sizes(hn, n, nq):
    w, db, q, o_idx, o_sim = oracle_case(n, nq, max(1, n // 5), 22, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=DENSE)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("k,alpha", [(8, 1 / 32), (16, 0.0), (16, 0.25), (24, 1 / 16), (32, 1 / 8), (64, 1 / 8),
                                     (3, 0.5)])
def test_dense_k_alpha(hn, k, alpha):
    w, db, q, o_idx, o_sim = oracle_case(9001, 700, 1500, 23, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=DENSE)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_dense_config0(hn):
    c = hn_synth.CONFIGS["c0"]
    w, db, q, o_idx, o_sim = oracle_case(c["n"], c["nq"], c["n_centres"], c["seed"], c["k"], c["alpha"])
    with hn.Index(to_dev(db), c["k"], c["alpha"], prefix=1) as ix:
        r = ix.search(to_dev(q), scan=DENSE, stats=True)
        assert_parity(r.idx, r.sim, o_idx, o_sim)
        assert r.stats["survivors"] >= c["nq"]


def test_dense_ties_and_duplicates(hn):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 256, 300, seed=31)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 2000), (10, 2999), (255, 256), (511, 0), (1024, 1023)]:
        db[b] = db[a]
    q[0], q[130], q[255] = db[10], db[255], db[0]
    o_idx, o_sim = oracle.search(db, q)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=DENSE)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_dense_equals_stream_and_repeats(hn):
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(50000, 3000, 10000, 24, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        qd = to_dev(q)
        ref = ix.search(qd, scan=STREAM)
        outs = [ix.search(qd, scan=DENSE) for _ in range(3)]
        for r in outs:
            assert torch.equal(r.idx, ref.idx) and torch.equal(r.sim, ref.sim)
        assert_parity(outs[0].idx, outs[0].sim, o_idx, o_sim)


def test_dense_overflow_rerun(hn):
    k, alpha = 8, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 500, 4000, 5, k, alpha, 0.3, 0.2)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=DENSE, bucket_cap=16, stats=True)
        assert r.stats["reruns"] >= 1
        assert_parity(r.idx, r.sim, o_idx, o_sim)
