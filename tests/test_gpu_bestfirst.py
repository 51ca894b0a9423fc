"""Best-first rescore (the early exit of a sorted Phase 2, next row f4): the survivor
with the largest FP32 prefix score is scored first and the rest only while their
prefix bound reaches the best certified full score.  The answer must be the
oracle's, bit for bit, for every scan and prefix, with ties, and on noisy data where
survivors are many and most of them are dropped by the bound."""
import numpy as np
import pytest

import hn_synth
import oracle
from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@pytest.mark.parametrize("prefix,scan", [(0, 1), (1, 1), (1, 2), (1, 3), (2, 2), (3, 1)])
@pytest.mark.parametrize("k,alpha", [(16, 1 / 8), (8, 1 / 32), (32, 1 / 16), (16, 0.0)])
def test_best_first_equals_oracle(hn, prefix, scan, k, alpha):
    w, db, q, o_idx, o_sim = oracle_case(20011, 700, 4000, 51, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
        r = ix.search(to_dev(q), scan=scan, best_first=True, stats=True)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("prefix,scan", [(0, 1), (1, 2)])
def test_best_first_drops_survivors_on_noisy_data(hn, prefix, scan):
    k, alpha = 8, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 500, 4000, 5, k, alpha, 0.3, 0.2)
    with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
        qd = to_dev(q)
        plain = ix.search(qd, scan=scan, stats=True)
        bf = ix.search(qd, scan=scan, stats=True, best_first=True)
        assert_parity(bf.idx, bf.sim, o_idx, o_sim)
        assert bf.stats["survivors"] == plain.stats["survivors"]
        assert plain.stats["rescore_skipped"] == 0
        assert 0 < bf.stats["rescore_skipped"] < bf.stats["survivors"]


def test_best_first_ties_and_duplicates(hn):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 256, 300, seed=52)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 2000), (10, 2999), (255, 256), (511, 0), (1024, 1023)]:
        db[b] = db[a]
    q[0], q[130], q[255] = db[10], db[255], db[0]
    o_idx, o_sim = oracle.search(db, q)
    for prefix, scan in [(0, 1), (1, 2)]:
        with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
            r = ix.search(to_dev(q), scan=scan, best_first=True)
            assert_parity(r.idx, r.sim, o_idx, o_sim)
