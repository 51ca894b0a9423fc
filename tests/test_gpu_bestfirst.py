"""The 1-NN Phase-2 rescore modes against the oracle.

* HN_RESCORE_FILTER16 (the default): a certified upper bound from each survivor's FP16 row
  decides whether its FP32 row is read at all; the cut starts at the threshold candidates'
  certified bound and rises with the FP32 best.
* HN_RESCORE_BEST_FIRST (the early exit of a sorted Phase 2, next row f4): the same cut
  against the FP32 prefix bound.
* HN_RESCORE_FULL: every survivor scored in FP32 (Algorithm 1's Phase 2 in index order).

The answer must be the oracle's, bit for bit, for every scan and prefix, with ties, and on
noisy data where survivors are many and most of them are dropped by the bound."""
import numpy as np
import pytest

import hn_synth
import oracle
from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu

FILTER16, BEST_FIRST, FULL = 0, 1, 2
MODES = pytest.mark.parametrize("mode", [FILTER16, BEST_FIRST, FULL])


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@MODES
@pytest.mark.parametrize("prefix,scan", [(0, 1), (1, 1), (1, 2), (1, 3), (2, 2), (3, 1)])
@pytest.mark.parametrize("k,alpha", [(16, 1 / 8), (8, 1 / 32), (32, 1 / 16), (16, 0.0)])
def test_rescore_modes_equal_oracle(hn, mode, prefix, scan, k, alpha):
    w, db, q, o_idx, o_sim = oracle_case(20011, 700, 4000, 51, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
        r = ix.search(to_dev(q), scan=scan, rescore=mode, stats=True)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("prefix,scan", [(0, 1), (1, 2), (2, 2)])
def test_bounds_drop_survivors_on_noisy_data(hn, prefix, scan):
    """Many survivors (noisy data, K = 8, alpha = 1/8): both bounds drop survivors without
    changing the answer; the FP16 row bound is far tighter than the prefix bound."""
    k, alpha = 8, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 500, 4000, 5, k, alpha, 0.3, 0.2)
    with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
        qd = to_dev(q)
        full = ix.search(qd, scan=scan, stats=True, rescore=FULL)
        bf = ix.search(qd, scan=scan, stats=True, best_first=True)
        f16 = ix.search(qd, scan=scan, stats=True)
        for r in (full, bf, f16):
            assert_parity(r.idx, r.sim, o_idx, o_sim)
            assert r.stats["survivors"] == full.stats["survivors"]
        assert full.stats["rescore_skipped"] == 0
        assert 0 < bf.stats["rescore_skipped"] < bf.stats["survivors"]
        # the FP16 bound is within ~5e-4 of the similarity: nearly every survivor is dropped
        assert f16.stats["rescore_skipped"] >= 0.9 * f16.stats["survivors"]
        assert f16.stats["rescore_skipped"] > bf.stats["rescore_skipped"]


@MODES
def test_rescore_ties_and_duplicates(hn, mode):
    """Duplicated rows (exact ties of the binary64 similarity, at tile borders and far apart)
    and queries equal to an entry: every tied entry's bound reaches the cut, so the lowest
    index still wins."""
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 256, 300, seed=52)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 2000), (10, 2999), (255, 256), (511, 0), (1024, 1023)]:
        db[b] = db[a]
    q[0], q[130], q[255] = db[10], db[255], db[0]
    o_idx, o_sim = oracle.search(db, q)
    for prefix, scan in [(0, 1), (1, 2), (2, 2)]:
        with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
            r = ix.search(to_dev(q), scan=scan, rescore=mode)
            assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_filter16_soft_mode_and_seed(hn):
    """The filter under the soft ANN mode (the kept best candidate) and with a proposal seed:
    the same answers as the full rescore."""
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(30000, 600, 5000, 53, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=1, n_blocks=64) as ix:
        qd = to_dev(q)
        for beta in (alpha, alpha / 2, 0.0):
            a = ix.search(qd, beta=beta, rescore=FULL)
            b = ix.search(qd, beta=beta)
            assert np.array_equal(a.idx.cpu().numpy(), b.idx.cpu().numpy())
            assert np.array_equal(a.sim.cpu().numpy(), b.sim.cpu().numpy())
        tq_raw, _ = hn_synth.queries_from(w.db_raw, 4000, seed=54)
        with hn.Proposal.train(ix, to_dev(oracle.normalize(tq_raw, k, alpha)), hidden1=64, hidden2=64, epochs=1,
                               batch=1024, seed=5) as prop:
            r = ix.search(qd, proposal=prop)
            assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_rescore_mode_rejects_bad_value(hn):
    w, db, q, o_idx, o_sim = oracle_case(300, 10, 60, 45, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        with pytest.raises(hn.HNError) as e:
            ix.search(to_dev(q), rescore=3)
        from paper_2606_27280_b300 import hn as binding
        assert e.value.status == binding.ERR_INVALID_ARG
