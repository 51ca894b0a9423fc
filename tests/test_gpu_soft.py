"""GPU tests of the soft ANN mode (threshold relaxation, alpha -> beta in the skip
test): beta = alpha is the exact search, smaller beta prunes more and returns
entries no better than the oracle's."""
import numpy as np
import pytest

from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@pytest.mark.parametrize("prefix,scan", [(0, 1), (1, 2), (2, 2), (1, 3), (2, 3)])
def test_soft_beta_equal_alpha_is_exact(hn, prefix, scan):
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(30000, 800, 6000, 71, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
        exact = ix.search(to_dev(q), scan=scan, stats=True)
        soft = ix.search(to_dev(q), scan=scan, stats=True, beta=alpha)
        assert_parity(soft.idx, soft.sim, o_idx, o_sim)
        assert soft.stats["survivors"] == exact.stats["survivors"]


def test_soft_beta_trades_recall_for_pruning(hn):
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(30000, 800, 6000, 72, k, alpha, 0.3, 0.2)
    sims = (q.astype(np.float64) @ db.astype(np.float64).T)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        prev_surv, recalls = None, []
        for beta in [alpha, alpha / 2, alpha / 4, alpha / 16, 0.0]:
            r = ix.search(to_dev(q), scan=2, stats=True, beta=beta)
            gi, gs = r.idx.cpu().numpy(), r.sim.cpu().numpy()
            # every answer is a real entry with its exact binary64 similarity, never above the optimum
            assert np.all(gs <= o_sim)
            assert np.allclose(gs, sims[np.arange(len(q)), gi], atol=1e-12)
            recalls.append(np.mean(gi == o_idx))
            if prev_surv is not None:
                assert r.stats["survivors"] <= prev_surv
            prev_surv = r.stats["survivors"]
        assert recalls[0] == 1.0
        assert recalls[-1] < 1.0   # on this noisy data beta = 0 misses some neighbours


def test_soft_rejects_bad_beta(hn):
    w, db, q, _, _ = oracle_case(100, 4, 30, 73, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        for beta in (-0.01, 0.2):
            with pytest.raises(hn.HNError):
                ix.search(to_dev(q), beta=beta)
