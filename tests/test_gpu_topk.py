"""GPU parity of the exact top-k search (hn_search_topk) against the oracle's
exhaustive top-k: both scan kernels, every prefix precision, ties, ragged sizes."""
import numpy as np
import pytest

import hn_synth
import oracle
from tests._gpu_util import oracle_case, to_dev

pytestmark = pytest.mark.gpu

STREAM, DENSE, DENSE2 = 1, 2, 3


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


def _check(res, o_idx, o_sim):
    gi = res.idx.cpu().numpy()
    gs = res.sim.cpu().numpy()
    bad = np.argwhere(gi != o_idx)
    assert bad.size == 0, f"{len(bad)} rank mismatches, first (query, rank) {bad[:3].tolist()}"
    assert np.array_equal(gs, o_sim), "similarities differ from the oracle's binary64 values"


@pytest.mark.parametrize("rescore", [0, 2])   # FP16-row filter (default), every survivor in FP32
@pytest.mark.parametrize("k", [1, 2, 5, 16, 32])
@pytest.mark.parametrize("prefix,scan", [(0, STREAM), (1, STREAM), (1, DENSE), (2, DENSE), (1, DENSE2), (2, DENSE2)])
def test_topk_matches_oracle(hn, k, prefix, scan, rescore):
    w, db, q, _, _ = oracle_case(20011, 700, 4000, 61, 16, 1 / 8)
    o_idx, o_sim = oracle.search_topk(db, q, k)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=prefix) as ix:
        r = ix.search_topk(to_dev(q), k, scan=scan, stats=True, rescore=rescore)
        assert r.stats["scan"] == scan
        _check(r, o_idx, o_sim)
        if k == 1:
            r1 = ix.search(to_dev(q), scan=scan)
            assert np.array_equal(r1.idx.cpu().numpy(), r.idx.cpu().numpy()[:, 0])


def test_topk_rank0_is_the_1nn_and_pruning_holds(hn):
    c = hn_synth.CONFIGS["c0"]
    w, db, q, o1, s1 = oracle_case(c["n"], c["nq"], c["n_centres"], c["seed"], c["k"], c["alpha"])
    o_idx, o_sim = oracle.search_topk(db, q, 8)
    assert np.array_equal(o_idx[:, 0], o1)
    with hn.Index(to_dev(db), c["k"], c["alpha"], prefix=1) as ix:
        r = ix.search_topk(to_dev(q), 8, scan=DENSE, stats=True)
        _check(r, o_idx, o_sim)
        assert r.stats["survivors"] < 0.2 * c["nq"] * c["n"]   # the bound still prunes


def test_topk_duplicates_and_ties(hn):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 256, 300, seed=62)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 2000), (10, 2999), (10, 5), (127, 128), (511, 0), (1024, 1023)]:
        db[b] = db[a]
    q[0], q[130], q[255] = db[10], db[127], db[0]
    o_idx, o_sim = oracle.search_topk(db, q, 6)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        for scan in (STREAM, DENSE):
            _check(ix.search_topk(to_dev(q), 6, scan=scan), o_idx, o_sim)


@pytest.mark.parametrize("n,nq,k", [(1, 3, 1), (5, 4, 5), (33, 7, 32), (300, 129, 10), (4097, 257, 7)])
def test_topk_ragged_sizes(hn, n, nq, k):
    w, db, q, _, _ = oracle_case(n, nq, max(1, n // 5), 63, 16, 1 / 8)
    o_idx, o_sim = oracle.search_topk(db, q, k)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        for scan in (STREAM, DENSE):
            _check(ix.search_topk(to_dev(q), k, scan=scan), o_idx, o_sim)


def test_topk_hard_data_overflow_rerun(hn):
    w, db, q, _, _ = oracle_case(20000, 300, 4000, 5, 8, 1 / 8, 0.3, 0.2)
    o_idx, o_sim = oracle.search_topk(db, q, 10)
    for scan in (STREAM, DENSE):
        with hn.Index(to_dev(db), 8, 1 / 8, prefix=1) as ix:
            r = ix.search_topk(to_dev(q), 10, scan=scan, bucket_cap=16, stats=True)
            assert r.stats["reruns"] >= 1
            _check(r, o_idx, o_sim)


def test_topk_rejects_bad_k(hn):
    w, db, q, _, _ = oracle_case(100, 4, 30, 64, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        for k in (0, 33, 101):
            with pytest.raises(hn.HNError):
                ix.search_topk(to_dev(q), k)


@pytest.mark.parametrize("k", [4, 32])
def test_topk_filter_skips_survivors_on_noisy_data(hn, k):
    """Many survivors (noisy data, K = 8, alpha = 1/8): the FP16-row bound against the k-th
    best certified score drops most of them, the answer stays the oracle's, and the
    survivor count is that of the full rescore."""
    w, db, q, _, _ = oracle_case(20000, 400, 4000, 63, 8, 1 / 8, 0.3, 0.2)
    o_idx, o_sim = oracle.search_topk(db, q, k)
    with hn.Index(to_dev(db), 8, 1 / 8, prefix=1) as ix:
        qd = to_dev(q)
        full = ix.search_topk(qd, k, scan=DENSE, stats=True, rescore=2)
        f16 = ix.search_topk(qd, k, scan=DENSE, stats=True)
        _check(full, o_idx, o_sim)
        _check(f16, o_idx, o_sim)
        assert f16.stats["survivors"] == full.stats["survivors"]
        assert full.stats["rescore_skipped"] == 0
        assert f16.stats["rescore_skipped"] >= 0.8 * f16.stats["survivors"]


def test_topk_filter_cache_overflow(hn):
    """A query whose kept survivors pass the per-warp cache (128): every entry is a duplicate of
    one of 40 rows, so the top-32 band holds far more than 128 kept survivors and pass 2 bounds
    the survivors again; the answer (ties by index) is the oracle's."""
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(4000, 8, 400, seed=64)
    db = oracle.normalize(w.db_raw, k, alpha)
    db = db[np.arange(4000) % 40]
    q = oracle.normalize(w.q_raw, k, alpha)
    q[0] = db[3]
    o_idx, o_sim = oracle.search_topk(db, q, 32)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        for scan in (STREAM, DENSE):
            _check(ix.search_topk(to_dev(q), 32, scan=scan), o_idx, o_sim)
