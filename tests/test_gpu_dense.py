"""GPU parity of the tcgen05 dense prefix scan (BF16 prefix) against the oracle, in both
forms: one pass (group codes, HN_SCAN_DENSE) and Algorithm 1's two passes
(HN_SCAN_DENSE_TWO_PASS)."""
import numpy as np
import pytest
import torch

import hn_synth
import oracle
from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu

DENSE, STREAM, DENSE2 = 2, 1, 3
FORMS = pytest.mark.parametrize("form", [DENSE, DENSE2])


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@FORMS
def test_dense_one_tile(hn, form):
    """One query tile, one entry tile: the smallest launch."""
    w, db, q, o_idx, o_sim = oracle_case(256, 128, 40, 21, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=form, stats=True)
        assert r.stats["scan"] == form
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("n,nq", [(1, 1), (2, 3), (255, 1), (257, 129), (1000, 200), (4097, 300), (20011, 1000)])
@FORMS
def test_dense_ragged_sizes(hn, n, nq, form):
    w, db, q, o_idx, o_sim = oracle_case(n, nq, max(1, n // 5), 22, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=form)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("k,alpha", [(8, 1 / 32), (16, 0.0), (16, 0.25), (24, 1 / 16), (32, 1 / 8), (64, 1 / 8),
                                     (3, 0.5)])
@FORMS
def test_dense_k_alpha(hn, k, alpha, form):
    w, db, q, o_idx, o_sim = oracle_case(9001, 700, 1500, 23, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=form)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_dense_config0(hn):
    c = hn_synth.CONFIGS["c0"]
    w, db, q, o_idx, o_sim = oracle_case(c["n"], c["nq"], c["n_centres"], c["seed"], c["k"], c["alpha"])
    with hn.Index(to_dev(db), c["k"], c["alpha"], prefix=1) as ix:
        r = ix.search(to_dev(q), scan=DENSE, stats=True)
        assert_parity(r.idx, r.sim, o_idx, o_sim)
        assert r.stats["survivors"] >= c["nq"]


@FORMS
def test_dense_ties_and_duplicates(hn, form):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 256, 300, seed=31)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 2000), (10, 2999), (255, 256), (511, 0), (1024, 1023)]:
        db[b] = db[a]
    q[0], q[130], q[255] = db[10], db[255], db[0]
    o_idx, o_sim = oracle.search(db, q)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=form)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_dense_equals_stream_and_repeats(hn):
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(50000, 3000, 10000, 24, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        qd = to_dev(q)
        ref = ix.search(qd, scan=STREAM)
        outs = [ix.search(qd, scan=DENSE) for _ in range(3)] + [ix.search(qd, scan=DENSE2)]
        for r in outs:
            assert torch.equal(r.idx, ref.idx) and torch.equal(r.sim, ref.sim)
        assert_parity(outs[0].idx, outs[0].sim, o_idx, o_sim)


@FORMS
def test_dense_overflow_rerun(hn, form):
    k, alpha = 8, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 500, 4000, 5, k, alpha, 0.3, 0.2)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        r = ix.search(to_dev(q), scan=form, bucket_cap=16, stats=True)
        assert r.stats["reruns"] >= 1
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("prefix", [1, 2])
@pytest.mark.parametrize("limit", [1, 600_000])
@FORMS
def test_dense_passes_over_query_tiles(hn, prefix, limit, form):
    """A scratch limit below the group map's size runs the dense scan in passes over
    256-query tiles (11 tiles here, the last one holding 40 queries): limit 1 takes one
    tile a pass, 600 kB a few tiles a pass with a shorter last pass.  Same answers as
    the oracle, and as one pass."""
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20011, 2600, 4000, 25, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
        qd = to_dev(q)
        one = ix.search(qd, scan=form, stats=True)
        assert one.stats["passes"] == 1
        r = ix.search(qd, scan=form, stats=True, scratch_limit=limit)
        assert r.stats["passes"] >= 3, r.stats
        if limit == 1:
            assert r.stats["passes"] == 11
        assert_parity(r.idx, r.sim, o_idx, o_sim)
        assert r.stats["survivors"] == one.stats["survivors"]


@pytest.mark.parametrize("prefix", [1, 2])
@pytest.mark.parametrize("k,n,nq", [(16, 20011, 1000), (16, 3001, 257), (32, 9001, 700), (64, 4097, 300)])
def test_plain_epilogue_matches_oracle(hn, prefix, k, n, nq):
    """The one-pass scan's unsplit form (one reducing TMEM load in flight per epilogue warp, no
    register split), which a build without the split falls back to: the oracle's answers, and
    the same survivors and group visits as the default form on the same batch."""
    alpha = 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(n, nq, max(1, n // 5), 41 + k, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
        r0 = ix.search(to_dev(q), scan=DENSE, stats=True)
        r1 = ix.search(to_dev(q), scan=DENSE, stats=True, test_plain_epilogue=True)
        assert_parity(r1.idx, r1.sim, o_idx, o_sim)
        assert_parity(r0.idx, r0.sim, o_idx, o_sim)
        for key in ("survivors", "groups_scored", "fp64_rescored"):
            assert r1.stats[key] == r0.stats[key], key


def test_plain_epilogue_rejects_bad_value(hn):
    from paper_2606_27280_b300 import hn as binding
    w, db, q, o_idx, o_sim = oracle_case(300, 10, 60, 45, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        opts = binding.SearchOpts(scan=DENSE, test_plain_epilogue=2)
        qd = to_dev(q)
        oi = torch.empty(qd.shape[0], dtype=torch.int64, device=qd.device)
        os_ = torch.empty(qd.shape[0], dtype=torch.float64, device=qd.device)
        st = binding._lib.hn_search_batch(ix._h, qd.data_ptr(), qd.shape[0], binding.ctypes.byref(opts),
                                          oi.data_ptr(), os_.data_ptr(), None, None)
        assert st == binding.ERR_INVALID_ARG
