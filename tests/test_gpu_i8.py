"""GPU parity of the 8-bit fixed-point prefix (one power-of-two code scale per
index, one per query, integer dp4a scan) against the oracle: config c0, ragged
sizes, every supported K and several alpha, ties, near-duplicate data, the
proposal seed, top-k and the soft mode at beta = alpha."""
import numpy as np
import pytest
import torch

import hn_synth
import oracle
from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu

STREAM, DENSE = 1, 2


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


def test_i8_config0(hn):
    c = hn_synth.CONFIGS["c0"]
    w, db, q, o_idx, o_sim = oracle_case(c["n"], c["nq"], c["n_centres"], c["seed"], c["k"], c["alpha"])
    with hn.Index(to_dev(db), c["k"], c["alpha"], prefix=hn.PREFIX_I8) as ix:
        r = ix.search(to_dev(q), stats=True)
        assert r.stats["scan"] == STREAM   # the AUTO choice for an int8 index
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("n,nq", [(1, 1), (2, 3), (127, 5), (255, 64), (257, 65), (4097, 300), (20011, 1000)])
def test_i8_ragged_sizes(hn, n, nq):
    w, db, q, o_idx, o_sim = oracle_case(n, nq, max(1, n // 5), 51, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=hn.PREFIX_I8) as ix:
        r = ix.search(to_dev(q))
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("k,alpha", [(3, 0.5), (8, 1 / 32), (16, 0.0), (16, 1 / 16), (16, 0.25), (24, 1 / 8),
                                     (32, 1 / 8), (40, 1 / 32), (64, 1 / 8)])
def test_i8_k_alpha(hn, k, alpha):
    w, db, q, o_idx, o_sim = oracle_case(9001, 700, 1500, 52, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_I8) as ix:
        inf = ix.info()
        assert inf["prefix"] == hn.PREFIX_I8 and inf["k_pad"] == max(16, 1 << (k - 1).bit_length())
        # one code scale s <= 2 max|x_d| / 127 <= 2 / 127 and |error| <= s / 2 per coordinate
        assert 0 < inf["resid_norm_max"] <= np.sqrt(k) / 127 * 1.0001
        r = ix.search(to_dev(q))
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_i8_ties_and_duplicates(hn):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 256, 300, seed=53)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 2000), (10, 2999), (127, 128), (255, 256), (511, 0), (1024, 1023)]:
        db[b] = db[a]
    q[0], q[130], q[255] = db[10], db[127], db[0]
    o_idx, o_sim = oracle.search(db, q)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_I8) as ix:
        r = ix.search(to_dev(q))
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_i8_near_duplicates(hn):
    """Entries that differ by far less than one code step: the integer scan cannot tell them
    apart, so most of them survive to the FP32/binary64 rescore, which must still pick the
    oracle's answer."""
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(6000, 200, 3, 54, k, alpha, 0.002, 0.001)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_I8) as ix:
        r = ix.search(to_dev(q), stats=True)
        assert r.stats["max_survivors"] > 100, r.stats
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_i8_agrees_with_f32_and_repeats(hn):
    """Same answers as the FP32 index, byte for byte, over repeated runs with identical
    survivor counts (the integer scan has no rounding to race on)."""
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(50000, 3000, 10000, 55, k, alpha)
    qd = to_dev(q)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_F32) as f32:
        ref = f32.search(qd, stats=True)
    assert_parity(ref.idx, ref.sim, o_idx, o_sim)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_I8) as ix:
        runs = [ix.search(qd, stats=True) for _ in range(3)]
        for r in runs:
            assert torch.equal(r.idx, ref.idx) and torch.equal(r.sim, ref.sim)
        assert runs[0].stats["survivors"] >= ref.stats["survivors"]
        assert runs[0].stats["survivors"] == runs[1].stats["survivors"] == runs[2].stats["survivors"]


def test_i8_dense_scan_unsupported(hn):
    w, db, q, o_idx, o_sim = oracle_case(1000, 10, 100, 56, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=hn.PREFIX_I8) as ix:
        with pytest.raises(hn.HNError):
            ix.search(to_dev(q), scan=DENSE)


def test_i8_hard_data_and_overflow_rerun(hn):
    """Noisier data (far more survivors) with tiny survivor storage: re-runs, still exact."""
    k, alpha = 8, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 500, 4000, 5, k, alpha, 0.3, 0.2)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_I8) as ix:
        r = ix.search(to_dev(q), bucket_cap=2, stats=True)
        assert r.stats["max_survivors"] > 2 and r.stats["reruns"] >= 1, r.stats
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_i8_seeded_search_exact(hn):
    """The learned proposal's threshold path on an int8 index (candidates scored on master rows)."""
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 600, 4000, 57, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_I8, n_blocks=64) as ix:
        with hn.Proposal.train(ix, to_dev(q), hidden1=64, hidden2=64, epochs=2, batch=256, seed=3) as prop:
            r = ix.search(to_dev(q), proposal=prop, seed_topk=4)
            assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("topk", [1, 5, 32])
def test_i8_topk_matches_oracle(hn, topk):
    k, alpha = 16, 1 / 8
    w, db, q, _, _ = oracle_case(8000, 300, 1600, 58, k, alpha)
    o_idx, o_sim = oracle.search_topk(db, q, topk)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_I8) as ix:
        r = ix.search_topk(to_dev(q), topk)
        assert np.array_equal(r.idx.cpu().numpy(), o_idx)
        assert np.array_equal(r.sim.cpu().numpy(), o_sim)


def test_i8_soft_mode_at_alpha_is_exact(hn):
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(8000, 300, 1600, 59, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_I8) as ix:
        r = ix.search(to_dev(q), beta=alpha)
        assert_parity(r.idx, r.sim, o_idx, o_sim)
        a = ix.search(to_dev(q), beta=alpha / 2)   # relaxed: a valid entry and its exact similarity
        ai, asim = a.idx.cpu().numpy(), a.sim.cpu().numpy()
        assert np.all((ai >= 0) & (ai < len(db)))
        assert all(asim[i] == oracle.dot(q[i], db[ai[i]]) for i in range(len(q)))
        assert np.all(asim <= o_sim)
