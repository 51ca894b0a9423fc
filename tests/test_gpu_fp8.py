"""GPU parity of the FP8-e4m3 prefix (per-entry power-of-two scale, per-entry error
term) against the oracle: both scan kernels, ragged sizes, every supported K,
ties, and agreement with the BF16 and FP32 indexes."""
import numpy as np
import pytest
import torch

import hn_synth
import oracle
from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu

STREAM, DENSE, DENSE2 = 1, 2, 3


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@pytest.mark.parametrize("scan", [STREAM, DENSE, DENSE2])
def test_fp8_config0(hn, scan):
    c = hn_synth.CONFIGS["c0"]
    w, db, q, o_idx, o_sim = oracle_case(c["n"], c["nq"], c["n_centres"], c["seed"], c["k"], c["alpha"])
    with hn.Index(to_dev(db), c["k"], c["alpha"], prefix=hn.PREFIX_FP8) as ix:
        r = ix.search(to_dev(q), scan=scan, stats=True)
        assert r.stats["scan"] == scan
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("n,nq", [(1, 1), (2, 3), (127, 5), (129, 257), (4097, 300), (20011, 1000)])
@pytest.mark.parametrize("scan", [STREAM, DENSE, DENSE2])
def test_fp8_ragged_sizes(hn, n, nq, scan):
    w, db, q, o_idx, o_sim = oracle_case(n, nq, max(1, n // 5), 41, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=hn.PREFIX_FP8) as ix:
        r = ix.search(to_dev(q), scan=scan)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("k,alpha", [(3, 0.5), (8, 1 / 32), (16, 0.0), (16, 0.25), (24, 1 / 16), (32, 1 / 8),
                                     (64, 1 / 8)])
@pytest.mark.parametrize("scan", [STREAM, DENSE, DENSE2])
def test_fp8_k_alpha(hn, k, alpha, scan):
    w, db, q, o_idx, o_sim = oracle_case(9001, 700, 1500, 42, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_FP8) as ix:
        inf = ix.info()
        assert inf["k_pad"] == max(16, 1 << (k - 1).bit_length())
        r = ix.search(to_dev(q), scan=scan)
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_fp8_ties_and_duplicates(hn):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 256, 300, seed=43)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 2000), (10, 2999), (127, 128), (511, 0), (1024, 1023)]:
        db[b] = db[a]
    q[0], q[130], q[255] = db[10], db[127], db[0]
    o_idx, o_sim = oracle.search(db, q)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_FP8) as ix:
        for scan in (STREAM, DENSE, DENSE2):
            r = ix.search(to_dev(q), scan=scan)
            assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_fp8_agrees_with_bf16_and_repeats(hn):
    """Same answers from every prefix precision and both kernels, byte for byte,
    over repeated runs; the FP8 bound is looser, so at least as many survive."""
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(50000, 3000, 10000, 44, k, alpha)
    qd = to_dev(q)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_BF16) as bf:
        ref = bf.search(qd, scan=DENSE, stats=True)
    assert_parity(ref.idx, ref.sim, o_idx, o_sim)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_FP8) as ix:
        inf = ix.info()
        assert inf["prefix"] == hn.PREFIX_FP8 and 0 < inf["resid_norm_max"] < 0.12
        runs = [ix.search(qd, scan=DENSE, stats=True) for _ in range(3)] + [ix.search(qd, scan=STREAM, stats=True),
                                                                            ix.search(qd, scan=DENSE2, stats=True)]
        for r in runs:
            assert torch.equal(r.idx, ref.idx) and torch.equal(r.sim, ref.sim)
        assert runs[0].stats["survivors"] >= ref.stats["survivors"]
        assert runs[0].stats["survivors"] == runs[1].stats["survivors"]   # deterministic counts


def test_fp8_hard_data_and_overflow_rerun(hn):
    """Noisier data (far more survivors) with tiny survivor storage: re-runs, still exact."""
    k, alpha = 8, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 500, 4000, 5, k, alpha, 0.3, 0.2)
    for scan in (STREAM, DENSE, DENSE2):   # a fresh index each: its survivor storage only grows
        with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_FP8) as ix:
            r = ix.search(to_dev(q), scan=scan, bucket_cap=2, stats=True)
            assert r.stats["max_survivors"] > 2 and r.stats["reruns"] >= 1, r.stats
            assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_fp8_seeded_search_exact(hn):
    """The learned proposal's threshold path on an FP8 index (candidates scored on master rows)."""
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 600, 4000, 45, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=hn.PREFIX_FP8, n_blocks=64) as ix:
        with hn.Proposal.train(ix, to_dev(q), hidden1=64, hidden2=64, epochs=2, batch=256, seed=3) as prop:
            for scan in (STREAM, DENSE):
                r = ix.search(to_dev(q), scan=scan, proposal=prop, seed_topk=4)
                assert_parity(r.idx, r.sim, o_idx, o_sim)
