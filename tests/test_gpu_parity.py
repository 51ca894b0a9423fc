"""GPU parity: the CUDA path (through the C ABI) against the binary64 oracle.

Index bit-exact for every query; similarity within 1e-6 (and, by design,
bit-identical: the winner is re-scored in the oracle's own summation order).
"""
import numpy as np
import pytest
import torch

import hn_synth
import oracle
from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


# ---------------------------------------------------------------- Eq. 1
@pytest.mark.parametrize("k,alpha", [(8, 1 / 32), (16, 1 / 8), (16, 0.0), (16, 0.25), (1, 0.5), (127, 1 / 3), (64, 0.1)])
def test_normalize_bit_exact(hn, k, alpha):
    w = hn_synth.make_workload(3001, 17, 100, seed=7)
    raw = np.concatenate([w.db_raw, w.q_raw])
    raw[5, :k] *= 1e-30
    raw[9, k:] *= 3e30
    want = oracle.normalize(raw, k, alpha)
    got = hn.normalize(to_dev(raw), k, alpha).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_normalize_in_place_and_zero_norm(hn):
    raw = hn_synth.make_workload(100, 0, 10, seed=1).db_raw
    x = to_dev(raw)
    hn.normalize(x, 16, 0.125, out=x)
    assert np.array_equal(x.cpu().numpy(), oracle.normalize(raw, 16, 0.125))
    bad = raw.copy()
    bad[37, :16] = 0
    with pytest.raises(hn.HNError) as e:
        hn.normalize(to_dev(bad), 16, 0.125)
    assert e.value.status == 3


@pytest.mark.parametrize("k,alpha", [(16, 1 / 8), (1, 0.0), (127, 0.9)])
def test_normalize_async_bit_exact(hn, k, alpha):
    """The stream-ordered form: the same bits as the oracle, in place too, status untouched."""
    w = hn_synth.make_workload(2049, 300, 100, seed=8)
    raw = np.concatenate([w.db_raw, w.q_raw])
    raw[7, :k] *= 1e-30
    want = oracle.normalize(raw, k, alpha)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    got = hn.normalize_async(to_dev(raw), k, alpha, status=status)
    x = to_dev(raw)
    hn.normalize_async(x, k, alpha, out=x)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))
    assert np.array_equal(x.cpu().numpy().view(np.uint32), want.view(np.uint32))
    assert status.cpu().tolist() == [0, 0]


def test_normalize_async_bad_rows(hn):
    """A zero-norm or non-finite row: flagged in status, copied unchanged, and the search of
    a batch holding it reports HN_ERR_NOT_NORMALIZED; the other rows are normalised."""
    from paper_2606_27280_b300 import hn as binding
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(4000, 64, 400, seed=9)
    db = oracle.normalize(w.db_raw, k, alpha)
    raw = w.q_raw.copy()
    raw[5, :k] = 0
    raw[40, 100] = np.nan
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    q = hn.normalize_async(to_dev(raw), k, alpha, status=status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [1, 1]
    got = q.cpu().numpy()
    assert np.array_equal(got[5], raw[5]) and np.isnan(got[40, 100])
    good = np.ones(len(raw), bool)
    good[[5, 40]] = False
    assert np.array_equal(got[good], oracle.normalize(raw[good], k, alpha))
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        for scan in (hn.SCAN_DENSE, hn.SCAN_STREAM):
            with pytest.raises(hn.HNError) as e:
                ix.search(q, scan=scan)
            assert e.value.status == binding.ERR_NOT_NORMALIZED
    with pytest.raises(ValueError):
        hn.normalize_async(to_dev(raw), k, alpha, status=torch.zeros(2, dtype=torch.int64, device="cuda"))


def test_index_rejects_unnormalized(hn):
    raw = hn_synth.make_workload(1000, 0, 10, seed=1).db_raw
    with pytest.raises(hn.HNError) as e:
        hn.Index(to_dev(raw), 16, 0.125)
    assert e.value.status == 2
    x = oracle.normalize(raw, 16, 0.125)
    x[400, 3] *= 1.001
    with pytest.raises(hn.HNError) as e:
        hn.Index(to_dev(x), 16, 0.125)
    assert e.value.status == 2 and "400" in str(e.value)


def _gpu_norm(hn, raw, k, alpha):
    return hn.normalize(to_dev(raw), k, alpha)


# ---------------------------------------------------------------- config 0
@pytest.mark.parametrize("prefix,scan", [(0, 1), (1, 1)])
def test_config0_full_parity(hn, prefix, scan):
    c = hn_synth.CONFIGS["c0"]
    w, db, q, o_idx, o_sim = oracle_case(c["n"], c["nq"], c["n_centres"], c["seed"], c["k"], c["alpha"])
    with hn.Index(_gpu_norm(hn, w.db_raw, c["k"], c["alpha"]), c["k"], c["alpha"], prefix=prefix) as ix:
        r = ix.search(_gpu_norm(hn, w.q_raw, c["k"], c["alpha"]), scan=scan, stats=True)
        assert_parity(r.idx, r.sim, o_idx, o_sim)
        st = r.stats
        assert st["survivors"] >= c["nq"]           # every Phase-1 winner survives
        assert st["survivors"] < 0.05 * c["n"] * c["nq"]


@pytest.mark.parametrize("k,alpha,prefix", [(16, 1 / 8, 0), (16, 0.0, 0), (16, 0.25, 1), (4, 0.5, 0), (32, 1 / 16, 1),
                                            (64, 1 / 8, 0), (9, 1 / 32, 1)])
def test_parity_k_alpha_grid(hn, k, alpha, prefix):
    w, db, q, o_idx, o_sim = oracle_case(6007, 333, 700, 3, k, alpha)
    with hn.Index(_gpu_norm(hn, w.db_raw, k, alpha), k, alpha, prefix=prefix) as ix:
        r = ix.search(_gpu_norm(hn, w.q_raw, k, alpha))
        assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_hard_variant_many_survivors(hn):
    """Large noise: survivors reach percent level; tiny slots force overflow re-runs."""
    k, alpha = 8, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(20000, 500, 4000, 5, k, alpha, 0.3, 0.2)
    with hn.Index(_gpu_norm(hn, w.db_raw, k, alpha), k, alpha) as ix:
        qd = _gpu_norm(hn, w.q_raw, k, alpha)
        r = ix.search(qd, stats=True, bucket_cap=16)
        assert_parity(r.idx, r.sim, o_idx, o_sim)
        assert r.stats["reruns"] >= 1
        r2 = ix.search(qd, stats=True)
        assert_parity(r2.idx, r2.sim, o_idx, o_sim)


def test_ties_lowest_index(hn):
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(3000, 64, 300, seed=11)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 2000), (10, 2999), (255, 256), (511, 0)]:
        db[b] = db[a]
    q[0] = db[10]
    q[1] = db[255]
    q[2] = db[0]
    o_idx, o_sim = oracle.search(db, q)
    assert o_idx[0] == 10 and o_idx[1] == 255 and o_idx[2] == 0
    for prefix in (0, 1):
        with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
            r = ix.search(to_dev(q))
            assert_parity(r.idx, r.sim, o_idx, o_sim)


@pytest.mark.parametrize("n,nq", [(1, 1), (2, 3), (255, 1), (256, 64), (257, 65), (1000, 129), (513, 7)])
def test_edge_sizes(hn, n, nq):
    k, alpha = 8, 1 / 32
    w, db, q, o_idx, o_sim = oracle_case(n, nq, max(1, n // 5), 13, k, alpha)
    for prefix in (0, 1):
        with hn.Index(to_dev(db), k, alpha, prefix=prefix) as ix:
            r = ix.search(to_dev(q))
            assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_empty_query_batch(hn):
    k, alpha = 8, 1 / 32
    w, db, q, _, _ = oracle_case(300, 4, 30, 13, k, alpha)
    with hn.Index(to_dev(db), k, alpha) as ix:
        r = ix.search(torch.empty(0, 128, device="cuda"))
        assert r.idx.numel() == 0


def test_deterministic_across_runs_and_slots(hn):
    k, alpha = 16, 1 / 8
    w, db, q, o_idx, o_sim = oracle_case(30000, 2000, 6000, 17, k, alpha)
    outs = []
    with hn.Index(to_dev(db), k, alpha) as ix:
        qd = to_dev(q)
        for cap in (0, 0, 8, 4096):
            r = ix.search(qd, bucket_cap=cap)
            outs.append((r.idx.cpu().numpy().copy(), r.sim.cpu().numpy().copy()))
    for i, s in outs:
        assert np.array_equal(i, outs[0][0]) and np.array_equal(s, outs[0][1])
    assert np.array_equal(outs[0][0], o_idx)


def test_bruteforce_baseline(hn):
    c = hn_synth.CONFIGS["c0"]
    w, db, q, o_idx, o_sim = oracle_case(c["n"], c["nq"], c["n_centres"], c["seed"], c["k"], c["alpha"])
    with hn.Index(to_dev(db), c["k"], c["alpha"]) as ix:
        r = ix.bruteforce(to_dev(q))
        gi = r.idx.cpu().numpy()
        # FP32 ranking: same winner unless two scores are within FP32 rounding
        assert np.mean(gi == o_idx) > 0.99
        assert np.max(np.abs(r.sim.cpu().numpy() - o_sim)) < 1e-5


def test_index_info(hn):
    k, alpha = 16, 1 / 8
    w, db, q, _, _ = oracle_case(1000, 4, 30, 13, k, alpha)
    with hn.Index(to_dev(db), k, alpha, prefix=1) as ix:
        inf = ix.info()
    assert inf["n"] == 1000 and inf["k"] == 16 and inf["k_pad"] == 16 and inf["prefix"] == 1
    maj2, min2 = oracle.part_norms2(db, k)
    assert inf["minor_norm_max"] >= np.sqrt(min2.max())
    assert inf["major_norm_max"] >= np.sqrt(maj2.max())
    assert 0 < inf["resid_norm_max"] < 0.02


# ---------------------------------------------------------------- full-size configs, sampled queries
def _sampled_parity(hn, name, prefix, scan, n_sample):
    wl, c = hn_synth.config_workload(name)
    k, alpha = c["k"], c["alpha"]
    db_o = oracle.normalize(wl.db_raw, k, alpha)
    rng = np.random.default_rng(123)
    pick = np.sort(rng.choice(c["nq"], n_sample, replace=False))
    q_o = oracle.normalize(wl.q_raw[pick], k, alpha)
    o_idx, o_sim = oracle.search(db_o, q_o)
    del db_o
    with hn.Index(_gpu_norm(hn, wl.db_raw, k, alpha), k, alpha, prefix=prefix) as ix:
        r = ix.search(_gpu_norm(hn, wl.q_raw, k, alpha), scan=scan, stats=True)
        sel = torch.from_numpy(pick).cuda()
        assert_parity(r.idx[sel], r.sim[sel], o_idx, o_sim)
        return r.stats


def test_config1_full_size_sampled(hn):
    st = _sampled_parity(hn, "c1", prefix=0, scan=1, n_sample=256)
    assert st["n_queries"] == 16384


def test_config2_full_size_sampled_bf16(hn):
    st = _sampled_parity(hn, "c2", prefix=1, scan=0, n_sample=128)
    assert st["n_queries"] == 65536


def test_config2_full_size_sampled_fp8(hn):
    st = _sampled_parity(hn, "c2", prefix=2, scan=0, n_sample=128)
    assert st["n_queries"] == 65536 and st["scan"] == 2
