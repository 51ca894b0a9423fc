"""Entry-range sharding on the GPU: the merge kernel against the library's host merge,
and the sharded search of one database cut into three entry ranges (three indexes on
one GPU standing in for three ranks; the all-gather is the stacking of their answers)
against the oracle's search over the whole database."""
import numpy as np
import pytest
import torch

import hn_synth
import oracle
from tests._gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@pytest.mark.parametrize("shards,k", [(1, 1), (3, 1), (4, 8), (64, 32)])
def test_merge_kernel_equals_host_merge(hn, shards, k):
    rng = np.random.default_rng(shards + 100 * k)
    nq = 777
    idx = np.sort(rng.integers(-1, 50, size=(shards, nq, k)), axis=2)       # -1 = empty slot
    sim = np.where(idx >= 0, rng.integers(0, 3, size=idx.shape) / 2.0, -np.inf)
    # each list in (sim desc, idx asc) order, empty slots last
    for r in range(shards):
        for j in range(nq):
            order = np.lexsort((np.where(idx[r, j] < 0, 1 << 40, idx[r, j]), -sim[r, j]))
            idx[r, j], sim[r, j] = idx[r, j][order], sim[r, j][order]
    off = (np.arange(shards) * 50).astype(np.int64)
    hi, hs = hn.merge_topk_host(idx, sim, off)
    gi, gs = hn.merge_topk(to_dev(idx), to_dev(sim), to_dev(off))
    assert np.array_equal(gi.cpu().numpy(), hi) and np.array_equal(gs.cpu().numpy(), hs)


@pytest.mark.parametrize("prefix", [1, 2])
def test_three_shard_search_equals_oracle(hn, prefix):
    from paper_2606_27280_b300.shard import shard_range
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(30011, 1500, 6000, seed=62)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    for a, b in [(10, 29000), (10009, 10010), (5, 20100)]:      # ties across the range boundaries
        db[b] = db[a]
    q[0], q[1] = db[10], db[10009]
    o1 = oracle.search(db, q)
    o5 = oracle.search_topk(db, q, 5)
    qd = to_dev(q)
    parts, offs = [], []
    for r in range(3):
        lo, hi = shard_range(db.shape[0], r, 3)
        parts.append(hn.Index(to_dev(db[lo:hi]), k, alpha, prefix=prefix))
        offs.append(lo)
    try:
        off = torch.tensor(offs, dtype=torch.int64, device="cuda")
        r1 = [p.search(qd) for p in parts]
        gi, gs = hn.merge_topk(torch.stack([r.idx for r in r1])[:, :, None], torch.stack([r.sim for r in r1])[:, :, None], off)
        assert np.array_equal(gi[:, 0].cpu().numpy(), o1[0]) and np.array_equal(gs[:, 0].cpu().numpy(), o1[1])
        r5 = [p.search_topk(qd, 5) for p in parts]
        gi, gs = hn.merge_topk(torch.stack([r.idx for r in r5]), torch.stack([r.sim for r in r5]), off)
        assert np.array_equal(gi.cpu().numpy(), o5[0]) and np.array_equal(gs.cpu().numpy(), o5[1])
    finally:
        for p in parts:
            p.close()
