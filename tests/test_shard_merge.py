"""Entry-range sharding on CPU: the merge of per-shard exact answers (similarity
descending, global index ascending -- the tie rule of Theorem 2) against a plain
sort of the union, and the whole exchange step (gloo all-gather + merge) run by
world_size 2 and 3 ranks whose per-shard answers come from the oracle: the
merged answer must equal the oracle's search over the whole database, bit for bit.
No GPU is used: the library's host merge does the merging."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hn():
    from paper_2606_27280_b300 import hn as mod
    return mod


def _sorted_lists(rng, shards, nq, k, n_local):
    """Per-shard answer lists already in (sim desc, local idx asc) order, with repeated
    similarities (ties inside and across shards) and empty slots."""
    idx = np.full((shards, nq, k), -1, np.int64)
    sim = np.full((shards, nq, k), -np.inf)
    for r in range(shards):
        for j in range(nq):
            m = min(k, n_local[r])
            ids = rng.choice(n_local[r], size=m, replace=False)
            s = rng.integers(0, 4, size=m) / 4.0          # few distinct values: many ties
            order = np.lexsort((ids, -s))
            idx[r, j, :m], sim[r, j, :m] = ids[order], s[order]
    return idx, sim


@pytest.mark.parametrize("shards,k", [(1, 1), (2, 1), (3, 4), (5, 7), (64, 2)])
def test_host_merge_equals_sorted_union(hn, shards, k):
    rng = np.random.default_rng(shards * 31 + k)
    n_local = rng.integers(1, 12, size=shards)
    off = np.concatenate([[0], np.cumsum(n_local)[:-1]]).astype(np.int64)
    idx, sim = _sorted_lists(rng, shards, 50, k, n_local)
    got_i, got_s = hn.merge_topk_host(idx, sim, off)
    for j in range(50):
        cand = [(sim[r, j, t], idx[r, j, t] + off[r]) for r in range(shards) for t in range(k) if idx[r, j, t] >= 0]
        cand.sort(key=lambda c: (-c[0], c[1]))
        want = cand[:k] + [(-np.inf, -1)] * (k - len(cand[:k]))
        assert [int(i) for i in got_i[j]] == [int(c[1]) for c in want]
        assert [float(s) for s in got_s[j]] == [float(c[0]) for c in want]


def test_host_merge_rejects_bad_args(hn):
    z = np.zeros((65, 1, 1), np.int64)
    with pytest.raises(hn.HNError):
        hn.merge_topk_host(z, z.astype(np.float64), np.zeros(65, np.int64))      # more than 64 shards
    z = np.zeros((2, 1, 33), np.int64)
    with pytest.raises(hn.HNError):
        hn.merge_topk_host(z, z.astype(np.float64), np.zeros(2, np.int64))       # k > 32


def test_shard_ranges_cover_the_database():
    sys.path.insert(0, ROOT)
    from paper_2606_27280_b300.shard import shard_range
    for n, world in [(0, 1), (1, 3), (10, 3), (1000, 7), (4_000_000, 8)]:
        parts = [shard_range(n, r, world) for r in range(world)]
        assert parts[0][0] == 0 and parts[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [hi - lo for lo, hi in parts]
        assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    """c0-like data, K = 8, alpha = 1/32, with entries duplicated across shard boundaries
    so that exact similarity ties must resolve to the lower global index."""
    import hn_synth
    import oracle
    w = hn_synth.make_workload(3001, 120, 300, seed=61)
    db = oracle.normalize(w.db_raw, 8, 1 / 32)
    q = oracle.normalize(w.q_raw, 8, 1 / 32)
    for a, b in [(10, 2990), (1499, 1500), (1000, 2000), (5, 1001)]:
        db[b] = db[a]
    q[0], q[1], q[2] = db[10], db[1499], db[1000]
    return db, q


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2606_27280_b300.shard import gather_and_merge, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        db, q = _case()
        lo, hi = shard_range(db.shape[0], rank, world)
        res = {}
        for k in (1, 5):
            if k == 1:
                li, ls = oracle.search(db[lo:hi], q)
                li, ls = li[:, None], ls[:, None]
            else:
                li, ls = oracle.search_topk(db[lo:hi], q, k)
            gi, gs = gather_and_merge(torch.from_numpy(li), torch.from_numpy(ls), lo)
            res[k] = (gi.numpy(), gs.numpy())
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_exchange_equals_whole_database_oracle(world):
    import oracle
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = dict(out.get() for _ in range(world))
    db, q = _case()
    o1 = oracle.search(db, q)
    o5 = oracle.search_topk(db, q, 5)
    assert o1[0][0] == 10 and o1[0][1] == 1499 and o1[0][2] == 1000   # the planted ties
    for r in range(world):
        gi, gs = got[r][1]
        assert np.array_equal(gi[:, 0], o1[0]) and np.array_equal(gs[:, 0], o1[1])
        gi, gs = got[r][5]
        assert np.array_equal(gi, o5[0]) and np.array_equal(gs, o5[1])
