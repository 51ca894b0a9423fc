"""Host logic of the N > 1 bench path on CPU: world_size-2 gloo ranks agree on the
slowest rank's time, and every rank gets its own query batch."""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(torch, 1.0 + 2.5 * rank, dist, "cpu")
        out.put((rank, t))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(out.get() for _ in range(2))
    assert got == {0: 3.5, 1: 3.5}


def test_single_process_time_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, 0.25, None, "cpu") == 0.25


def test_rank_batches_are_distinct_and_shaped_like_the_workload():
    sys.path.insert(0, ROOT)
    import bench
    import hn_synth
    wl, c = hn_synth.config_workload("c0")
    q0, q1, q2 = (bench.rank_queries(wl, c, r) for r in range(3))
    assert q0 is wl.q_raw
    assert q1.shape == q0.shape == q2.shape and q1.dtype == np.float32
    assert not np.array_equal(q0, q1) and not np.array_equal(q1, q2)
    assert np.array_equal(q1, bench.rank_queries(wl, c, 1))   # seeded
    # same distribution: a raw entry plus N(0, 0.1^2) noise per dimension, so the nearest raw
    # entry lies about 0.1 * sqrt(128) = 1.13 away
    d = np.linalg.norm(q1[:50, None, :] - wl.db_raw[None, :, :], axis=2).min(1)
    assert 0.9 < np.median(d) < 1.3
