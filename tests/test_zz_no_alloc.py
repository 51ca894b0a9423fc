"""hn_bruteforce_static, the allocation-free brute force, against hn_bruteforce.

Callers that cannot allocate device memory while serving queries (a
latency-critical thread, a fixed device-memory budget, an allocator owned by
another framework) use hn_bruteforce_static, whose only scratch is a fixed
array inside the library.  This file is collected last on purpose; it must
pass both on its own in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import hn_synth
import oracle

pytestmark = pytest.mark.gpu


def _static_call(hn, ix, q, nq=None):
    nq = q.shape[0] if nq is None else nq
    idx = torch.full((q.shape[0],), -7, dtype=torch.int64, device=q.device)
    sim = torch.full((q.shape[0],), -7.0, dtype=torch.float64, device=q.device)
    st = hn._lib.hn_bruteforce_static(ix._h, q.data_ptr(), nq, idx.data_ptr(), sim.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    return st, idx, sim


def test_static_bruteforce_matches_allocating_one(gpu):
    from paper_2606_27280_b300 import hn
    k, alpha = 16, 1 / 8
    w = hn_synth.make_workload(5000, 700, 600, seed=41)
    db = torch.from_numpy(oracle.normalize(w.db_raw, k, alpha)).cuda()
    q = torch.from_numpy(oracle.normalize(w.q_raw, k, alpha)).cuda()
    with hn.Index(db, k, alpha) as ix:
        ref = ix.bruteforce(q)
        torch.cuda.synchronize()
        # two calls in a row: the shared scratch keeps the first call's keys and
        # must be cleared by the second
        for _ in range(2):
            st, idx, sim = _static_call(hn, ix, q)
            torch.cuda.synchronize()
            assert st == hn.OK, hn._lib.hn_last_error()
            assert torch.equal(idx, ref.idx)
            assert np.max(np.abs(sim.cpu().numpy() - ref.sim.cpu().numpy())) <= 1e-6
        # a smaller batch after a larger one: stale keys past nq must not leak in
        st, idx, sim = _static_call(hn, ix, q[:37].contiguous())
        torch.cuda.synchronize()
        assert st == hn.OK
        assert torch.equal(idx, ref.idx[:37])


def test_static_bruteforce_rejects_oversized_batch(gpu):
    from paper_2606_27280_b300 import hn
    k, alpha = 8, 1 / 32
    w = hn_synth.make_workload(300, 4, 30, seed=42)
    db = torch.from_numpy(oracle.normalize(w.db_raw, k, alpha)).cuda()
    q = torch.from_numpy(oracle.normalize(w.q_raw, k, alpha)).cuda()
    with hn.Index(db, k, alpha) as ix:
        st, idx, _ = _static_call(hn, ix, q, nq=hn.STATIC_MAX_QUERIES + 1)
        assert st == hn.ERR_INVALID_ARG
        assert b"HN_STATIC_MAX_QUERIES" in hn._lib.hn_last_error()
        assert torch.all(idx == -7)   # nothing was written
