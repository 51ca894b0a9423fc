"""Helpers shared by the GPU parity tests (inputs, oracle results, comparisons)."""
import functools

import numpy as np
import torch

import hn_synth
import oracle


@functools.lru_cache(maxsize=4)
def oracle_case(n, nq, n_centres, seed, k, alpha, entry_noise=0.15, query_noise=0.10):
    """Raw inputs plus the oracle's normalised data and exact answers."""
    w = hn_synth.make_workload(n, nq, n_centres, seed, entry_noise, query_noise)
    db = oracle.normalize(w.db_raw, k, alpha)
    q = oracle.normalize(w.q_raw, k, alpha)
    idx, sim = oracle.search(db, q)
    return w, db, q, idx, sim


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_parity(res_idx, res_sim, o_idx, o_sim, tol=1e-6, exact_sim=True):
    gi = res_idx.cpu().numpy()
    gs = res_sim.cpu().numpy()
    mism = np.flatnonzero(gi != o_idx)
    assert mism.size == 0, f"{mism.size} index mismatches, first {mism[:5]}: gpu {gi[mism[:5]]} oracle {o_idx[mism[:5]]}"
    err = np.max(np.abs(gs - o_sim)) if gs.size else 0.0
    assert err <= tol, f"max |sim - oracle| = {err}"
    if exact_sim:
        assert np.array_equal(gs, o_sim), "similarities differ from the oracle's binary64 values"
