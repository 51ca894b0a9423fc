"""Every query of the c2 workload (N = 4,000,000, Q = 65,536, K = 16, alpha = 1/8)
against the binary64 oracle's stored answers.

tests/golden/c2_oracle_nn.npz was written by tests/golden/make_c2_golden.py, which
calls only oracle/ (exhaustive search, Theorem 1; lowest index on ties, Theorem 2)
on the inputs hn_synth generates.  The test regenerates the same raw inputs (their
sha256 must match the file's), normalises and searches them on the GPU through the
C ABI, and compares all 65,536 indices (exactly) and similarities (bit for bit, so
also within the 1e-6 the method requires) for the BF16 and FP8 prefixes, in both
dense forms, at the launch configuration bench.py times.
"""
import hashlib
import os

import numpy as np
import pytest
import torch

import hn_synth
from tests._gpu_util import to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_oracle_nn.npz")


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


@pytest.fixture(scope="module")
def c2(hn):
    g = np.load(GOLDEN)
    wl, c = hn_synth.config_workload("c2")
    assert hashlib.sha256(wl.db_raw.view(np.uint8)).hexdigest() == str(g["db_sha256"]), "c2 entries changed"
    assert hashlib.sha256(wl.q_raw.view(np.uint8)).hexdigest() == str(g["q_sha256"]), "c2 queries changed"
    db = hn.normalize(to_dev(wl.db_raw), c["k"], c["alpha"])
    q = hn.normalize(to_dev(wl.q_raw), c["k"], c["alpha"])
    return db, q, c, g["idx"].astype(np.int64), g["sim"]


@pytest.mark.parametrize("prefix", [1, 2])
def test_c2_every_query_equals_oracle(hn, c2, prefix):
    db, q, c, o_idx, o_sim = c2
    with hn.Index(db, c["k"], c["alpha"], prefix=prefix) as ix:
        for scan in (hn.SCAN_DENSE, hn.SCAN_DENSE_TWO_PASS):
            r = ix.search(q, scan=scan, stats=True)
            gi, gs = r.idx.cpu().numpy(), r.sim.cpu().numpy()
            bad = np.flatnonzero(gi != o_idx)
            assert bad.size == 0, f"scan {scan}: {bad.size} of {len(gi)} indices differ, first {bad[:5]}"
            assert np.max(np.abs(gs - o_sim)) <= 1e-6
            assert np.array_equal(gs, o_sim), f"scan {scan}: similarities differ from the oracle's binary64 values"
            assert r.stats["n_queries"] == 65536
