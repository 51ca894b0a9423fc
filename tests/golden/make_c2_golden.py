"""Write the binary64 oracle's exact 1-NN answer for every query of the c2 workload.

    python tests/golden/make_c2_golden.py [--threads T]

Workload c2 (N = 4,000,000 entries, Q = 65,536 queries, D = 128, K = 16,
alpha = 1/8, 800,000 centres, seed 2) is generated by ``hn_synth``; both the
entries and the queries are HN-normalised (Eq. 1) by ``oracle.normalize`` and
searched exhaustively by ``oracle.search`` (Theorem 1: the result of exhaustive
full-vector search; Theorem 2: the lowest index among equal maxima).  Nothing
here calls the CUDA library.

Output ``c2_oracle_nn.npz``:
  idx   int32[65536]   the oracle's index per query
  sim   float64[65536] its binary64 similarity
  db_sha256, q_sha256  sha256 of the raw (pre-normalisation) float32 bytes that
                       hn_synth produced, so a test can check that it regenerates
                       the same inputs before comparing
The run takes about an hour on 8 cores; it resumes from ``c2_oracle_nn.partial.npz``.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import hn_synth  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "c2_oracle_nn.npz")
PARTIAL = os.path.join(HERE, "c2_oracle_nn.partial.npz")
CHUNK = 2048


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8)).hexdigest()


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    wl, c = hn_synth.config_workload("c2")
    db_sha, q_sha = sha256(wl.db_raw), sha256(wl.q_raw)
    db = oracle.normalize(wl.db_raw, c["k"], c["alpha"])
    q = oracle.normalize(wl.q_raw, c["k"], c["alpha"])
    nq = q.shape[0]
    idx = np.full(nq, -1, np.int64)
    sim = np.full(nq, np.nan)
    done = 0
    if os.path.exists(PARTIAL):
        p = np.load(PARTIAL)
        if str(p["db_sha256"]) == db_sha and str(p["q_sha256"]) == q_sha:
            done = int(p["done"])
            idx[:done], sim[:done] = p["idx"][:done], p["sim"][:done]
    t0 = time.time()
    while done < nq:
        hi = min(nq, done + CHUNK)
        i, s = oracle.search(db, q[done:hi], nthreads=args.threads)
        idx[done:hi], sim[done:hi] = i, s
        done = hi
        np.savez(PARTIAL, idx=idx, sim=sim, done=done, db_sha256=db_sha, q_sha256=q_sha)
        print(f"{done}/{nq} queries, {time.time() - t0:.0f} s", flush=True)
    assert idx.min() >= 0 and idx.max() < c["n"]
    np.savez_compressed(OUT, idx=idx.astype(np.int32), sim=sim, db_sha256=db_sha, q_sha256=q_sha)
    os.remove(PARTIAL)
    print(f"wrote {OUT}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
