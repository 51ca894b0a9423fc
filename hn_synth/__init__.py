"""Seeded synthetic descriptor generator (pre-normalisation feature vectors).

This module is shared by the CPU oracle, the CUDA path's tests and the
benchmark.  It produces *raw* feature vectors f (the input of Eq. 1, the
Hierarchical Normalization of §3.1) and nothing else: no normalisation, no
inner product, no search.  Each side applies its own HN normalisation.

Workload recipe (clustered stand-in for the paper's UBC patch descriptors,
§4 "Dataset"; D = 128 as for HardNet):

* ``n_centres`` cluster centres, each a standard-normal 128-vector scaled to
  unit length (uniform on the 128-sphere);
* database entry i = centre[c_i] + ``entry_noise`` * g_i, c_i uniform over the
  centres, g_i standard normal per dimension;
* query j = raw database entry e_j + ``query_noise`` * h_j, e_j uniform over
  the entries.

Randomness comes from numpy's counter-based Philox4x32-10 bit generator.
Every array is drawn from its own stream keyed by (seed, stream id, chunk), so
the bytes do not depend on the number of worker threads.  Values are float32.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

D = 128
_CHUNK = 1 << 16  # rows per independent Philox stream

# stream ids
_S_CENTRES, _S_ASSIGN, _S_ENTRY_NOISE, _S_QPICK, _S_QNOISE, _S_PERM = 1, 2, 3, 4, 5, 6


def _gen(seed: int, stream: int, chunk: int = 0) -> np.random.Generator:
    key = (int(seed) & 0xFFFFFFFF) | ((int(stream) & 0xFFFF) << 32) | ((int(chunk) & 0xFFFF) << 48)
    return np.random.Generator(np.random.Philox(key=key))


def _normal_rows(seed: int, stream: int, n: int, d: int = D) -> np.ndarray:
    """n x d float32 standard normals, drawn chunk by chunk from independent streams."""
    out = np.empty((n, d), dtype=np.float32)
    chunks = [(c, c * _CHUNK, min(n, (c + 1) * _CHUNK)) for c in range((n + _CHUNK - 1) // _CHUNK)]

    def fill(job):
        c, lo, hi = job
        _gen(seed, stream, c).standard_normal(out=out[lo:hi], dtype=np.float32)

    workers = min(len(chunks), os.cpu_count() or 1, 32)
    if workers <= 1:
        for j in chunks:
            fill(j)
    else:
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(fill, chunks))
    return out


@dataclass
class Workload:
    db_raw: np.ndarray       # (n, 128) float32, pre-normalisation entries
    q_raw: np.ndarray        # (nq, 128) float32, pre-normalisation queries
    centre_of: np.ndarray    # (n,) int64, generating centre of each entry
    source_of: np.ndarray    # (nq,) int64, database entry each query was drawn from


def centres(seed: int, n_centres: int) -> np.ndarray:
    c = _gen(seed, _S_CENTRES).standard_normal((n_centres, D))  # float64
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    return c.astype(np.float32)


def make_workload(n: int, nq: int, n_centres: int, seed: int,
                  entry_noise: float = 0.15, query_noise: float = 0.10) -> Workload:
    """Clustered raw descriptors: ``n`` database entries and ``nq`` queries."""
    if n < 1 or nq < 0 or n_centres < 1:
        raise ValueError("need n >= 1, nq >= 0, n_centres >= 1")
    cen = centres(seed, n_centres)
    centre_of = _gen(seed, _S_ASSIGN).integers(0, n_centres, size=n, dtype=np.int64)
    db = _normal_rows(seed, _S_ENTRY_NOISE, n)
    _add_scaled(db, cen, centre_of, np.float32(entry_noise))
    source_of = _gen(seed, _S_QPICK).integers(0, n, size=nq, dtype=np.int64)
    q = _normal_rows(seed, _S_QNOISE, nq) if nq else np.empty((0, D), np.float32)
    if nq:
        q *= np.float32(query_noise)
        q += db[source_of]
    return Workload(db, q, centre_of, source_of)


def _add_scaled(db: np.ndarray, cen: np.ndarray, centre_of: np.ndarray, s: np.float32) -> None:
    """db[i] <- cen[centre_of[i]] + s * db[i], in place, chunked to bound memory."""
    def work(lo):
        hi = min(len(db), lo + _CHUNK)
        blk = db[lo:hi]
        blk *= s
        blk += cen[centre_of[lo:hi]]

    starts = list(range(0, len(db), _CHUNK))
    workers = min(len(starts), os.cpu_count() or 1, 32)
    if workers <= 1:
        for lo in starts:
            work(lo)
    else:
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(work, starts))


def queries_from(db_raw: np.ndarray, nq: int, seed: int, query_noise: float = 0.10) -> tuple[np.ndarray, np.ndarray]:
    """nq raw queries drawn like make_workload's (a random raw entry plus noise), from
    streams of their own (e.g. training queries for the block proposal)."""
    src = _gen(seed, _S_QPICK + 32).integers(0, db_raw.shape[0], size=nq, dtype=np.int64)
    q = _normal_rows(seed, _S_QNOISE + 32, nq)
    q *= np.float32(query_noise)
    q += db_raw[src]
    return q, src


def uniform_queries(seed: int, nq: int) -> np.ndarray:
    """Unclustered standard-normal raw queries (no source entry), e.g. for training sets."""
    return _normal_rows(seed, _S_QNOISE + 16, nq)


def permutation(seed: int, n: int) -> np.ndarray:
    return _gen(seed, _S_PERM).permutation(n).astype(np.int64)


def log_uniform_sizes(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Batch sizes round(exp(U * ln(hi/lo))) * lo clamped to [lo, hi]."""
    u = _gen(seed, 7).random(count)
    s = np.rint(lo * np.exp(u * np.log(hi / lo))).astype(np.int64)
    return np.clip(s, lo, hi)


# Workload recipes: sizes, centre counts, prefix width K, energy split alpha, seed.
CONFIGS = {
    # plain FP32 branch-and-bound, small enough for the oracle in seconds
    "c0": dict(n=10_000, nq=1_000, n_centres=2_000, k=8, alpha=1 / 32, seed=0),
    # FP32 at the recommended operating point (K = 16, alpha = 1/8, §7)
    "c1": dict(n=1_000_000, nq=16_384, n_centres=200_000, k=16, alpha=1 / 8, seed=1),
    # reduced-precision prefix at N = 4M
    "c2": dict(n=4_000_000, nq=65_536, n_centres=800_000, k=16, alpha=1 / 8, seed=2),
    # c2's data with 4,096 blocks for the learned proposal (1M training pairs from seed 1003)
    "c3": dict(n=4_000_000, nq=65_536, n_centres=800_000, k=16, alpha=1 / 8, seed=2, n_blocks=4096,
               n_train=1_000_000, train_seed=1003),
}

# Batched serving: 256 batches of log-uniform size in [1, 4096] over four databases
# (N = 100k, 1M, 4M, 10M; centres N/5; seeds 1..4), each indexed for K in {8, 16} and
# alpha in {1/32, 1/8}; every batch picks one of the 16 indexes uniformly.
SERVING = dict(db_sizes=(100_000, 1_000_000, 4_000_000, 10_000_000), ks=(8, 16), alphas=(1 / 32, 1 / 8),
               n_batches=256, min_batch=1, max_batch=4096, seed=4)


def config_workload(name: str, n: int | None = None, nq: int | None = None) -> tuple[Workload, dict]:
    c = dict(CONFIGS[name])
    if n is not None:
        c["n_centres"] = max(1, c["n_centres"] * n // c["n"])
        c["n"] = n
    if nq is not None:
        c["nq"] = nq
    return make_workload(c["n"], c["nq"], c["n_centres"], c["seed"]), c
