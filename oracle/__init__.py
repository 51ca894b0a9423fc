"""CPU oracle for exact HN 1-NN search -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never imports, links or calls
it, and this package imports nothing from the CUDA library.

``hn_oracle.c`` holds the arithmetic (binary64, sequential summation order);
this module compiles it with gcc on first use and exposes numpy wrappers.
``mlp.py`` holds the binary64 oracle of the learned block proposal.

Pins (tests/test_oracle_*.py) tie these functions to what the paper and the
mathematics fix: closed-form normalisation cases, the norm identities below
Eq. 1, the bound of Eq. 3 on every pair, Theorem 1 (two-phase = exhaustive),
the tie rule of Theorem 2, the alpha = 0 reduction, exact rational arithmetic
on small-integer inputs, and an independent float64 matrix product.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None

OK, BAD_ARG, ZERO_NORM = 0, 1, 3


def _cpu_has(*flags: str) -> bool:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("flags"):
                    have = set(line.split(":", 1)[1].split())
                    return all(fl in have for fl in flags)
    except OSError:
        pass
    return False


def _variant() -> tuple[str, list[str]]:
    if _cpu_has("avx2", "fma", "bmi2"):
        return "liboracle_v3.so", ["-march=x86-64-v3"]
    return "liboracle.so", []


def build(force: bool = False) -> str:
    """Compile hn_oracle.c (gcc -O3 -fopenmp, no fast-math); return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    name, march = _variant()
    out = os.path.join(_BUILD, name)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O3", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               *march, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, i32, f64, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            L.hno_normalize.argtypes = [vp, vp, i64, i32, i32, f64, vp]
            L.hno_normalize.restype = i32
            L.hno_part_norms2.argtypes = [vp, i64, i32, i32, vp, vp]
            L.hno_part_norms2.restype = None
            L.hno_dot.argtypes = [vp, vp, i32]
            L.hno_dot.restype = f64
            L.hno_sims.argtypes = [vp, i64, vp, i32, vp]
            L.hno_sims.restype = None
            L.hno_search.argtypes = [vp, i64, vp, i64, i32, vp, vp, i32]
            L.hno_search.restype = i32
            L.hno_search_topk.argtypes = [vp, i64, vp, i64, i32, i32, vp, vp, i32]
            L.hno_search_topk.restype = i32
            L.hno_two_phase.argtypes = [vp, i64, vp, i64, i32, i32, f64, i32, vp, vp, vp]
            L.hno_two_phase.restype = i32
            _lib = L
    return _lib


def _f32(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("expected a 2-D array")
    return a


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleError(RuntimeError):
    def __init__(self, status: int, row: int = -1):
        super().__init__(f"oracle status {status} (row {row})")
        self.status, self.row = status, row


def normalize(raw, k: int, alpha: float) -> np.ndarray:
    """Eq. 1 applied row by row (binary64 arithmetic, binary32 result)."""
    raw = _f32(raw)
    out = np.empty_like(raw)
    bad = ctypes.c_int64(-1)
    st = lib().hno_normalize(_p(raw), _p(out), raw.shape[0], raw.shape[1], k, float(alpha),
                             ctypes.addressof(bad))
    if st != OK:
        raise OracleError(st, bad.value)
    return out


def part_norms2(x, k: int) -> tuple[np.ndarray, np.ndarray]:
    x = _f32(x)
    a = np.empty(x.shape[0]); b = np.empty(x.shape[0])
    lib().hno_part_norms2(_p(x), x.shape[0], x.shape[1], k, _p(a), _p(b))
    return a, b


def dot(a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    b = np.ascontiguousarray(b, dtype=np.float32).ravel()
    if a.shape != b.shape:
        raise ValueError("shape mismatch")
    return lib().hno_dot(_p(a), _p(b), a.size)


def sims(db, q) -> np.ndarray:
    """All similarities of one query q against db (binary64, sequential order)."""
    db = _f32(db)
    q = np.ascontiguousarray(q, dtype=np.float32).ravel()
    out = np.empty(db.shape[0])
    lib().hno_sims(_p(db), db.shape[0], _p(q), db.shape[1], _p(out))
    return out


def search(db, q, nthreads: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Exact 1-NN: (index int64, similarity float64) per query, lowest index on ties."""
    db, q = _f32(db), _f32(q)
    if db.shape[1] != q.shape[1]:
        raise ValueError("dimension mismatch")
    idx = np.empty(q.shape[0], np.int64)
    sim = np.empty(q.shape[0], np.float64)
    st = lib().hno_search(_p(db), db.shape[0], _p(q), q.shape[0], db.shape[1], _p(idx), _p(sim),
                          int(nthreads))
    if st != OK:
        raise OracleError(st)
    return idx, sim


def search_topk(db, q, topk: int, nthreads: int = 0) -> tuple[np.ndarray, np.ndarray]:
    db, q = _f32(db), _f32(q)
    idx = np.empty((q.shape[0], topk), np.int64)
    sim = np.empty((q.shape[0], topk), np.float64)
    st = lib().hno_search_topk(_p(db), db.shape[0], _p(q), q.shape[0], db.shape[1], int(topk),
                               _p(idx), _p(sim), int(nthreads))
    if st != OK:
        raise OracleError(st)
    return idx, sim


def two_phase(db, q, k: int, alpha: float, literal_bound: bool = False):
    """Algorithm 1; returns (index, similarity, number of Phase-2 full evaluations)."""
    db, q = _f32(db), _f32(q)
    idx = np.empty(q.shape[0], np.int64)
    sim = np.empty(q.shape[0], np.float64)
    nfull = ctypes.c_int64(0)
    st = lib().hno_two_phase(_p(db), db.shape[0], _p(q), q.shape[0], db.shape[1], k, float(alpha),
                             int(bool(literal_bound)), _p(idx), _p(sim), ctypes.addressof(nfull))
    if st != OK:
        raise OracleError(st)
    return idx, sim, nfull.value
