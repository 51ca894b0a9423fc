"""Thin ctypes binding of libhn (include/hn.h).

Argument marshalling only: every step of normalisation, index packing and
search runs in the library's CUDA kernels.  PyTorch supplies device memory
and the current stream.  If libhn.so is missing this module raises on
import; build it with ``python paper_2606_27280_b300/build.py``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libhn.so")

OK, ERR_INVALID_ARG, ERR_NOT_NORMALIZED, ERR_ZERO_NORM, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_OVERFLOW, \
    ERR_UNSUPPORTED = range(9)
PREFIX_F32, PREFIX_BF16 = 0, 1
SCAN_AUTO, SCAN_STREAM, SCAN_DENSE = 0, 1, 2
D = 128

_STATUS_NAMES = {0: "HN_OK", 1: "HN_ERR_INVALID_ARG", 2: "HN_ERR_NOT_NORMALIZED", 3: "HN_ERR_ZERO_NORM",
                 4: "HN_ERR_OOM", 5: "HN_ERR_CUDA", 6: "HN_ERR_TIMEOUT", 7: "HN_ERR_OVERFLOW",
                 8: "HN_ERR_UNSUPPORTED"}


class IndexOpts(ctypes.Structure):
    _fields_ = [("prefix", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class SearchOpts(ctypes.Structure):
    _fields_ = [("scan", ctypes.c_int32), ("bucket_cap", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class SearchStats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("n_entries", ctypes.c_int64), ("survivors", ctypes.c_int64),
                ("max_survivors", ctypes.c_int64), ("fp64_rescored", ctypes.c_int64), ("reruns", ctypes.c_int32),
                ("scan", ctypes.c_int32), ("kernels", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms_prep", ctypes.c_float), ("ms_phase1", ctypes.c_float), ("ms_threshold", ctypes.c_float),
                ("ms_phase2", ctypes.c_float), ("ms_rescore", ctypes.c_float), ("ms_total", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("k", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("prefix", ctypes.c_int32), ("k_pad", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("minor_norm_max", ctypes.c_float), ("major_norm_max", ctypes.c_float),
                ("resid_norm_max", ctypes.c_float), ("prefix_norm_max", ctypes.c_float)]


# exported symbol -> (argtypes, restype); the ABI test checks these against include/hn.h
_vp, _i64, _i32, _f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
SIGNATURES = {
    "hn_version": ([], _i32),
    "hn_last_error": ([], ctypes.c_char_p),
    "hn_normalize": ([_vp, _vp, _i64, _i32, _i32, _f64, _vp], _i32),
    "hn_index_build": ([_vp, _i64, _i32, _i32, _f64, _vp, _vp, _vp], _i32),
    "hn_index_destroy": ([_vp], _i32),
    "hn_index_get_info": ([_vp, _vp], _i32),
    "hn_search_batch": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp], _i32),
    "hn_bruteforce": ([_vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "hn_bruteforce_static": ([_vp, _vp, _i64, _vp, _vp, _vp], _i32),
}
STATIC_MAX_QUERIES = 65536


def load_library(path: str = _LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libhn.so not found at {path}; build it with `python paper_2606_27280_b300/build.py`")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        try:
            fn = getattr(lib, name)
        except AttributeError as e:
            raise ImportError(f"{path} lacks {name}: rebuild with `python paper_2606_27280_b300/build.py`") from e
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = load_library()


class HNError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.hn_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, where: str) -> None:
    if status != OK:
        raise HNError(status, where)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != D:
        raise ValueError(f"{name} must be float32 of shape (n, {D})")
    return t.contiguous()


def version() -> tuple[int, int]:
    v = _lib.hn_version()
    return v >> 16, v & 0xFFFF


def normalize(x: torch.Tensor, k: int, alpha: float, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """HN normalisation (Eq. 1) of the rows of x on the GPU; returns out."""
    x = _dev_f32(x, "x")
    if out is None:
        out = torch.empty_like(x)
    _check(_lib.hn_normalize(x.data_ptr(), out.data_ptr(), x.shape[0], D, int(k), float(alpha), _stream(stream)),
           "hn_normalize")
    return out


@dataclass
class SearchResult:
    idx: torch.Tensor     # int64 [nq]
    sim: torch.Tensor     # float64 [nq]
    stats: dict | None


class Index:
    """Owning handle of an hn_index (device memory held by libhn)."""

    def __init__(self, x: torch.Tensor, k: int, alpha: float, prefix: int = PREFIX_F32, stream=None):
        x = _dev_f32(x, "x")
        self._h = ctypes.c_void_p()
        opts = IndexOpts(prefix=int(prefix))
        _check(_lib.hn_index_build(x.data_ptr(), x.shape[0], D, int(k), float(alpha), ctypes.byref(opts),
                                   ctypes.byref(self._h), _stream(stream)), "hn_index_build")
        self.k, self.alpha, self.prefix, self.n = int(k), float(alpha), int(prefix), x.shape[0]

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib.hn_index_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self) -> dict:
        inf = IndexInfo()
        _check(_lib.hn_index_get_info(self._h, ctypes.byref(inf)), "hn_index_get_info")
        return {name: getattr(inf, name) for name, _ in inf._fields_}

    def search(self, q: torch.Tensor, scan: int = SCAN_AUTO, bucket_cap: int = 0, stats: bool = False,
               timing: bool = False,
               out_idx: torch.Tensor | None = None, out_sim: torch.Tensor | None = None,
               stream=None) -> SearchResult:
        """Exact 1-NN of every row of q (HN-normalised, float32, device)."""
        q = _dev_f32(q, "q")
        nq = q.shape[0]
        if out_idx is None:
            out_idx = torch.empty(nq, dtype=torch.int64, device=q.device)
        if out_sim is None:
            out_sim = torch.empty(nq, dtype=torch.float64, device=q.device)
        opts = SearchOpts(scan=int(scan), bucket_cap=int(bucket_cap), timing=int(bool(timing)))
        st = SearchStats() if (stats or timing) else None
        _check(_lib.hn_search_batch(self._h, q.data_ptr(), nq, ctypes.byref(opts), out_idx.data_ptr(),
                                    out_sim.data_ptr(), ctypes.byref(st) if st is not None else None,
                                    _stream(stream)), "hn_search_batch")
        return SearchResult(out_idx, out_sim, st.as_dict() if st is not None else None)

    def bruteforce(self, q: torch.Tensor, stream=None) -> SearchResult:
        """FP32 128-dim brute force (baseline; ranks by FP32 scores)."""
        q = _dev_f32(q, "q")
        nq = q.shape[0]
        out_idx = torch.empty(nq, dtype=torch.int64, device=q.device)
        out_sim = torch.empty(nq, dtype=torch.float64, device=q.device)
        _check(_lib.hn_bruteforce(self._h, q.data_ptr(), nq, out_idx.data_ptr(), out_sim.data_ptr(),
                                  _stream(stream)), "hn_bruteforce")
        return SearchResult(out_idx, out_sim, None)
