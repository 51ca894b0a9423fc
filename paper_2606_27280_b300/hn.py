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
PREFIX_F32, PREFIX_BF16, PREFIX_FP8, PREFIX_I8 = 0, 1, 2, 3
SCAN_AUTO, SCAN_STREAM, SCAN_DENSE, SCAN_DENSE_TWO_PASS = 0, 1, 2, 3
RESCORE_FILTER16, RESCORE_BEST_FIRST, RESCORE_FULL = 0, 1, 2
D = 128

_STATUS_NAMES = {0: "HN_OK", 1: "HN_ERR_INVALID_ARG", 2: "HN_ERR_NOT_NORMALIZED", 3: "HN_ERR_ZERO_NORM",
                 4: "HN_ERR_OOM", 5: "HN_ERR_CUDA", 6: "HN_ERR_TIMEOUT", 7: "HN_ERR_OVERFLOW",
                 8: "HN_ERR_UNSUPPORTED"}


class IndexOpts(ctypes.Structure):
    _fields_ = [("prefix", ctypes.c_int32), ("n_blocks", ctypes.c_int32), ("kmeans_iters", ctypes.c_int32),
                ("seed", ctypes.c_uint32), ("reserved", ctypes.c_int32 * 4)]


class SearchOpts(ctypes.Structure):
    _fields_ = [("scan", ctypes.c_int32), ("bucket_cap", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("seed_topk", ctypes.c_int32), ("seed", ctypes.c_void_p), ("soft", ctypes.c_int32),
                ("beta", ctypes.c_float), ("scratch_limit", ctypes.c_int64), ("wait_limit_ns", ctypes.c_uint64),
                ("rescore", ctypes.c_int32), ("test_stall", ctypes.c_int32),
                ("test_plain_epilogue", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("hidden1", ctypes.c_int32), ("hidden2", ctypes.c_int32), ("epochs", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("seed", ctypes.c_uint32),
                ("init", ctypes.c_void_p), ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class ProposalInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("hidden1", ctypes.c_int32), ("hidden2", ctypes.c_int32),
                ("n_blocks", ctypes.c_int32), ("n_params", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("epochs", ctypes.c_int32), ("last_loss", ctypes.c_float)]


class SearchStats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("n_entries", ctypes.c_int64), ("survivors", ctypes.c_int64),
                ("max_survivors", ctypes.c_int64), ("fp64_rescored", ctypes.c_int64), ("reruns", ctypes.c_int32),
                ("scan", ctypes.c_int32), ("kernels", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("ms_prep", ctypes.c_float), ("ms_phase1", ctypes.c_float), ("ms_threshold", ctypes.c_float),
                ("ms_phase2", ctypes.c_float), ("ms_rescore", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("groups_scored", ctypes.c_int64), ("rescore_skipped", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("k", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("prefix", ctypes.c_int32), ("k_pad", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("minor_norm_max", ctypes.c_float), ("major_norm_max", ctypes.c_float),
                ("resid_norm_max", ctypes.c_float), ("prefix_norm_max", ctypes.c_float),
                ("n_blocks", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Batch(ctypes.Structure):
    _fields_ = [("index", ctypes.c_void_p), ("q", ctypes.c_void_p), ("nq", ctypes.c_int64),
                ("out_idx", ctypes.c_void_p), ("out_sim", ctypes.c_void_p)]


class MultiOpts(ctypes.Structure):
    _fields_ = [("use_graph", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class MultiStats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("n_batches", ctypes.c_int32), ("n_groups", ctypes.c_int32),
                ("graph_replayed", ctypes.c_int32), ("reruns", ctypes.c_int32), ("ms_total", ctypes.c_float),
                ("batch_ms_p50", ctypes.c_float), ("batch_ms_p99", ctypes.c_float), ("batch_ms_max", ctypes.c_float),
                ("joined", ctypes.c_int32), ("survivors", ctypes.c_int64)]


TUNE_MAX = 16


class TuneResult(ctypes.Structure):
    _fields_ = [("n_sizes", ctypes.c_int32), ("dense_min_q", ctypes.c_int32), ("units_per_cta", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("sizes", ctypes.c_int64 * TUNE_MAX),
                ("ms_stream", ctypes.c_float * TUNE_MAX), ("ms_dense", ctypes.c_float * TUNE_MAX),
                ("ms_units", ctypes.c_float * 4)]


# exported symbol -> (argtypes, restype); the ABI test checks these against include/hn.h
_vp, _i64, _i32, _f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
SIGNATURES = {
    "hn_version": ([], _i32),
    "hn_last_error": ([], ctypes.c_char_p),
    "hn_normalize": ([_vp, _vp, _i64, _i32, _i32, _f64, _vp], _i32),
    "hn_normalize_async": ([_vp, _vp, _i64, _i32, _i32, _f64, _vp, _vp], _i32),
    "hn_index_build": ([_vp, _i64, _i32, _i32, _f64, _vp, _vp, _vp], _i32),
    "hn_index_destroy": ([_vp], _i32),
    "hn_index_get_info": ([_vp, _vp], _i32),
    "hn_search_batch": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp], _i32),
    "hn_search_topk": ([_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "hn_bruteforce": ([_vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "hn_prefix_scores": ([_vp, _vp, _i64, _i32, _vp, _vp, _vp], _i32),
    "hn_merge_topk": ([_vp, _vp, _vp, _i32, _i64, _i32, _vp, _vp, _vp], _i32),
    "hn_merge_topk_host": ([_vp, _vp, _vp, _i32, _i64, _i32, _vp, _vp], _i32),
    "hn_index_blocks": ([_vp, _vp, _vp, _vp, _vp], _i32),
    "hn_search_multi": ([_vp, _i32, _vp, _vp, _vp], _i32),
    "hn_autotune": ([_vp, _vp, _i32, _vp, _vp], _i32),
    "hn_proposal_train": ([_vp, _vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "hn_proposal_infer": ([_vp, _vp, _i64, _i32, _vp, _vp], _i32),
    "hn_proposal_get_info": ([_vp, _vp], _i32),
    "hn_proposal_save": ([_vp, ctypes.c_char_p], _i32),
    "hn_proposal_load": ([ctypes.c_char_p, _vp], _i32),
    "hn_proposal_destroy": ([_vp], _i32),
    "hn_mlp_loss_grad": ([_vp, _i32, _i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _vp], _i32),
    "hn_mlp_loss_grad_bf16": ([_vp, _i32, _i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _vp], _i32),
    "hn_gemm_bf16": ([_i32, _i32, _i32, _vp, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _vp], _i32),
    "hn_linear_bf16": ([_vp, _i32, _i32, _vp, _i32, _vp, _i32, _vp, _vp], _i32),
    "hn_proposal_logits": ([_vp, _vp, _i64, _vp, _vp], _i32),
    "hn_bruteforce_static": ([_vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "hn_selftest_wait_timeout": ([ctypes.c_uint64, _vp], _i32),
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


def normalize_async(x: torch.Tensor, k: int, alpha: float, out: torch.Tensor | None = None,
                    status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """normalize() enqueued without synchronising the stream.  A bad row (non-finite, or a zero
    major / minor part) is copied unchanged, so a search of it raises HN_ERR_NOT_NORMALIZED;
    `status` (int32 [2] on the device, not cleared here) records such rows: [0] non-finite,
    [1] zero norm."""
    x = _dev_f32(x, "x")
    if out is None:
        out = torch.empty_like(x)
    sp = None
    if status is not None:
        if status.dtype != torch.int32 or not status.is_cuda or status.numel() < 2 or not status.is_contiguous():
            raise ValueError("status must be a contiguous int32 CUDA tensor of at least 2 elements")
        sp = status.data_ptr()
    _check(_lib.hn_normalize_async(x.data_ptr(), out.data_ptr(), x.shape[0], D, int(k), float(alpha), sp,
                                   _stream(stream)), "hn_normalize_async")
    return out


@dataclass
class SearchResult:
    idx: torch.Tensor     # int64 [nq]
    sim: torch.Tensor     # float64 [nq]
    stats: dict | None


class Index:
    """Owning handle of an hn_index (device memory held by libhn)."""

    def __init__(self, x: torch.Tensor, k: int, alpha: float, prefix: int = PREFIX_F32, n_blocks: int = 0,
                 kmeans_iters: int = 0, stream=None):
        x = _dev_f32(x, "x")
        self._h = ctypes.c_void_p()
        opts = IndexOpts(prefix=int(prefix), n_blocks=int(n_blocks), kmeans_iters=int(kmeans_iters))
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

    def autotune(self, sizes, stream=None) -> dict:
        """Time the streaming and dense scans at these batch sizes; the index keeps the choices."""
        sizes = [int(x) for x in sizes]
        arr = (ctypes.c_int64 * len(sizes))(*sizes)
        r = TuneResult()
        _check(_lib.hn_autotune(self._h, arr, len(sizes), ctypes.byref(r), _stream(stream)), "hn_autotune")
        n = r.n_sizes
        return {"dense_min_q": r.dense_min_q, "units_per_cta": r.units_per_cta, "sizes": list(r.sizes[:n]),
                "ms_stream": list(r.ms_stream[:n]), "ms_dense": list(r.ms_dense[:n]), "ms_units": list(r.ms_units)}

    def blocks(self, stream=None):
        """(block_start [B+1], block_ids [n], block_of [n]) int32 device tensors."""
        b = self.info()["n_blocks"]
        dev = torch.device("cuda", torch.cuda.current_device())
        start = torch.empty(b + 1, dtype=torch.int32, device=dev)
        ids = torch.empty(self.n, dtype=torch.int32, device=dev)
        of = torch.empty(self.n, dtype=torch.int32, device=dev)
        _check(_lib.hn_index_blocks(self._h, start.data_ptr(), ids.data_ptr(), of.data_ptr(), _stream(stream)),
               "hn_index_blocks")
        return start, ids, of

    def search(self, q: torch.Tensor, scan: int = SCAN_AUTO, bucket_cap: int = 0, stats: bool = False,
               timing: bool = False,
               out_idx: torch.Tensor | None = None, out_sim: torch.Tensor | None = None,
               proposal: "Proposal | None" = None, seed_topk: int = 0, beta: float | None = None,
               scratch_limit: int = 0, wait_limit_ns: int = 0, best_first: bool = False, rescore: int | None = None,
               test_stall: bool = False, test_plain_epilogue: bool = False, stream=None) -> SearchResult:
        """Exact 1-NN of every row of q (HN-normalised, float32, device).  With a trained
        `proposal`, its top `seed_topk` blocks give the threshold and Phase 1 is skipped.
        `beta` (0 <= beta <= alpha) selects the soft ANN mode: alpha in the skip test becomes
        beta (beta = alpha is exact).  `scratch_limit` caps the bytes of the dense scan's group
        map (larger batches run in passes); `wait_limit_ns` sets the dense scan's device-side
        wait limit (0 = 2 s).  `rescore` picks how Phase 2 scores the survivors (same result):
        RESCORE_FILTER16 (default) bounds each from its FP16 row and reads the FP32 row only where
        the bound reaches the best certified score; RESCORE_BEST_FIRST (also `best_first=True`)
        uses the FP32 prefix bound; RESCORE_FULL scores every survivor in FP32.  `test_stall`
        (failure-path tests only) withholds the scan's copies after each CTA's first work unit,
        so its waits run out after `wait_limit_ns` and the call raises HN_ERR_TIMEOUT.
        `test_plain_epilogue` (tests only) runs the one-pass scan's unsplit form, the fallback
        of a build without the register split (same result)."""
        q = _dev_f32(q, "q")
        nq = q.shape[0]
        if out_idx is None:
            out_idx = torch.empty(nq, dtype=torch.int64, device=q.device)
        if out_sim is None:
            out_sim = torch.empty(nq, dtype=torch.float64, device=q.device)
        opts = SearchOpts(scan=int(scan), bucket_cap=int(bucket_cap), timing=int(bool(timing)),
                          seed_topk=int(seed_topk), seed=proposal._h.value if proposal is not None else None,
                          soft=int(beta is not None), beta=float(beta) if beta is not None else 0.0,
                          scratch_limit=int(scratch_limit), wait_limit_ns=int(wait_limit_ns),
                          rescore=int(rescore) if rescore is not None else (RESCORE_BEST_FIRST if best_first else RESCORE_FILTER16),
                          test_stall=int(bool(test_stall)),
                          test_plain_epilogue=int(bool(test_plain_epilogue)))
        st = SearchStats() if (stats or timing) else None
        _check(_lib.hn_search_batch(self._h, q.data_ptr(), nq, ctypes.byref(opts), out_idx.data_ptr(),
                                    out_sim.data_ptr(), ctypes.byref(st) if st is not None else None,
                                    _stream(stream)), "hn_search_batch")
        return SearchResult(out_idx, out_sim, st.as_dict() if st is not None else None)

    def search_topk(self, q: torch.Tensor, k: int, scan: int = SCAN_AUTO, bucket_cap: int = 0,
                    stats: bool = False, rescore: int = RESCORE_FILTER16, stream=None) -> SearchResult:
        """Exact top-k of every row of q: idx / sim of shape (nq, k), by similarity
        descending then index ascending (rank 0 = the 1-NN).  `rescore`: RESCORE_FILTER16
        (FP16-row bound first) or RESCORE_FULL (every survivor in FP32); same result."""
        q = _dev_f32(q, "q")
        nq = q.shape[0]
        out_idx = torch.empty((nq, k), dtype=torch.int64, device=q.device)
        out_sim = torch.empty((nq, k), dtype=torch.float64, device=q.device)
        opts = SearchOpts(scan=int(scan), bucket_cap=int(bucket_cap), rescore=int(rescore))
        st = SearchStats() if stats else None
        _check(_lib.hn_search_topk(self._h, q.data_ptr(), nq, int(k), ctypes.byref(opts), out_idx.data_ptr(),
                                   out_sim.data_ptr(), ctypes.byref(st) if st is not None else None,
                                   _stream(stream)), "hn_search_topk")
        return SearchResult(out_idx, out_sim, st.as_dict() if st is not None else None)

    def prefix_scores(self, q: torch.Tensor, path: int, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        """(scores [nq, n] float32, slack [nq] float32): every prefix score as the search computes
        it (path 0: tensor-core scan, 1: CUDA-core FMA chain) and the slack E_q of its bound test."""
        q = _dev_f32(q, "q")
        nq = q.shape[0]
        scores = torch.empty((nq, self.n), dtype=torch.float32, device=q.device)
        slack = torch.empty(nq, dtype=torch.float32, device=q.device)
        _check(_lib.hn_prefix_scores(self._h, q.data_ptr(), nq, int(path), scores.data_ptr(), slack.data_ptr(),
                                     _stream(stream)), "hn_prefix_scores")
        return scores, slack

    def bruteforce(self, q: torch.Tensor, stream=None) -> SearchResult:
        """FP32 128-dim brute force (baseline; ranks by FP32 scores)."""
        q = _dev_f32(q, "q")
        nq = q.shape[0]
        out_idx = torch.empty(nq, dtype=torch.int64, device=q.device)
        out_sim = torch.empty(nq, dtype=torch.float64, device=q.device)
        _check(_lib.hn_bruteforce(self._h, q.data_ptr(), nq, out_idx.data_ptr(), out_sim.data_ptr(),
                                  _stream(stream)), "hn_bruteforce")
        return SearchResult(out_idx, out_sim, None)


class Proposal:
    """Owning handle of an hn_proposal: the learned block proposal MLP."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @classmethod
    def train(cls, index: Index, train_q: torch.Tensor, labels: torch.Tensor | None = None, hidden1: int = 0,
              hidden2: int = 0, epochs: int = 0, batch: int = 0, lr: float = 0.0, seed: int = 0,
              init: "Proposal | None" = None, precision: int = 0, stream=None) -> "Proposal":
        """precision 0: the training GEMMs on the tensor cores (BF16 operands, FP32 sums); 1: FP32
        CUDA-core GEMMs.  The master weights and Adam state are FP32 either way."""
        train_q = _dev_f32(train_q, "train_q")
        if labels is not None:
            if labels.dtype != torch.int32 or not labels.is_cuda or labels.numel() != train_q.shape[0]:
                raise ValueError("labels must be a CUDA int32 tensor with one entry per query")
            labels = labels.contiguous()
        opts = TrainOpts(hidden1=hidden1, hidden2=hidden2, epochs=epochs, batch=batch, lr=lr, seed=seed,
                         init=init._h.value if init is not None else None, precision=int(precision))
        h = ctypes.c_void_p()
        _check(_lib.hn_proposal_train(index._h, train_q.data_ptr(), labels.data_ptr() if labels is not None else None,
                                      train_q.shape[0], ctypes.byref(opts), ctypes.byref(h), _stream(stream)),
               "hn_proposal_train")
        return cls(h)

    @classmethod
    def load(cls, path: str) -> "Proposal":
        h = ctypes.c_void_p()
        _check(_lib.hn_proposal_load(str(path).encode(), ctypes.byref(h)), "hn_proposal_load")
        return cls(h)

    def save(self, path: str) -> None:
        _check(_lib.hn_proposal_save(self._h, str(path).encode()), "hn_proposal_save")

    def info(self) -> dict:
        inf = ProposalInfo()
        _check(_lib.hn_proposal_get_info(self._h, ctypes.byref(inf)), "hn_proposal_get_info")
        return {name: getattr(inf, name) for name, _ in inf._fields_}

    def infer(self, q: torch.Tensor, topk: int, stream=None) -> torch.Tensor:
        q = _dev_f32(q, "q")
        out = torch.empty((q.shape[0], topk), dtype=torch.int32, device=q.device)
        _check(_lib.hn_proposal_infer(self._h, q.data_ptr(), q.shape[0], int(topk), out.data_ptr(), _stream(stream)),
               "hn_proposal_infer")
        return out

    def logits(self, q: torch.Tensor, stream=None) -> torch.Tensor:
        """Block scores (nq, n_blocks) float32 as inference computes them (tensor cores, BF16 operands)."""
        q = _dev_f32(q, "q")
        out = torch.empty((q.shape[0], self.info()["n_blocks"]), dtype=torch.float32, device=q.device)
        _check(_lib.hn_proposal_logits(self._h, q.data_ptr(), q.shape[0], out.data_ptr(), _stream(stream)),
               "hn_proposal_logits")
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib.hn_proposal_destroy(self._h)
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


def mlp_loss_grad(params: torch.Tensor, dims, x: torch.Tensor, y: torch.Tensor, bf16: bool = False, stream=None):
    """(mean cross-entropy, gradient) of the proposal MLP, from the library's training kernels:
    FP32 CUDA-core GEMMs, or with `bf16` the tensor-core GEMMs (BF16 operands, FP32 sums)."""
    k, h1, h2, c = (int(v) for v in dims)
    params = params.contiguous()
    x = x.contiguous()
    y = y.contiguous()
    if params.dtype != torch.float32 or x.dtype != torch.float32 or y.dtype != torch.int32:
        raise TypeError("params/x float32, y int32")
    grads = torch.empty_like(params)
    loss = ctypes.c_float()
    fn = _lib.hn_mlp_loss_grad_bf16 if bf16 else _lib.hn_mlp_loss_grad
    _check(fn(params.data_ptr(), k, h1, h2, c, x.data_ptr(), y.data_ptr(), x.shape[0],
              ctypes.byref(loss), grads.data_ptr(), _stream(stream)), "hn_mlp_loss_grad")
    return loss.value, grads


def gemm_bf16(a: torch.Tensor, b: torch.Tensor, m: int, n: int, k: int, sai: int, sak: int, sbk: int, sbj: int,
              stream=None) -> torch.Tensor:
    """out[i, j] = sum_t bf16(a_flat[i*sai + t*sak]) * bf16(b_flat[t*sbk + j*sbj]) on the tensor cores
    (FP32 sums); a, b float32 CUDA tensors addressed through their flat storage; out (m, n)."""
    if a.dtype != torch.float32 or b.dtype != torch.float32 or not a.is_cuda or not b.is_cuda:
        raise TypeError("a and b: float32 CUDA tensors")
    a = a.contiguous()
    b = b.contiguous()
    if min(m, n, k) < 0 or min(sai, sak, sbk, sbj) < 0:
        raise ValueError("sizes and strides must be non-negative")
    if m and n and k:
        # the library reads a and b through these strides: keep every read inside the tensors
        if (m - 1) * sai + (k - 1) * sak >= a.numel() or (k - 1) * sbk + (n - 1) * sbj >= b.numel():
            raise ValueError("strides address elements outside a or b")
    out = torch.empty((m, n), dtype=torch.float32, device=a.device)
    _check(_lib.hn_gemm_bf16(int(m), int(n), int(k), a.data_ptr(), int(sai), int(sak), b.data_ptr(), int(sbk),
                             int(sbj), out.data_ptr(), int(n), _stream(stream)), "hn_gemm_bf16")
    return out


def linear_bf16(x: torch.Tensor, w: torch.Tensor, bias: torch.Tensor | None = None, act: int = 0,
                stream=None) -> torch.Tensor:
    """One fully connected layer on the tensor cores as proposal inference runs it:
    act(bf16(x) @ bf16(w).T + bias), FP32 accumulation; act 0 none, 1 GELU.  x (m, k), w (n, k)."""
    x = x.contiguous()
    w = w.contiguous()
    if x.dtype != torch.float32 or w.dtype != torch.float32 or not x.is_cuda or not w.is_cuda:
        raise TypeError("x and w: float32 CUDA tensors")
    if x.dim() != 2 or w.dim() != 2 or x.shape[1] != w.shape[1]:
        raise ValueError("x (m, k), w (n, k)")
    if bias is not None:
        bias = bias.contiguous()
        if bias.dtype != torch.float32 or bias.shape != (w.shape[0],):
            raise ValueError("bias: (n,) float32")
    out = torch.empty((x.shape[0], w.shape[0]), dtype=torch.float32, device=x.device)
    _check(_lib.hn_linear_bf16(x.data_ptr(), x.shape[0], x.shape[1], w.data_ptr(), w.shape[0],
                               bias.data_ptr() if bias is not None else None, int(act), out.data_ptr(),
                               _stream(stream)), "hn_linear_bf16")
    return out


def search_multi(batches, use_graph: bool = True, stream=None) -> dict:
    """Answer many batches in one call.  `batches`: list of (Index, q, out_idx, out_sim) with
    q a (nq, 128) float32 CUDA tensor and the outputs int64 / float64 CUDA tensors of nq
    entries.  Returns the call's statistics."""
    arr = (Batch * max(1, len(batches)))()
    keep = []
    for i, (ix, q, oi, os_) in enumerate(batches):
        q = _dev_f32(q, "q") if q.shape[0] else q
        keep.append(q)
        if oi.dtype != torch.int64 or os_.dtype != torch.float64 or oi.numel() != q.shape[0] or os_.numel() != q.shape[0]:
            raise ValueError("outputs must be int64 / float64 tensors of nq entries")
        arr[i] = Batch(index=ix._h.value, q=q.data_ptr() if q.numel() else None, nq=q.shape[0],
                       out_idx=oi.data_ptr() if oi.numel() else None, out_sim=os_.data_ptr() if os_.numel() else None)
    opts = MultiOpts(use_graph=int(bool(use_graph)))
    st = MultiStats()
    _check(_lib.hn_search_multi(arr, len(batches), ctypes.byref(opts), ctypes.byref(st), _stream(stream)),
           "hn_search_multi")
    return {name: getattr(st, name) for name, _ in st._fields_ if name != "reserved"}


def merge_topk(idx: torch.Tensor, sim: torch.Tensor, id_offset: torch.Tensor, stream=None):
    """Merge per-shard answers: idx int64 / sim float64 of shape (n_shards, nq, k) with
    shard-local indices, id_offset int64 (n_shards,), all on the device.  Returns the
    (nq, k) global answers in the order (similarity desc, index asc)."""
    if idx.dim() != 3 or sim.shape != idx.shape or id_offset.numel() != idx.shape[0]:
        raise ValueError("idx, sim: (n_shards, nq, k); id_offset: (n_shards,)")
    if idx.dtype != torch.int64 or sim.dtype != torch.float64 or id_offset.dtype != torch.int64:
        raise TypeError("idx and id_offset int64, sim float64")
    if not (idx.is_cuda and sim.is_cuda and id_offset.is_cuda):
        raise TypeError("merge_topk takes device tensors (merge_topk_host: numpy arrays)")
    r, nq, k = idx.shape
    idx, sim, id_offset = idx.contiguous(), sim.contiguous(), id_offset.contiguous()
    out_idx = torch.empty((nq, k), dtype=torch.int64, device=idx.device)
    out_sim = torch.empty((nq, k), dtype=torch.float64, device=idx.device)
    _check(_lib.hn_merge_topk(idx.data_ptr(), sim.data_ptr(), id_offset.data_ptr(), r, nq, k, out_idx.data_ptr(),
                              out_sim.data_ptr(), _stream(stream)), "hn_merge_topk")
    return out_idx, out_sim


def merge_topk_host(idx, sim, id_offset):
    """merge_topk on host (numpy) arrays, computed by the library's host merge."""
    import numpy as np
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    sim = np.ascontiguousarray(sim, dtype=np.float64)
    off = np.ascontiguousarray(id_offset, dtype=np.int64)
    if idx.ndim != 3 or sim.shape != idx.shape or off.size != idx.shape[0]:
        raise ValueError("idx, sim: (n_shards, nq, k); id_offset: (n_shards,)")
    r, nq, k = idx.shape
    out_idx = np.empty((nq, k), np.int64)
    out_sim = np.empty((nq, k), np.float64)
    _check(_lib.hn_merge_topk_host(idx.ctypes.data, sim.ctypes.data, off.ctypes.data, r, nq, k, out_idx.ctypes.data,
                                   out_sim.ctypes.data), "hn_merge_topk_host")
    return out_idx, out_sim


def selftest_wait_timeout(limit_ns: int, stream=None) -> int:
    """Run the bounded-wait self-test; returns the hn_status (HN_ERR_TIMEOUT = 6 is the
    expected outcome: the device-side wait gave up and the kernel returned)."""
    return int(_lib.hn_selftest_wait_timeout(int(limit_ns), _stream(stream)))
