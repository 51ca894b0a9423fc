"""C-ABI checks that need no GPU: the library loads, exports every entry
point include/hn.h declares with the binding's signatures, and rejects bad
arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hn.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hn_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def hn():
    from paper_2606_27280_b300 import hn as mod
    return mod


def test_header_declares_api():
    fns = declared_functions()
    for name in ["hn_normalize", "hn_index_build", "hn_index_destroy", "hn_search_batch", "hn_bruteforce",
                 "hn_last_error", "hn_version", "hn_index_get_info"]:
        assert name in fns


def test_library_exports_every_declared_symbol(hn):
    lib = ctypes.CDLL(hn._LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(hn.SIGNATURES), "binding and header disagree"


def test_struct_sizes_match_header(hn):
    # sizes implied by the field lists in include/hn.h (x86-64 ABI)
    assert ctypes.sizeof(hn.IndexOpts) == 32
    assert ctypes.sizeof(hn.SearchOpts) == 64
    assert ctypes.sizeof(hn.SearchStats) == 96
    assert hn.SearchStats.passes.offset == 52
    assert ctypes.sizeof(hn.IndexInfo) == 64
    assert ctypes.sizeof(hn.TrainOpts) == 40
    assert ctypes.sizeof(hn.ProposalInfo) == 40
    assert ctypes.sizeof(hn.Batch) == 40
    assert ctypes.sizeof(hn.MultiOpts) == 32
    assert ctypes.sizeof(hn.MultiStats) == 56
    assert ctypes.sizeof(hn.TuneResult) == 288


def header_enums():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\b(HN_[A-Z0-9_]+)\s*=\s*(\d+)", text)}


def test_binding_constants_match_header_enums(hn):
    e = header_enums()
    pairs = {"HN_PREFIX_F32": hn.PREFIX_F32, "HN_PREFIX_BF16": hn.PREFIX_BF16, "HN_PREFIX_FP8_E4M3": hn.PREFIX_FP8,
             "HN_PREFIX_I8": hn.PREFIX_I8, "HN_SCAN_AUTO": hn.SCAN_AUTO, "HN_SCAN_STREAM": hn.SCAN_STREAM,
             "HN_SCAN_DENSE": hn.SCAN_DENSE, "HN_SCAN_DENSE_TWO_PASS": hn.SCAN_DENSE_TWO_PASS}
    for name, value in pairs.items():
        assert e[name] == value, name
    for code, name in hn._STATUS_NAMES.items():
        assert e[name] == code, name


def test_version(hn):
    assert hn.version() == (0, 1)


@pytest.mark.parametrize("d,k,alpha,status", [
    (64, 8, 0.1, 8),      # d != 128 -> unsupported
    (128, 0, 0.1, 1),     # k < 1
    (128, 128, 0.1, 1),   # k >= d
    (128, 8, 1.0, 1),     # alpha >= 1
    (128, 8, -0.5, 1),    # alpha < 0
])
def test_normalize_rejects_bad_dims_on_host(hn, d, k, alpha, status):
    assert hn._lib.hn_normalize(None, None, 10, d, k, alpha, None) == status
    assert hn._lib.hn_last_error() != b""


def test_index_k_limit(hn):
    h = ctypes.c_void_p()
    assert hn._lib.hn_index_build(ctypes.c_void_p(0x1000), 10, 128, 65, 0.1, None, ctypes.byref(h), None) == \
        hn.ERR_UNSUPPORTED
    # normalisation itself accepts any 1 <= k < 128 (it fails later only on the null pointer)
    assert hn._lib.hn_normalize(None, None, 10, 128, 127, 0.1, None) == hn.ERR_INVALID_ARG


def test_normalize_null_and_unaligned(hn):
    assert hn._lib.hn_normalize(None, None, 10, 128, 8, 0.1, None) == hn.ERR_INVALID_ARG
    assert hn._lib.hn_normalize(ctypes.c_void_p(0x1004), ctypes.c_void_p(0x2000), 10, 128, 8, 0.1, None) == \
        hn.ERR_INVALID_ARG
    assert hn._lib.hn_normalize(None, None, 0, 128, 8, 0.1, None) == hn.OK   # empty input: nothing to do
    assert hn._lib.hn_normalize(None, None, -1, 128, 8, 0.1, None) == hn.ERR_INVALID_ARG


def test_index_build_host_checks(hn):
    h = ctypes.c_void_p(123)
    assert hn._lib.hn_index_build(None, 10, 128, 8, 0.1, None, None, None) == hn.ERR_INVALID_ARG
    assert hn._lib.hn_index_build(None, 10, 128, 8, 0.1, None, ctypes.byref(h), None) == hn.ERR_INVALID_ARG
    assert h.value is None  # *out cleared on failure
    assert hn._lib.hn_index_build(ctypes.c_void_p(0x1000), 0, 128, 8, 0.1, None, ctypes.byref(h), None) == \
        hn.ERR_INVALID_ARG
    bad = hn.IndexOpts(prefix=4)   # one past HN_PREFIX_I8
    assert hn._lib.hn_index_build(ctypes.c_void_p(0x1000), 10, 128, 8, 0.1, ctypes.byref(bad), ctypes.byref(h),
                                  None) == hn.ERR_INVALID_ARG
    res = hn.IndexOpts(prefix=0)
    res.reserved[3] = 1
    assert hn._lib.hn_index_build(ctypes.c_void_p(0x1000), 10, 128, 8, 0.1, ctypes.byref(res), ctypes.byref(h),
                                  None) == hn.ERR_INVALID_ARG


def test_search_host_checks(hn):
    assert hn._lib.hn_search_batch(None, None, 4, None, None, None, None, None) == hn.ERR_INVALID_ARG
    assert hn._lib.hn_bruteforce(None, None, 4, None, None, None) == hn.ERR_INVALID_ARG
    assert hn._lib.hn_index_destroy(None) == hn.OK
    assert hn._lib.hn_index_get_info(None, None) == hn.ERR_INVALID_ARG
    assert hn._lib.hn_prefix_scores(None, None, 4, 0, None, None, None) == hn.ERR_INVALID_ARG


def test_multi_and_autotune_host_checks(hn):
    assert hn._lib.hn_search_multi(None, 3, None, None, None) == hn.ERR_INVALID_ARG
    assert hn._lib.hn_search_multi(None, 0, None, None, None) == hn.OK
    bad = (hn.Batch * 1)()
    assert hn._lib.hn_search_multi(bad, 1, None, None, None) == hn.ERR_INVALID_ARG   # NULL index
    assert hn._lib.hn_autotune(None, None, 1, None, None) == hn.ERR_INVALID_ARG


def test_python_wrappers_reject_cpu_tensors(hn):
    import torch
    with pytest.raises(TypeError):
        hn.normalize(torch.zeros(4, 128), 8, 0.1)


def test_selftest_rejects_bad_limit_on_host(hn):
    # argument checks happen before any device work
    assert hn._lib.hn_selftest_wait_timeout(10, None) == hn.ERR_INVALID_ARG
    assert hn._lib.hn_selftest_wait_timeout(20_000_000_000, None) == hn.ERR_INVALID_ARG
