"""Failure detection on the GPU without a fault: a device-side wait on a barrier
nothing arrives on gives up after its limit, the kernel returns, the host reads
HN_ERR_TIMEOUT, and the context keeps working."""
import time

import pytest

from tests._gpu_util import assert_parity, oracle_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hn(gpu):
    import paper_2606_27280_b300 as mod
    return mod


def test_bounded_wait_times_out_and_context_survives(hn):
    from paper_2606_27280_b300 import hn as binding
    t0 = time.perf_counter()
    st = hn.selftest_wait_timeout(50_000_000)   # 50 ms
    dt = time.perf_counter() - t0
    assert st == binding.ERR_TIMEOUT
    assert 0.04 < dt < 5.0
    # the context is still usable: an exact search right after
    w, db, q, o_idx, o_sim = oracle_case(3000, 200, 600, 81, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=1) as ix:
        for scan in (1, 2):
            r = ix.search(to_dev(q), scan=scan)
            assert_parity(r.idx, r.sim, o_idx, o_sim)


def test_repeated_timeouts(hn):
    from paper_2606_27280_b300 import hn as binding
    for _ in range(3):
        assert hn.selftest_wait_timeout(2_000_000) == binding.ERR_TIMEOUT


@pytest.mark.parametrize("prefix,scan", [(1, 2), (2, 2), (1, 3), (2, 3)])
def test_dense_scan_abort_and_drain(hn, prefix, scan):
    """test_stall makes each CTA's copy producer stop after its first work unit, so the MMA
    warps wait for a query copy that never comes: that wait runs out after wait_limit_ns
    (1 us), the CTA raises its abort flag, the other roles leave their loops, copies and MMAs
    still in flight drain (with the full 2 s limit), tensor memory is freed and the kernel
    returns.  Every such call reports HN_ERR_TIMEOUT, and an exact search right after, on
    the same index, is the oracle's.  Without the stall a 1 us limit may or may not run out
    under normal load; either way the call is exact or reports the timeout."""
    from paper_2606_27280_b300 import hn as binding
    # 60k entries and 700 queries: every CTA has several work units, so every CTA stalls
    w, db, q, o_idx, o_sim = oracle_case(60013, 700, 12000, 82, 16, 1 / 8)
    with hn.Index(to_dev(db), 16, 1 / 8, prefix=prefix) as ix:
        qd = to_dev(q)
        for _ in range(3):
            with pytest.raises(hn.HNError) as e:
                ix.search(qd, scan=scan, wait_limit_ns=1000, test_stall=True)
            assert e.value.status == binding.ERR_TIMEOUT, str(e.value)
            r = ix.search(qd, scan=scan)
            assert_parity(r.idx, r.sim, o_idx, o_sim)
        for _ in range(3):
            try:
                r = ix.search(qd, scan=scan, wait_limit_ns=1000)
            except hn.HNError as e:
                assert e.status == binding.ERR_TIMEOUT, str(e)
            else:
                assert_parity(r.idx, r.sim, o_idx, o_sim)
        r = ix.search(qd, scan=scan)
        assert_parity(r.idx, r.sim, o_idx, o_sim)
        for kw in (dict(wait_limit_ns=999),                          # below the documented range
                   dict(test_stall=True),                            # the stall needs a short limit
                   dict(test_stall=True, wait_limit_ns=20_000_000),
                   dict(test_stall=True, wait_limit_ns=1000, scan=1)):   # and a dense scan
            kw.setdefault("scan", scan)
            with pytest.raises(hn.HNError) as e:
                ix.search(qd, **kw)
            assert e.value.status == binding.ERR_INVALID_ARG
