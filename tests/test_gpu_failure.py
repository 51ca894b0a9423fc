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
