"""Failure detection without a GPU fault: every mbarrier wait in the
tensor-core GEMM update is bounded by the handle's wait budget. With the
budget cut to 1 microsecond the waits run out (the first accumulator of a
K = 1024 tile alone takes tens of microseconds), the kernel records
TRX_ERR_TIMEOUT in the handle's error word, drains what it has in flight,
frees its tensor memory and returns. The host reads the status; the context
stays usable and the next call with the normal budget is correct."""
import numpy as np
import pytest

from helpers import run_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import paper_2504_13821_gb300 as trx
    h = trx.Handle(0)
    h.set_option(trx.OPT_GEMM, trx.GEMM_TC)
    h.set_option(trx.OPT_GRAPH, 0)
    assert h.check_device_error() == 0
    h.set_option(trx.OPT_WAIT_LIMIT, 1000)            # 1 us
    run_case("trsm", "L", "L", "N", "N", 2048, 2048, 1.0, np.float32, seed=5,
             handle=h, check=False)                   # result invalid, must not hang
    assert h.check_device_error() == 4                # TRX_ERR_TIMEOUT
    assert h.check_device_error() == 0                # read-and-clear
    h.set_option(trx.OPT_WAIT_LIMIT, 2_000_000_000)
    run_case("trsm", "L", "L", "N", "N", 2048, 2048, 1.0, np.float32, seed=5, handle=h)
    assert h.check_device_error() == 0
    h.close()
