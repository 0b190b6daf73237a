"""Kernel attributes are per device: the library sets them in each device's
set-up (handle creation, the allocation-free entry), never lazily on the
first device used. On a second device, after the first one was used in the
same process, the calls whose kernels need a raised shared-memory limit
(the refined solve's residual, TRSM with tensor-core leaves, the thin and
device-scheduled solves, the tensor-core updates) must still launch and be
correct. Skipped on a box with one GPU.
"""
import numpy as np
import pytest

from helpers import run_case, to_dev
import oracle
from paper_2504_13821_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two GPUs")
def test_second_device_after_first():
    import paper_2504_13821_gb300 as trx
    run_case("trsm", "L", "L", "N", "N", 2048, 64, 1.0, np.float32, seed=1, device="cuda:0")
    for opts in ({}, {trx.OPT_TRSM_TC_LEAF: 1, trx.OPT_THIN: -1}, {trx.OPT_THIN: 1},
                 {trx.OPT_TRSM_DAG: 1, trx.OPT_THIN: -1}):
        h = trx.Handle(1)
        for o, v in opts.items():
            h.set_option(o, v)
        run_case("trsm", "L", "L", "N", "N", 2048, 64, 1.5, np.float32, seed=2, handle=h,
                 device="cuda:1")
        run_case("trmm", "R", "U", "T", "N", 300, 2048, 1.5, np.float32, seed=3, handle=h,
                 device="cuda:1")
        assert h.check_device_error() == 0
        h.close()
    k, n = 1024, 40
    A, B = inputs.problem("L", "L", k, n, seed=4, dtype=np.float32)
    with torch.cuda.device(1):
        h = trx.Handle(1)
        At, Bt = to_dev(A, "cuda:1"), to_dev(B, "cuda:1")
        X, _ = trx.trsm_refined("L", "L", "N", "N", 1.5, At, Bt, handle=h)
        torch.cuda.synchronize(1)
        eta = oracle.trsm_backward_error("L", "L", "N", "N", 1.5, A.astype(np.float64),
                                         np.asfortranarray(X.cpu().numpy()),
                                         B.astype(np.float64))["eta"]
        assert eta <= 8 * k * 2.0 ** -53
        h.close()
