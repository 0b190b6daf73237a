"""The device-scheduled FP32 TRSM (TRX_OPT_TRSM_DAG, csrc/trsm_dag.cu): the
recursion's blocks as one persistent launch (128-row blocks x 64-column
panels taken in order from a counter; off-diagonal products as soon as
the blocks they need are published; diagonal blocks solved by products
with their inverses), against the FP64 oracle and the recursive chain.

- all 16 variants, orders 256 and 1024, right-hand-side counts off the
  64-column panel (1, 70, 300) and at the automatic limit (1024), alpha
  1.5 / -2; the normwise backward error bound 8 k u of the problem
  statement, element by element through the oracle;
- the 6-term (FP32-grade) and 3-term splits;
- order 16384 with 256 right-hand sides (the thin benchmark shape),
  sampled columns against the oracle;
- bitwise repeatable run to run; results within the FP32 bound of the
  recursive chain's;
- a bounded wait run out (1 microsecond budget) is reported as
  TRX_ERR_TIMEOUT and the next call with the normal budget is correct.
"""
import numpy as np
import pytest

from helpers import bound, run_case, to_dev
import oracle
from paper_2504_13821_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = inputs.VARIANTS


@pytest.fixture(scope="module")
def trx():
    import paper_2504_13821_gb300 as trx
    return trx


def dag_handle(trx, terms=0):
    h = trx.Handle(0)
    h.set_option(trx.OPT_TRSM_DAG, 1)
    if terms:
        h.set_option(trx.OPT_SPLIT, terms)
    return h


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_dag_all_variants(trx, side, uplo, trans, diag):
    h = dag_handle(trx)
    vi = VARIANTS.index((side, uplo, trans, diag))
    for k, nrhs, alpha in ((256, 1, 1.5), (1024, 70, -2.0), (1024, 300, 1.5)):
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        run_case("trsm", side, uplo, trans, diag, m, n, alpha, np.float32,
                 seed=inputs.variant_seed(k + nrhs, vi), handle=h)
    h.close()


@pytest.mark.parametrize("terms", [6, 3])
def test_dag_splits_and_panel_limit(trx, terms):
    h = dag_handle(trx, terms)
    run_case("trsm", "L", "L", "N", "N", 2048, 1024, 1.5, np.float32, seed=31, handle=h)
    run_case("trsm", "R", "U", "N", "N", 640, 1280, 1.0, np.float32, seed=32, handle=h)
    h.close()


def test_dag_matches_chain_and_repeats(trx):
    k, n = 4096, 200
    A, B = inputs.problem("L", "L", k, n, seed=33, dtype=np.float32, scale=40.0)
    At = to_dev(A, "cuda:0")
    outs = []
    h = dag_handle(trx)
    for _ in range(2):
        Bt = to_dev(B, "cuda:0")
        trx.trsm("L", "L", "N", "N", 1.5, At, Bt, handle=h)
        outs.append(Bt)
    hc = trx.Handle(0)
    hc.set_option(trx.OPT_TRSM_DAG, -1)
    Bc = to_dev(B, "cuda:0")
    trx.trsm("L", "L", "N", "N", 1.5, At, Bc, handle=hc)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]), "not bitwise repeatable"
    X = outs[0].cpu().numpy().astype(np.float64)
    Xc = Bc.cpu().numpy().astype(np.float64)
    ninf = lambda a: np.abs(a).sum(axis=1).max()          # noqa: E731
    assert ninf(X - Xc) <= bound(k, np.float32) * ninf(Xc)
    eta = oracle.trsm_backward_error("L", "L", "N", "N", 1.5, A, np.asfortranarray(X), B)["eta"]
    assert eta <= bound(k, np.float32)
    h.close()
    hc.close()


def test_dag_thin_benchmark_shape_sampled(trx):
    k, n = 16384, 256
    A, B = inputs.problem("L", "L", k, n, seed=16384, dtype=np.float32)
    h = dag_handle(trx)
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    trx.trsm("L", "L", "N", "N", 1.5, At, Bt, handle=h)
    torch.cuda.synchronize()
    cols = np.sort(np.random.default_rng(5).choice(n, size=16, replace=False))
    X = np.asfortranarray(Bt.cpu().numpy()[:, cols].astype(np.float64))
    Bs = np.asfortranarray(B[:, cols].astype(np.float64))
    eta = oracle.trsm_backward_error("L", "L", "N", "N", 1.5, A.astype(np.float64), X, Bs)["eta"]
    assert eta <= bound(k, np.float32), eta
    assert h.check_device_error() == 0
    h.close()


def test_dag_bounded_wait_reports_timeout(trx):
    h = dag_handle(trx)
    h.set_option(trx.OPT_GRAPH, 0)
    assert h.check_device_error() == 0
    h.set_option(trx.OPT_WAIT_LIMIT, 1000)            # 1 us: the waits run out
    run_case("trsm", "L", "L", "N", "N", 4096, 256, 1.0, np.float32, seed=5, handle=h,
             check=False)
    assert h.check_device_error() == 4                # TRX_ERR_TIMEOUT
    assert h.check_device_error() == 0
    h.set_option(trx.OPT_WAIT_LIMIT, 2_000_000_000)
    run_case("trsm", "L", "L", "N", "N", 4096, 256, 1.0, np.float32, seed=5, handle=h)
    assert h.check_device_error() == 0
    h.close()
