"""The persistent CUDA-core FP32 TRSM and TRMM for thin right-hand sides
(TRX_OPT_THIN, csrc/thin.cu): 64-row blocks x 16-column panels; TRSM solved
left-looking in one launch, diagonal blocks by their inverses; TRMM summed
per block row from a packed copy of B. Against the FP64 oracle and the
recursive chain.

- all 16 variants at ragged orders (300, 1000) with 1, 17 and 64
  right-hand sides, alpha 1.5 / -2, padded lda / ldb (padding untouched):
  the normwise backward error within 8 k u of FP32, element by element
  through the oracle;
- forced on beyond the automatic range: order 40 (one block, rows past the
  order), 1024 with 200 right-hand sides (13 panels, a ragged last one);
- order 8192 with 16 right-hand sides (128 block rows): sampled columns
  against the oracle, bitwise repeatable, within the FP32 bound of the
  recursive chain; the default (automatic) mode takes this path;
- a bounded wait run out (the first block row withheld by the test hook,
  1 ms budget) is reported as TRX_ERR_TIMEOUT and the next call is correct;
- TRMM: all 16 variants at the same shapes (normwise error within 8 k u),
  order 40 and 1024 x 200 forced on, order 8192 with 16 right-hand sides
  against the oracle (sampled), bitwise repeatable, within the FP32 bound
  of the recursive product;
- thin solves as the recursion's leaves (TRX_OPT_THIN_LEAF) under
  tensor-core updates: all 16 variants at ragged orders (256-row leaves),
  order 8192 x 256 with 2048-row leaves sampled against the oracle,
  bitwise repeatable, within the FP32 bound of the ordinary recursion.
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


def thin_handle(trx, mode=1):
    h = trx.Handle(0)
    h.set_option(trx.OPT_THIN, mode)
    assert h.get_option(trx.OPT_THIN) == mode
    return h


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_thin_all_variants(trx, side, uplo, trans, diag):
    h = thin_handle(trx)
    vi = VARIANTS.index((side, uplo, trans, diag))
    for k, nrhs, alpha, pads in ((300, 1, 1.5, (0, 0)), (300, 17, -2.0, (3, 5)),
                                 (1000, 64, 1.5, (0, 7))):
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        run_case("trsm", side, uplo, trans, diag, m, n, alpha, np.float32,
                 seed=inputs.variant_seed(k + nrhs, vi), handle=h, lda_pad=pads[0],
                 ldb_pad=pads[1])
    assert h.check_device_error() == 0
    h.close()


def test_thin_forced_small_order_and_many_panels(trx):
    h = thin_handle(trx)
    run_case("trsm", "L", "U", "N", "U", 40, 9, 1.25, np.float32, seed=41, handle=h)
    run_case("trsm", "R", "L", "T", "N", 33, 40, -1.0, np.float32, seed=42, handle=h)
    run_case("trsm", "L", "L", "N", "N", 1024, 200, 1.5, np.float32, seed=43, handle=h)
    run_case("trsm", "R", "U", "T", "N", 200, 1024, 1.5, np.float32, seed=44, handle=h)
    assert h.check_device_error() == 0
    h.close()


def test_thin_large_order_sampled_repeatable_and_against_chain(trx):
    k, n = 8192, 16
    A, B = inputs.problem("L", "L", k, n, seed=8192, dtype=np.float32)
    At = to_dev(A, "cuda:0")
    h = trx.Handle(0)                                   # automatic: the thin solve
    outs = []
    for _ in range(2):
        Bt = to_dev(B, "cuda:0")
        trx.trsm("L", "L", "N", "N", 1.5, At, Bt, handle=h)
        outs.append(Bt)
    hc = thin_handle(trx, -1)
    Bc = to_dev(B, "cuda:0")
    trx.trsm("L", "L", "N", "N", 1.5, At, Bc, handle=hc)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]), "not bitwise repeatable"
    X = outs[0].cpu().numpy().astype(np.float64)
    Xc = Bc.cpu().numpy().astype(np.float64)
    ninf = lambda a: np.abs(a).sum(axis=1).max()          # noqa: E731
    assert ninf(X - Xc) <= bound(k, np.float32) * ninf(Xc)
    cols = np.array([0, 5, 11, 15])
    eta = oracle.trsm_backward_error("L", "L", "N", "N", 1.5, A.astype(np.float64),
                                     np.asfortranarray(X[:, cols]),
                                     np.asfortranarray(B[:, cols].astype(np.float64)))["eta"]
    assert eta <= bound(k, np.float32), eta
    assert h.check_device_error() == 0
    h.close()
    hc.close()


def test_thin_bounded_wait_reports_timeout(trx):
    from paper_2504_13821_gb300 import _binding
    h = thin_handle(trx)
    h.set_option(trx.OPT_GRAPH, 0)
    assert h.check_device_error() == 0
    h.set_option(trx.OPT_WAIT_LIMIT, 1_000_000)       # 1 ms
    h.set_option(_binding.OPT_TEST_WITHHOLD, 1)       # block row 0 is never published
    run_case("trsm", "L", "L", "N", "N", 4096, 16, 1.0, np.float32, seed=6, handle=h,
             check=False)
    assert h.check_device_error() == 4                # TRX_ERR_TIMEOUT
    assert h.check_device_error() == 0
    h.set_option(_binding.OPT_TEST_WITHHOLD, 0)
    h.set_option(trx.OPT_WAIT_LIMIT, 2_000_000_000)
    run_case("trsm", "L", "L", "N", "N", 4096, 16, 1.0, np.float32, seed=6, handle=h)
    assert h.check_device_error() == 0
    h.close()


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_thin_trmm_all_variants(trx, side, uplo, trans, diag):
    h = thin_handle(trx)
    vi = VARIANTS.index((side, uplo, trans, diag))
    for k, nrhs, alpha, pads in ((300, 1, 1.5, (0, 0)), (300, 17, -2.0, (3, 5)),
                                 (1000, 64, 1.5, (0, 7))):
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        run_case("trmm", side, uplo, trans, diag, m, n, alpha, np.float32,
                 seed=inputs.variant_seed(k + nrhs + 7, vi), handle=h, lda_pad=pads[0],
                 ldb_pad=pads[1])
    h.close()


def test_thin_trmm_forced_and_large(trx):
    h = thin_handle(trx)
    run_case("trmm", "L", "U", "N", "U", 40, 9, 1.25, np.float32, seed=51, handle=h)
    run_case("trmm", "R", "L", "T", "N", 200, 1024, -0.5, np.float32, seed=52, handle=h)
    h.close()
    k, n = 8192, 16
    A, B = inputs.problem("L", "U", k, n, seed=8193, dtype=np.float32)
    At = to_dev(A, "cuda:0")
    h = trx.Handle(0)                                   # automatic: the thin product
    outs = []
    for _ in range(2):
        Bt = to_dev(B, "cuda:0")
        trx.trmm("L", "U", "T", "N", 0.75, At, Bt, handle=h)
        outs.append(Bt)
    hc = thin_handle(trx, -1)
    Bc = to_dev(B, "cuda:0")
    trx.trmm("L", "U", "T", "N", 0.75, At, Bc, handle=hc)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]), "not bitwise repeatable"
    X = outs[0].cpu().numpy().astype(np.float64)
    Xc = Bc.cpu().numpy().astype(np.float64)
    ninf = lambda a: np.abs(a).sum(axis=1).max()          # noqa: E731
    A64 = np.triu(np.nan_to_num(A.astype(np.float64)))
    assert ninf(X - Xc) <= bound(k, np.float32) * ninf(A64) * ninf(B.astype(np.float64))
    cols = np.array([1, 8, 15])
    Bs = np.asfortranarray(B[:, cols].astype(np.float64))
    C_ref = oracle.trmm("L", "U", "T", "N", 0.75, A.astype(np.float64), Bs)
    err = oracle.trmm_error("L", "U", "T", "N", 0.75, A.astype(np.float64),
                            np.asfortranarray(X[:, cols]), C_ref, Bs)
    assert err <= bound(k, np.float32), err
    h.close()
    hc.close()


# ---- thin solves as the recursion's leaves (TRX_OPT_THIN_LEAF) -------------

def thin_leaf_handle(trx, rows):
    h = trx.Handle(0)
    h.set_option(trx.OPT_THIN, -1)
    h.set_option(trx.OPT_THIN_LEAF, rows)
    assert h.get_option(trx.OPT_THIN_LEAF) == rows
    return h


def test_thin_leaf_option_values(trx):
    h = trx.Handle(0)
    for bad in (-2, 1, 255, 300, 8320):
        with pytest.raises(trx.TrxError):
            h.set_option(trx.OPT_THIN_LEAF, bad)
    for ok in (-1, 0, 256, 2048, 8192):
        h.set_option(trx.OPT_THIN_LEAF, ok)
    h.close()


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_thin_leaves_all_variants(trx, side, uplo, trans, diag):
    """Leaves of 256 rows as thin solves under tensor-core updates: ragged
    orders (the last leaf shorter), padded storage, both alphas."""
    h = thin_leaf_handle(trx, 256)
    vi = VARIANTS.index((side, uplo, trans, diag))
    for k, nrhs, alpha, pads in ((1100, 40, 1.5, (0, 0)), (700, 130, -2.0, (3, 5))):
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        run_case("trsm", side, uplo, trans, diag, m, n, alpha, np.float32,
                 seed=inputs.variant_seed(k + nrhs + 7, vi), handle=h, lda_pad=pads[0],
                 ldb_pad=pads[1])
    assert h.check_device_error() == 0
    h.close()


def test_thin_leaves_large_sampled_repeatable(trx):
    """Order 8192, 256 right-hand sides, leaves of 2048 rows: sampled columns
    against the oracle, bitwise repeatable (graph replay included), within
    the FP32 bound of the ordinary recursion."""
    k, n = 8192, 256
    A, B = inputs.problem("L", "L", k, n, seed=8193, dtype=np.float32)
    At = to_dev(A, "cuda:0")
    h = thin_leaf_handle(trx, 2048)
    outs = []
    for _ in range(3):
        Bt = to_dev(B, "cuda:0")
        trx.trsm("L", "L", "N", "N", 1.5, At, Bt, handle=h)
        torch.cuda.synchronize()
        outs.append(Bt.cpu().numpy())
    assert h.check_device_error() == 0
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    X = np.asfortranarray(outs[0])
    cols = [0, 1, 100, 255]
    eta = oracle.trsm_backward_error("L", "L", "N", "N", 1.5, A.astype(np.float64),
                                     X[:, cols].astype(np.float64),
                                     np.asfortranarray(B[:, cols]).astype(np.float64))["eta"]
    assert eta <= bound(k, np.float32)
    h.close()
    hc = trx.Handle(0)
    hc.set_option(trx.OPT_THIN, -1)
    hc.set_option(trx.OPT_THIN_LEAF, -1)
    Bt = to_dev(B, "cuda:0")
    trx.trsm("L", "L", "N", "N", 1.5, At, Bt, handle=hc)
    torch.cuda.synchronize()
    Xc = Bt.cpu().numpy().astype(np.float64)
    hc.close()
    ninf = lambda a: np.abs(a).sum(axis=1).max()          # noqa: E731
    assert ninf(X.astype(np.float64) - Xc) <= bound(k, np.float32) * ninf(Xc)


def test_thin_precomputed_inverses_bitwise_equal(trx):
    """With several panels the diagonal blocks' inverses and Z are made once
    per block row by a separate pass (thin_prep_kernel); with one panel the
    task makes them. Same code, same values: the first 16 columns of a
    32-column solve equal a 16-column solve of those columns bitwise, and
    the last 8 of a 40-column solve (three panels) an 8-column one."""
    k = 1000
    A, B = inputs.problem("L", "L", k, 32, seed=1000, dtype=np.float32)
    At = to_dev(A, "cuda:0")
    h = thin_handle(trx)
    B32 = to_dev(B, "cuda:0")
    B16 = to_dev(np.asfortranarray(B[:, :16]), "cuda:0")
    trx.trsm("L", "L", "N", "N", 1.5, At, B32, handle=h)
    trx.trsm("L", "L", "N", "N", 1.5, At, B16, handle=h)
    # 40 columns: tasks over panel pairs, the last pair with one panel only
    A40, B40h = inputs.problem("L", "L", k, 40, seed=1001, dtype=np.float32)
    B40 = to_dev(B40h, "cuda:0")
    B8 = to_dev(np.asfortranarray(B40h[:, 32:]), "cuda:0")
    A40t = to_dev(A40, "cuda:0")
    trx.trsm("L", "L", "N", "N", -2.0, A40t, B40, handle=h)
    trx.trsm("L", "L", "N", "N", -2.0, A40t, B8, handle=h)
    torch.cuda.synchronize()
    assert h.check_device_error() == 0
    assert torch.equal(B32[:, :16], B16)
    assert torch.equal(B40[:, 32:], B8)
    h.close()
