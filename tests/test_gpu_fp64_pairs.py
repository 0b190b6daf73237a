"""FP64 TRMM in one float-float pass on the FP32 pipes (TRX_OPT_FP64_TRMM 1):
B := alpha op(A) B with A and B as float pairs, against the FP64 oracle.

- all 16 variants at orders 64 (the smallest the pass takes), 300 and 1000
  with ragged right-hand-side counts (1, 257, 64), alpha 1.5 / -2, padded
  lda / ldb (padding untouched): the normwise error within 8 k u of FP64,
  element by element through the oracle's triple-loop TRMM;
- order 4096 with 512 right-hand sides, sampled columns against the oracle;
- within the FP64 bound of the recursive DFMA product, bitwise repeatable;
- orders below 64 keep the DFMA product (same result as with the option
  off), and so does the mixed FP64 TRSM (TRX_OPT_FP64_TRSM) below 64;
  alpha = 0 zeroes B.
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


def pair_handle(trx, on=1):
    h = trx.Handle(0)
    h.set_option(trx.OPT_FP64_TRMM, on)
    assert h.get_option(trx.OPT_FP64_TRMM) == on
    return h


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_pair_trmm_all_variants(trx, side, uplo, trans, diag):
    h = pair_handle(trx)
    vi = VARIANTS.index((side, uplo, trans, diag))
    for k, nrhs, alpha, pads in ((64, 1, 1.5, (0, 0)), (300, 257, -2.0, (3, 5)),
                                 (1000, 64, 1.5, (0, 7))):
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        run_case("trmm", side, uplo, trans, diag, m, n, alpha, np.float64,
                 seed=inputs.variant_seed(k + nrhs, vi), handle=h, lda_pad=pads[0],
                 ldb_pad=pads[1])
    assert h.check_device_error() == 0
    h.close()


def test_pair_trmm_large_sampled_and_against_dfma(trx):
    k, n = 4096, 512
    A, B = inputs.problem("L", "U", k, n, seed=4096, dtype=np.float64)
    At = to_dev(A, "cuda:0")
    h, hd = pair_handle(trx), pair_handle(trx, 0)
    outs = []
    for _ in range(2):
        Bt = to_dev(B, "cuda:0")
        trx.trmm("L", "U", "T", "N", -0.75, At, Bt, handle=h)
        outs.append(Bt)
    Bd = to_dev(B, "cuda:0")
    trx.trmm("L", "U", "T", "N", -0.75, At, Bd, handle=hd)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]), "not bitwise repeatable"
    X, Xd = outs[0].cpu().numpy(), Bd.cpu().numpy()
    cols = np.sort(np.random.default_rng(3).choice(n, size=16, replace=False))
    Bs = np.asfortranarray(B[:, cols])
    C_ref = oracle.trmm("L", "U", "T", "N", -0.75, A, Bs)
    e = oracle.trmm_error("L", "U", "T", "N", -0.75, A, np.asfortranarray(X[:, cols]), C_ref, Bs)
    assert e <= bound(k, np.float64), e
    # against the DFMA product: |X - Xd| within the bound of |A| |B| (inf norms)
    ninf = lambda a: np.abs(a).sum(axis=1).max()          # noqa: E731
    assert ninf(X - Xd) <= bound(k, np.float64) * ninf(np.triu(A)) * ninf(B)
    assert h.check_device_error() == 0
    h.close()
    hd.close()


def test_pair_trmm_small_orders_and_alpha_zero(trx):
    h, hd = pair_handle(trx), pair_handle(trx, 0)
    A, B = inputs.problem("R", "L", 20, 40, seed=8, dtype=np.float64)
    At = to_dev(A, "cuda:0")
    B1, B2 = to_dev(B, "cuda:0"), to_dev(B, "cuda:0")
    trx.trmm("R", "L", "N", "U", 1.25, At, B1, handle=h)     # order 40 < 64: DFMA
    trx.trmm("R", "L", "N", "U", 1.25, At, B2, handle=hd)
    torch.cuda.synchronize()
    assert torch.equal(B1, B2)
    A, B = inputs.problem("L", "L", 128, 9, seed=9, dtype=np.float64)
    Bt = to_dev(B, "cuda:0")
    trx.trmm("L", "L", "N", "N", 0.0, to_dev(A, "cuda:0"), Bt, handle=h)
    torch.cuda.synchronize()
    assert not Bt.any()
    h.close()
    hd.close()


def test_mixed_fp64_trsm_keeps_dfma_below_order_64(trx):
    h = trx.Handle(0)
    h.set_option(trx.OPT_FP64_TRSM, 2)
    hd = trx.Handle(0)
    A, B = inputs.problem("L", "U", 40, 300, seed=10, dtype=np.float64)
    At = to_dev(A, "cuda:0")
    B1, B2 = to_dev(B, "cuda:0"), to_dev(B, "cuda:0")
    trx.trsm("L", "U", "T", "N", 0.5, At, B1, handle=h)
    trx.trsm("L", "U", "T", "N", 0.5, At, B2, handle=hd)
    torch.cuda.synchronize()
    assert torch.equal(B1, B2)
    h.close()
    hd.close()
