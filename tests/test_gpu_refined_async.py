"""Refinement with a fixed number of corrections and no host read-back
(trx_strsm_refined_async) and the mixed FP64 TRSM engine built on it
(TRX_OPT_FP64_TRSM), against the FP64 oracle.

- FP32 data: the FP32 solve plus two float-float corrections reaches the
  backward error of an FP64 solve, eta <= 8 k 2^-53, on factors with
  kappa_1 about 1e2 and 1e4 (stored scales at order 1024, and the default
  generator at ragged orders), all 16 variants; zero corrections is an
  FP32-grade solve (8 k 2^-24); runs are bitwise repeatable.
- FP64 data through the mixed engine (FP32 solve on fl32(A), residual with
  A and X as float pairs): trx_dtrsm's result meets the FP64 bound
  8 k 2^-53 on every variant at orders 64 .. 700, in place in B, padding
  untouched; alpha = 0 and empty problems behave as the BLAS call.
"""
import json
import os

import numpy as np
import pytest

from helpers import SENTINEL, to_dev
import oracle
from paper_2504_13821_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
VARIANTS = inputs.VARIANTS


@pytest.fixture(scope="module")
def trx():
    import paper_2504_13821_gb300 as trx
    return trx


def _stored(k, kappa):
    path = os.path.join(os.path.dirname(__file__), "golden", "condition_scales.json")
    with open(path) as f:
        for e in json.load(f)["entries"]:
            if e["k"] == k and e["target"] == kappa:
                return e["scale"], e["seed"]
    raise KeyError((k, kappa))


@pytest.mark.parametrize("kappa", [1e2, 1e4])
def test_async_two_corrections_reach_fp64_level(trx, kappa):
    k, n = 1024, 96
    scale, seed = _stored(k, kappa)
    A, B = inputs.problem("L", "L", k, n, seed=seed, dtype=np.float32, scale=scale)
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    X = trx.trsm_refined_async("L", "L", "N", "N", 1.5, At, Bt, corrections=2)
    X2 = trx.trsm_refined_async("L", "L", "N", "N", 1.5, At, Bt, corrections=2)
    torch.cuda.synchronize()
    assert torch.equal(X, X2), "not bitwise repeatable"
    Xh = np.asfortranarray(X.cpu().numpy())
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    eta = oracle.trsm_backward_error("L", "L", "N", "N", 1.5, A64, Xh, B64)["eta"]
    assert eta <= 8 * k * U64, eta
    assert np.array_equal(Bt.cpu().numpy(), B), "B modified"


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_async_all_variants(trx, side, uplo, trans, diag):
    m, n = (300, 70) if side == "L" else (70, 300)
    k = m if side == "L" else n
    vi = VARIANTS.index((side, uplo, trans, diag))
    A, B = inputs.problem(side, uplo, m, n, seed=inputs.variant_seed(k, vi) + 7,
                          dtype=np.float32, scale=20.0, poison_diag=(diag == "U"))
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    X = trx.trsm_refined_async(side, uplo, trans, diag, -0.75, At, Bt, corrections=2)
    X0 = trx.trsm_refined_async(side, uplo, trans, diag, -0.75, At, Bt, corrections=0)
    torch.cuda.synchronize()
    A64 = A.astype(np.float64)
    eta = oracle.trsm_backward_error(side, uplo, trans, diag, -0.75, A64,
                                     np.asfortranarray(X.cpu().numpy()), B.astype(np.float64))["eta"]
    assert eta <= 8 * k * U64, eta
    # zero corrections: the FP32 solve alone (orders up to 512 run it as one
    # batched launch over 64-column panels), FP32-grade
    eta0 = oracle.trsm_backward_error(side, uplo, trans, diag, -0.75, A64,
                                      np.asfortranarray(X0.cpu().numpy()),
                                      B.astype(np.float64))["eta"]
    assert eta0 <= 8 * k * 2.0 ** -24, eta0


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_mixed_fp64_trsm_all_variants(trx, side, uplo, trans, diag):
    h = trx.Handle(0)
    h.set_option(trx.OPT_FP64_TRSM, 3)
    vi = VARIANTS.index((side, uplo, trans, diag))
    for m, n in ((64, 40), (700, 129)):
        if side == "R":
            m, n = n, m
        k = m if side == "L" else n
        A, B = inputs.problem(side, uplo, m, n, seed=inputs.variant_seed(k, vi) + 11,
                              dtype=np.float64, poison_diag=(diag == "U"), ldb=m + 3)
        B[m:, :] = SENTINEL
        At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
        trx.trsm(side, uplo, trans, diag, 1.5, At, Bt[:m, :], handle=h)
        torch.cuda.synchronize()
        out = Bt.cpu().numpy()
        assert np.all(out[m:, :] == SENTINEL), "write into the ldb padding"
        eta = oracle.trsm_backward_error(side, uplo, trans, diag, 1.5, A,
                                         np.asfortranarray(out[:m]), np.asfortranarray(B[:m]))
        assert eta["eta"] <= 8 * k * U64, (m, n, eta)
    assert h.check_device_error() == 0
    h.close()


def test_mixed_fp64_trsm_quick_returns(trx):
    h = trx.Handle(0)
    h.set_option(trx.OPT_FP64_TRSM, 2)
    A, B = inputs.problem("L", "L", 200, 30, seed=3, dtype=np.float64)
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    trx.trsm("L", "L", "N", "N", 0.0, At, Bt, handle=h)
    torch.cuda.synchronize()
    assert torch.count_nonzero(Bt).item() == 0
    E = torch.empty((0, 30), dtype=torch.float64, device="cuda:0")
    trx.trsm("L", "L", "N", "N", 1.0, At[:0, :0], E, handle=h)
    h.close()
