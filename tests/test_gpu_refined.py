"""Refined FP32 TRSM (FP32 solve + FP64 iterative refinement) against the
FP64 oracle on condition-targeted inputs.

The factor's strict triangle is uniform(-1,1) * s / k with s found by the
oracle's 1-norm condition estimate (bisection on s) to reach kappa about
1e2, 1e4 and 1e6. A and B are FP32; the oracle solves the same data in
FP64. Checks:
- the refined X has the backward error of an FP64 solve, eta <= 8 k 2^-53
  (residual summed in twice-working precision by the oracle);
- its forward error against the oracle is within the FP64 bound
  8 k 2^-53 kappa, far below the plain FP32 solve's;
- the library's own record (backward error of the plain solve and of the
  result, corrections made) agrees with the oracle's;
- B is not modified, padding of X is not written, runs are bitwise
  repeatable; empty problems, alpha = 0 and unit diagonals (NaN-poisoned)
  behave.
"""
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


def _scale(k, kappa, uplo, seed):
    return 1.0 if kappa is None else oracle.scale_for_condition(k, kappa, seed=seed, uplo=uplo)


def _handle(trx, residual):
    h = trx.Handle(0)
    h.set_option(trx.OPT_RESIDUAL, residual)
    return h


def _refined_case(trx, side, uplo, trans, diag, m, n, alpha, kappa, seed, *, ldx_pad=0,
                  max_iter=30, handle=None):
    k = m if side == "L" else n
    s = _scale(k, kappa, uplo, seed)
    A, B = inputs.problem(side, uplo, m, n, seed=seed, dtype=np.float32, scale=s,
                          poison_diag=(diag == "U"))
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    B_before = Bt.clone()
    Xt = torch.full((n, m + ldx_pad), SENTINEL, dtype=torch.float64, device="cuda:0").t()
    X, info = trx.trsm_refined(side, uplo, trans, diag, alpha, At, Bt, out=Xt[:m, :],
                               max_iter=max_iter, handle=handle)
    torch.cuda.synchronize()
    assert torch.equal(Bt, B_before), "B modified"
    full = Xt.cpu().numpy()
    assert np.all(full[m:, :] == SENTINEL), "write into the ldx padding"
    Xh = np.asfortranarray(full[:m, :])
    A64, B64 = np.asfortranarray(A.astype(np.float64)), np.asfortranarray(B.astype(np.float64))
    return A64, B64, Xh, info, At, Bt


@pytest.mark.parametrize("residual", [1, 2], ids=["fp64", "float_float"])
@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
@pytest.mark.parametrize("side,uplo,trans,diag", [("L", "L", "N", "N"), ("R", "U", "T", "N"),
                                                  ("L", "U", "T", "U"), ("R", "L", "N", "U")])
def test_refined_reaches_fp64_accuracy(trx, side, uplo, trans, diag, kappa, residual):
    m, n = (700, 130) if side == "L" else (130, 700)
    k = 700
    alpha = 1.5
    seed = inputs.variant_seed(k, VARIANTS.index((side, uplo, trans, diag)))
    h = _handle(trx, residual)
    A, B, X, info, At, Bt = _refined_case(trx, side, uplo, trans, diag, m, n, alpha, kappa, seed,
                                          ldx_pad=3, handle=h)
    eta = oracle.trsm_backward_error(side, uplo, trans, diag, alpha, A, X, B)["eta"]
    assert np.isfinite(eta) and eta <= 8 * k * U64, (eta, info)
    X_ref = oracle.trsm(side, uplo, trans, diag, alpha, A, B)
    fwd = oracle.forward_error(X, X_ref)
    assert fwd <= 8 * k * U64 * kappa, (fwd, info)
    # the plain FP32 solve of the same data, for comparison and the record
    X32 = Bt.clone()
    trx.trsm(side, uplo, trans, diag, alpha, At, X32)
    X32 = np.asfortranarray(X32.cpu().numpy().astype(np.float64))
    eta32 = oracle.trsm_backward_error(side, uplo, trans, diag, alpha, A, X32, B)["eta"]
    assert fwd < oracle.forward_error(X32, X_ref)
    assert abs(info["initial_backward_error"] - eta32) <= 1e-3 * eta32 + 8 * k * U64
    assert info["backward_error"] <= max(8 * k * U64, 2 * eta)
    assert 1 <= info["iterations"] <= 30


@pytest.mark.parametrize("residual", [1, 2], ids=["fp64", "float_float"])
@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_refined_all_variants(trx, side, uplo, trans, diag, residual):
    """Every side/uplo/trans/diag at kappa about 1e4, ragged order 300 over
    several leaves and one tensor-core update, 257 right-hand sides (ragged
    64-row and 64-column residual tiles)."""
    m, n = (300, 257) if side == "L" else (257, 300)
    k = 300
    seed = inputs.variant_seed(301, VARIANTS.index((side, uplo, trans, diag)))
    A, B, X, info, _, _ = _refined_case(trx, side, uplo, trans, diag, m, n, -0.75, 1e4, seed,
                                        handle=_handle(trx, residual))
    eta = oracle.trsm_backward_error(side, uplo, trans, diag, -0.75, A, X, B)["eta"]
    assert np.isfinite(eta) and eta <= 8 * k * U64, (eta, info)
    assert info["iterations"] >= 1


def test_refined_is_repeatable(trx):
    A, B = inputs.problem("L", "L", 600, 200, seed=9, dtype=np.float32,
                          scale=oracle.scale_for_condition(600, 1e5, seed=9))
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    X1, i1 = trx.trsm_refined("L", "L", "N", "N", 2.0, At, Bt)
    X2, i2 = trx.trsm_refined("L", "L", "N", "N", 2.0, At, Bt)
    torch.cuda.synchronize()
    assert torch.equal(X1, X2) and i1 == i2


@pytest.mark.parametrize("residual", [1, 2], ids=["fp64", "float_float"])
@pytest.mark.parametrize("side,uplo,trans", [("R", "U", "N"), ("L", "L", "T"), ("L", "U", "N"),
                                             ("R", "L", "T")])
def test_refined_max_iter_zero_is_the_fp32_solve(trx, side, uplo, trans, residual):
    """No corrections: X is the plain FP32 solve widened to FP64, and the
    residual norm the library reports is the oracle's (summed in twice the
    working precision) to within 2^-40 ||op(A)|| ||X||: the float-float
    residual's accuracy, measured directly."""
    m, n = (90, 400) if side == "R" else (400, 90)
    A, B = inputs.problem(side, uplo, m, n, seed=4, dtype=np.float32, scale=30.0)
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    X, info = trx.trsm_refined(side, uplo, trans, "N", 1.25, At, Bt, max_iter=0,
                               handle=_handle(trx, residual))
    X32 = Bt.clone()
    trx.trsm(side, uplo, trans, "N", 1.25, At, X32)
    torch.cuda.synchronize()
    assert info["iterations"] == 0
    assert torch.equal(X, X32.double())
    assert info["backward_error"] == info["initial_backward_error"]
    ref = oracle.trsm_backward_error(side, uplo, trans, "N", 1.25, A.astype(np.float64),
                                     np.asfortranarray(X.cpu().numpy()), B.astype(np.float64))
    scale = ref["norm_a"] * ref["norm_x"]
    assert abs(info["residual_norm"] - ref["res"]) <= 2.0 ** -40 * scale, (info, ref)
    assert abs(info["backward_error"] - ref["eta"]) <= 2.0 ** -40


def test_refined_degenerate(trx):
    A, B = inputs.problem("L", "L", 64, 5, seed=2, dtype=np.float32)
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    X, info = trx.trsm_refined("L", "L", "N", "N", 0.0, At, Bt)
    torch.cuda.synchronize()
    assert torch.count_nonzero(X) == 0 and info["residual_norm"] == 0.0
    # empty right-hand side block: nothing to do
    Xe, ie = trx.trsm_refined("L", "L", "N", "N", 1.0, At, Bt[:, :0])
    assert Xe.shape == (64, 0) and ie["iterations"] == 0
    with pytest.raises(TypeError):
        trx.trsm_refined("L", "L", "N", "N", 1.0, At.double(), Bt)


@pytest.mark.parametrize("residual", [1, 2], ids=["fp64", "float_float"])
def test_refined_stored_condition_scales(trx, residual):
    """The refined workload's inputs: order 8192, 256 right-hand sides, the
    stored scales for kappa about 1e2, 1e4, 1e6; forward and backward error
    against the FP64 oracle."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "condition_scales.json")
    with open(path) as f:
        entries = json.load(f)["entries"]
    for e in entries:
        if e["k"] != 8192:
            continue
        k, n = e["k"], 256
        A, B = inputs.problem("L", "L", k, n, seed=e["seed"], dtype=np.float32, scale=e["scale"])
        At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
        X, info = trx.trsm_refined("L", "L", "N", "N", 1.5, At, Bt,
                                   handle=_handle(trx, residual))
        Xh = np.asfortranarray(X.cpu().numpy())
        A64, B64 = np.asfortranarray(A.astype(np.float64)), np.asfortranarray(B.astype(np.float64))
        eta = oracle.trsm_backward_error("L", "L", "N", "N", 1.5, A64, Xh, B64)["eta"]
        assert eta <= 8 * k * U64, (e, eta, info)
        fwd = oracle.forward_error(Xh, oracle.trsm("L", "L", "N", "N", 1.5, A64, B64))
        assert fwd <= 8 * k * U64 * e["kappa_estimate"], (e, fwd, info)


def test_refined_zero_tolerance_stops_on_stagnation(trx):
    """tol = 0 is never met: every update keeps the float-float
    accumulation, and the loop ends when a correction stops lowering the
    backward error (or after max_iter); the result is still FP64-accurate."""
    k = 500
    A, B = inputs.problem("L", "U", k, 70, seed=12, dtype=np.float32,
                          scale=oracle.scale_for_condition(k, 1e5, seed=12, uplo="U"))
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    X, info = trx.trsm_refined("L", "U", "N", "N", 1.0, At, Bt, tol=0.0, max_iter=8)
    assert 1 <= info["iterations"] <= 8
    eta = oracle.trsm_backward_error("L", "U", "N", "N", 1.0, A.astype(np.float64),
                                     np.asfortranarray(X.cpu().numpy()),
                                     B.astype(np.float64))["eta"]
    assert eta <= 8 * k * U64, (eta, info)


@pytest.mark.parametrize("side,uplo,trans,diag", [("L", "L", "N", "N"), ("L", "U", "N", "N"),
                                                  ("R", "L", "T", "U"), ("R", "U", "N", "N")])
def test_refined_cut_row_tiles(trx, side, uplo, trans, diag):
    """Order 2200: the longest 64-row tiles of the float-float residual span
    138 chunks of 16 columns and are cut into two pieces whose partial sums
    are combined. The first residual (max_iter = 0) must match the oracle's
    to 2^-40 ||op(A)|| ||X||, and the refined result must have an FP64-level
    backward error, for effectively lower and upper op(A)."""
    k, nr = 2200, 45
    m, n = (k, nr) if side == "L" else (nr, k)
    seed = inputs.variant_seed(k, VARIANTS.index((side, uplo, trans, diag)))
    A, B = inputs.problem(side, uplo, m, n, seed=seed, dtype=np.float32, scale=40.0,
                          poison_diag=(diag == "U"))
    At, Bt = to_dev(A, "cuda:0"), to_dev(B, "cuda:0")
    A64, B64 = np.asfortranarray(A.astype(np.float64)), np.asfortranarray(B.astype(np.float64))
    X0, i0 = trx.trsm_refined(side, uplo, trans, diag, 0.5, At, Bt, max_iter=0)
    ref = oracle.trsm_backward_error(side, uplo, trans, diag, 0.5, A64,
                                     np.asfortranarray(X0.cpu().numpy()), B64)
    assert abs(i0["residual_norm"] - ref["res"]) <= 2.0 ** -40 * ref["norm_a"] * ref["norm_x"]
    X, info = trx.trsm_refined(side, uplo, trans, diag, 0.5, At, Bt)
    eta = oracle.trsm_backward_error(side, uplo, trans, diag, 0.5, A64,
                                     np.asfortranarray(X.cpu().numpy()), B64)["eta"]
    assert eta <= 8 * k * U64, (eta, info)
