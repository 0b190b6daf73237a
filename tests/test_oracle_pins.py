"""Pins for the FP64 CPU oracle, independent of the oracle itself.

Each check fixes the oracle to something it does not compute itself:
exact rational arithmetic (brute-force inverse), closed forms, invariants,
a BLAS library routine, and the worked example in tests/golden/. The cases
are chosen so that a plausible slip in the oracle (a dropped term, a wrong
sign, a swapped index, a transposed operand, a read of the unreferenced
triangle) fails at least one of them.
"""
from fractions import Fraction
import itertools
import os
import zlib

import numpy as np
import pytest

import oracle
from paper_2504_13821_gb300 import inputs

VARIANTS = inputs.VARIANTS
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- brute force in exact rationals --------------------------------------
def dense_op(A, uplo, trans, diag):
    """op(A) as a dense exact matrix, built straight from BLAS semantics:
    keep the uplo triangle of the storage, force a unit diagonal, transpose."""
    k = A.shape[0]
    E = [[Fraction(0)] * k for _ in range(k)]
    for r in range(k):
        for c in range(k):
            inside = (r >= c) if uplo == "L" else (r <= c)
            if r == c and diag == "U":
                E[r][c] = Fraction(1)
            elif inside:
                E[r][c] = Fraction(float(A[r, c]))
    if trans != "N":
        E = [[E[c][r] for c in range(k)] for r in range(k)]
    return E


def inverse(E):
    """Gauss-Jordan inverse with exact rationals (full pivot search)."""
    k = len(E)
    M = [row[:] + [Fraction(int(i == j)) for j in range(k)] for i, row in enumerate(E)]
    for col in range(k):
        piv = next(r for r in range(col, k) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        p = M[col][col]
        M[col] = [v / p for v in M[col]]
        for r in range(k):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    return [row[k:] for row in M]


def matmul(X, Y):
    return [[sum(X[i][l] * Y[l][j] for l in range(len(Y))) for j in range(len(Y[0]))]
            for i in range(len(X))]


def to_frac(B):
    return [[Fraction(float(v)) for v in row] for row in B]


def int_problem(rng, side, uplo, diag, m, n):
    """Integer triangle (power-of-two diagonal), NaN outside the triangle and
    on a unit diagonal, integer right-hand side: every FP64 operation of a
    substitution is then exact, so the oracle must agree bit for bit."""
    k = m if side == "L" else n
    A = np.full((k, k), np.nan)
    for r in range(k):
        for c in range(k):
            if (r > c) if uplo == "L" else (r < c):
                A[r, c] = rng.integers(-3, 4)
    d = rng.choice([1.0, 2.0, 4.0, -2.0, 0.5], size=k)
    A[np.arange(k), np.arange(k)] = np.nan if diag == "U" else d
    B = rng.integers(-5, 6, size=(m, n)).astype(np.float64)
    return np.asfortranarray(A), np.asfortranarray(B)


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
@pytest.mark.parametrize("m,n", [(5, 3), (3, 6), (8, 8), (1, 4)])
def test_trsm_exact_against_rational_inverse(side, uplo, trans, diag, m, n):
    rng = np.random.default_rng(zlib.crc32(f"{side}{uplo}{trans}{diag}{m},{n}".encode()))
    A, B = int_problem(rng, side, uplo, diag, m, n)
    alpha = 2.0
    E = dense_op(A, uplo, trans, diag)
    Ei = inverse(E)
    aB = [[Fraction(2) * v for v in row] for row in to_frac(B)]
    X = matmul(Ei, aB) if side == "L" else matmul(aB, Ei)
    got = oracle.trsm(side, uplo, trans, diag, alpha, A, B)
    want = np.array([[float(v) for v in row] for row in X])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
@pytest.mark.parametrize("m,n", [(5, 3), (3, 6), (8, 8)])
def test_trmm_exact_against_rational_product(side, uplo, trans, diag, m, n):
    rng = np.random.default_rng(1 + zlib.crc32(f"{side}{uplo}{trans}{diag}{m},{n}".encode()))
    A, B = int_problem(rng, side, uplo, diag, m, n)
    alpha = -0.5
    E = dense_op(A, uplo, trans, diag)
    aB = [[Fraction(-1, 2) * v for v in row] for row in to_frac(B)]
    C = matmul(E, aB) if side == "L" else matmul(aB, E)
    got = oracle.trmm(side, uplo, trans, diag, alpha, A, B)
    want = np.array([[float(v) for v in row] for row in C])
    assert np.array_equal(got, want)


# ---- closed forms ----------------------------------------------------------
def bidiag(k, uplo):
    """1 on the diagonal, -1 on the sub- (L) or super- (U) diagonal."""
    A = np.full((k, k), np.nan)
    A[np.arange(k), np.arange(k)] = 1.0
    if uplo == "L":
        A[np.arange(1, k), np.arange(k - 1)] = -1.0
        A[np.triu_indices(k, 1)] = np.nan
        A[np.tril_indices(k, -2)] = 0.0
    else:
        A[np.arange(k - 1), np.arange(1, k)] = -1.0
        A[np.tril_indices(k, -1)] = np.nan
        A[np.triu_indices(k, 2)] = 0.0
    return np.asfortranarray(A)


@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_bidiagonal_inverse_is_prefix_sum(uplo, trans):
    # Lower bidiagonal (1, -1) has the all-ones lower triangle as inverse, so
    # a left solve is a running sum down each column (bottom-up for upper).
    k, n, alpha = 9, 4, 1.5
    A = bidiag(k, uplo)
    B = np.asfortranarray(np.random.default_rng(3).standard_normal((k, n)))
    X = oracle.trsm("L", uplo, trans, "N", alpha, A, B)
    eff_lower = (uplo == "L") == (trans == "N")
    want = alpha * (np.cumsum(B, axis=0) if eff_lower
                    else np.cumsum(B[::-1], axis=0)[::-1])
    np.testing.assert_allclose(X, want, rtol=1e-14, atol=1e-14)
    # Right side: X op(A) = alpha B -> running sums along each row, in the
    # direction opposite to the left-side one.
    Br = np.asfortranarray(B.T.copy())
    Xr = oracle.trsm("R", uplo, trans, "N", alpha, A, Br)
    want_r = alpha * (np.cumsum(Br[:, ::-1], axis=1)[:, ::-1] if eff_lower
                      else np.cumsum(Br, axis=1))
    np.testing.assert_allclose(Xr, want_r, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("uplo", "LU")
def test_ones_triangle_product_is_prefix_sum(uplo):
    k, n = 7, 3
    A = np.full((k, k), np.nan)
    idx = np.tril_indices(k) if uplo == "L" else np.triu_indices(k)
    A[idx] = 1.0
    A = np.asfortranarray(A)
    B = np.asfortranarray(np.random.default_rng(5).standard_normal((k, n)))
    C = oracle.trmm("L", uplo, "N", "N", 1.0, A, B)
    want = np.cumsum(B, axis=0) if uplo == "L" else np.cumsum(B[::-1], axis=0)[::-1]
    np.testing.assert_allclose(C, want, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_identity_and_diagonal(side, uplo, trans, diag):
    m, n = 6, 5
    k = m if side == "L" else n
    rng = np.random.default_rng(11)
    B = np.asfortranarray(rng.standard_normal((m, n)))
    d = 1.0 + np.abs(rng.standard_normal(k))
    A = np.full((k, k), np.nan)
    if uplo == "L":
        A[np.tril_indices(k, -1)] = 0.0
    else:
        A[np.triu_indices(k, 1)] = 0.0
    A[np.arange(k), np.arange(k)] = np.nan if diag == "U" else d
    A = np.asfortranarray(A)
    scale = np.ones(k) if diag == "U" else d
    X = oracle.trsm(side, uplo, trans, diag, -2.0, A, B)
    C = oracle.trmm(side, uplo, trans, diag, -2.0, A, B)
    if side == "L":
        np.testing.assert_allclose(X, -2.0 * B / scale[:, None], rtol=1e-15)
        np.testing.assert_allclose(C, -2.0 * B * scale[:, None], rtol=1e-15)
    else:
        np.testing.assert_allclose(X, -2.0 * B / scale[None, :], rtol=1e-15)
        np.testing.assert_allclose(C, -2.0 * B * scale[None, :], rtol=1e-15)


def test_worked_example_golden():
    """Hand-worked 3x3 lower system (Eq. 3), values in tests/golden."""
    path = os.path.join(GOLDEN, "trsm_lower_3x3.txt")
    rows = [l.split("#")[0].split() for l in open(path)]
    rows = [list(map(float, r)) for r in rows if r]
    A = np.asfortranarray(np.array(rows[0:3]))
    B = np.asfortranarray(np.array(rows[3:6]))
    X = np.array(rows[6:9])
    alpha = rows[9][0]
    got = oracle.trsm("L", "L", "N", "N", alpha, A, B)
    assert np.array_equal(got, X)
    # the same numbers read as TRMM: alpha * A * X == alpha^2 * B
    C = oracle.trmm("L", "L", "N", "N", alpha, A, X)
    assert np.array_equal(C, alpha * alpha * B)


# ---- invariants ------------------------------------------------------------
@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_round_trip_and_side_duality(side, uplo, trans, diag):
    m, n = 40, 24
    A, B = inputs.problem(side, uplo, m, n, seed=7, dtype=np.float64,
                          poison_diag=(diag == "U"))
    C = oracle.trmm(side, uplo, trans, diag, 1.5, A, B)
    X = oracle.trsm(side, uplo, trans, diag, 1.0 / 1.5, A, C)
    np.testing.assert_allclose(X, B, rtol=0, atol=1e-13 * np.abs(B).max())
    # X op(A) = aB  <=>  op(A)^T X^T = a B^T: identical operations, so the
    # results agree bit for bit.
    flip = "N" if trans != "N" else "T"
    other = "R" if side == "L" else "L"
    Xd = oracle.trsm(other, uplo, flip, diag, 1.5, A, np.asfortranarray(B.T))
    Xs = oracle.trsm(side, uplo, trans, diag, 1.5, A, B)
    assert np.array_equal(Xd.T, Xs)
    Cd = oracle.trmm(other, uplo, flip, diag, 1.5, A, np.asfortranarray(B.T))
    np.testing.assert_allclose(Cd.T, C, rtol=1e-15, atol=1e-15)


# ---- library special case --------------------------------------------------
@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_against_reference_blas(side, uplo, trans, diag):
    blas = pytest.importorskip("scipy.linalg.blas")
    m, n = 33, 21
    A, B = inputs.problem(side, uplo, m, n, seed=13, dtype=np.float64)
    Az = np.where(np.isnan(A), 0.0, A)  # the library may touch the other half
    kw = dict(side=int(side == "R"), lower=int(uplo == "L"),
              trans_a=int(trans != "N"), diag=int(diag == "U"))
    X = oracle.trsm(side, uplo, trans, diag, 1.5, A, B)
    np.testing.assert_allclose(X, blas.dtrsm(1.5, Az, B, **kw), rtol=1e-12, atol=1e-12)
    C = oracle.trmm(side, uplo, trans, diag, 1.5, A, B)
    np.testing.assert_allclose(C, blas.dtrmm(1.5, Az, B, **kw), rtol=1e-12, atol=1e-12)


# ---- BLAS argument semantics -----------------------------------------------
def test_argument_positions():
    A = np.asfortranarray(np.eye(4))
    B = np.asfortranarray(np.ones((4, 3)))
    for name in ("oracle_dtrsm", "oracle_dtrmm"):
        call = lambda *a: oracle.raw_call(name, *a)
        assert call("X", "L", "N", "N", 4, 3, 1.0, A, 4, B, 4) == -1
        assert call("L", "X", "N", "N", 4, 3, 1.0, A, 4, B, 4) == -2
        assert call("L", "L", "X", "N", 4, 3, 1.0, A, 4, B, 4) == -3
        assert call("L", "L", "N", "X", 4, 3, 1.0, A, 4, B, 4) == -4
        assert call("L", "L", "N", "N", -1, 3, 1.0, A, 4, B, 4) == -5
        assert call("L", "L", "N", "N", 4, -1, 1.0, A, 4, B, 4) == -6
        assert call("L", "L", "N", "N", 4, 3, 1.0, None, 4, B, 4) == -8
        assert call("L", "L", "N", "N", 4, 3, 1.0, A, 3, B, 4) == -9
        assert call("R", "L", "N", "N", 4, 3, 1.0, A, 2, B, 4) == -9
        assert call("L", "L", "N", "N", 4, 3, 1.0, A, 4, None, 4) == -10
        assert call("L", "L", "N", "N", 4, 3, 1.0, A, 4, B, 3) == -11
        assert call("l", "u", "c", "u", 4, 3, 1.0, A, 4, B, 4) == 0


def test_alpha_zero_and_empty():
    A = np.asfortranarray(np.full((5, 5), np.nan))
    B = np.asfortranarray(np.ones((5, 2)))
    assert np.array_equal(oracle.trsm("L", "L", "N", "N", 0.0, A, B), np.zeros((5, 2)))
    assert np.array_equal(oracle.trmm("R", "U", "T", "U", 0.0, np.full((2, 2), np.nan), B),
                          np.zeros((5, 2)))
    E = np.zeros((0, 3), order="F")
    assert oracle.trsm("L", "L", "N", "N", 1.0, np.zeros((0, 0)), E).shape == (0, 3)


# ---- error metrics -----------------------------------------------------------
def test_backward_error_exact_cases():
    # Exact solution of an integer system: residual exactly zero.
    rng = np.random.default_rng(2)
    A, B = int_problem(rng, "L", "L", "N", 6, 4)
    X = oracle.trsm("L", "L", "N", "N", 1.0, A, B)
    assert oracle.trsm_backward_error("L", "L", "N", "N", 1.0, A, X, B)["eta"] == 0.0
    # Identity factor: residual = perturbation, eta = ||E|| / ||X||.
    k, n = 5, 3
    Id = np.asfortranarray(np.eye(k))
    B = np.asfortranarray(rng.standard_normal((k, n)))
    E = np.asfortranarray(rng.standard_normal((k, n)) * 2.0**-30)
    Xp = np.asfortranarray(B + E)
    Ex = Xp - B  # exact (Sterbenz): the perturbation actually stored
    r = oracle.trsm_backward_error("L", "U", "N", "N", 1.0, Id, Xp, B)
    want = np.abs(Ex).sum(1).max() / np.abs(Xp).sum(1).max()
    assert abs(r["eta"] - want) <= 1e-12 * want


def test_backward_error_residual_is_twice_working_precision():
    # The residual of the oracle's own FP64 solution is at rounding level;
    # a plain FP64 sum would get it wrong by O(100%). Compare with the exact
    # rational residual of the same floating-point numbers.
    k, n = 30, 3
    A, B = inputs.problem("L", "L", k, n, seed=21, dtype=np.float64)
    X = oracle.trsm("L", "L", "N", "N", 1.0, A, B)
    r = oracle.trsm_backward_error("L", "L", "N", "N", 1.0, A, X, B)
    exact_rows = []
    for i in range(k):
        s = Fraction(0)
        for j in range(n):
            t = sum(Fraction(float(A[i, l])) * Fraction(float(X[l, j])) for l in range(i + 1))
            s += abs(t - Fraction(float(B[i, j])))
        exact_rows.append(s)
    exact = float(max(exact_rows))
    assert exact > 0
    assert abs(r["res"] - exact) <= 1e-6 * exact


def _op_exact(uplo, trans, diag, A, k):
    """op(A) of the referenced triangle as a k x k list of Fractions (unit
    diagonal 1, the other triangle 0)."""
    T = [[Fraction(0)] * k for _ in range(k)]
    for i in range(k):
        for l in range(k):
            if i == l:
                T[i][l] = Fraction(1) if diag == "U" else Fraction(float(A[i, l]))
            elif (uplo == "L" and i > l) or (uplo == "U" and i < l):
                T[i][l] = Fraction(float(A[i, l]))
    if trans != "N":
        T = [[T[l][i] for l in range(k)] for i in range(k)]
    return T


@pytest.mark.parametrize("uplo,trans,diag", [("U", "T", "U"), ("L", "N", "N"),
                                             ("U", "N", "N"), ("L", "T", "U")])
def test_backward_error_side_right_exact_residual(uplo, trans, diag):
    # Side R: R = X op(A) - alpha B (Eq. 4), eta = ||R|| / (||op(A)|| ||X||).
    # Every quantity is recomputed here in exact rationals from the stored
    # floating-point numbers (X perturbed away from the solution so that R is
    # well above rounding); a transposed residual, a row/column mix-up in
    # either norm or a wrong triangle all fail.
    m, k = 7, 6
    alpha = 1.5
    A, B = inputs.problem("R", uplo, m, k, seed=77, dtype=np.float64,
                          poison_diag=(diag == "U"))
    X = oracle.trsm("R", uplo, trans, diag, alpha, A, B)
    rng = np.random.default_rng(78)
    X = np.asfortranarray(X + rng.standard_normal(X.shape) * 1e-6)
    r = oracle.trsm_backward_error("R", uplo, trans, diag, alpha, A, X, B)
    T = _op_exact(uplo, trans, diag, A, k)
    res_rows = []
    for i in range(m):
        row = Fraction(0)
        for j in range(k):
            v = sum(Fraction(float(X[i, l])) * T[l][j] for l in range(k))
            row += abs(v - Fraction(alpha) * Fraction(float(B[i, j])))
        res_rows.append(row)
    res = max(res_rows)
    norm_a = max(sum(abs(T[i][j]) for j in range(k)) for i in range(k))
    norm_x = max(sum(abs(Fraction(float(X[i, j]))) for j in range(k)) for i in range(m))
    assert r["res"] == pytest.approx(float(res), rel=1e-12)
    assert r["norm_a"] == pytest.approx(float(norm_a), rel=1e-15)
    assert r["norm_x"] == pytest.approx(float(norm_x), rel=1e-15)
    assert r["eta"] == pytest.approx(float(res / (norm_a * norm_x)), rel=1e-12)


def test_backward_error_side_right_exact_zero_and_identity():
    # Exact integer system on side R: X op(A) = B solved exactly -> eta 0;
    # identity factor: eta = ||X - B|| / ||X|| with the row-sum norm.
    rng = np.random.default_rng(5)
    A, B = int_problem(rng, "R", "U", "U", 4, 6)
    X = oracle.trsm("R", "U", "N", "U", 1.0, A, B)
    assert oracle.trsm_backward_error("R", "U", "N", "U", 1.0, A, X, B)["eta"] == 0.0
    m, k = 4, 5
    Id = np.asfortranarray(np.eye(k))
    B = np.asfortranarray(rng.standard_normal((m, k)))
    Xp = np.asfortranarray(B + rng.standard_normal((m, k)) * 2.0**-30)
    Ex = Xp - B
    r = oracle.trsm_backward_error("R", "L", "T", "N", 1.0, Id, Xp, B)
    want = np.abs(Ex).sum(1).max() / np.abs(Xp).sum(1).max()
    assert abs(r["eta"] - want) <= 1e-12 * want


# ---- condition estimate (inputs of the precision-form configuration) ------

def _exact_kappa_one(uplo, trans, diag, A):
    T = np.where(np.isnan(A), 0.0, np.asarray(A, dtype=np.float64))
    T = np.tril(T) if uplo == "L" else np.triu(T)
    if diag == "U":
        np.fill_diagonal(T, 1.0)
    op = T if trans == "N" else T.T
    return np.abs(op).sum(axis=0).max() * np.abs(np.linalg.inv(op)).sum(axis=0).max()


def test_cond_estimate_closed_forms():
    # identity: 1; diagonal: max|d| / min|d|; unit lower bidiagonal with -1
    # below: ||T||_1 = 2 and T^-1 is the lower triangle of ones, ||T^-1||_1 = k
    k = 40
    assert oracle.cond_one_estimate("L", "N", "N", np.eye(k)) == pytest.approx(1.0, rel=1e-14)
    d = np.linspace(0.5, 8.0, k)
    assert oracle.cond_one_estimate("U", "T", "N", np.diag(d)) == pytest.approx(16.0, rel=1e-14)
    T = np.eye(k) - np.eye(k, k=-1)
    assert oracle.cond_one_estimate("L", "N", "N", T) == pytest.approx(2.0 * k, rel=1e-14)
    assert oracle.cond_one_estimate("U", "T", "U", T.T) == pytest.approx(2.0 * k, rel=1e-14)


@pytest.mark.parametrize("k", [2, 7, 33, 120])
@pytest.mark.parametrize("uplo,trans", [("L", "N"), ("U", "N"), ("L", "T"), ("U", "T")])
def test_cond_estimate_is_a_close_lower_bound(k, uplo, trans):
    A = inputs.tri_matrix(k, uplo, seed=3 * k, dtype=np.float64, scale=4.0)
    exact = _exact_kappa_one(uplo, trans, "N", A)
    est = oracle.cond_one_estimate(uplo, trans, "N", A)
    assert est <= exact * (1 + 1e-10)
    assert est >= exact / 3


@pytest.mark.parametrize("target", [1e2, 1e4])
def test_scale_for_condition_hits_the_target(target):
    s = oracle.scale_for_condition(128, target, seed=5)
    A = inputs.tri_matrix(128, "L", seed=5, dtype=np.float64, scale=s)
    kappa = _exact_kappa_one("L", "N", "N", A)
    assert target / 3 <= kappa <= 3 * target


# ---- the oracle's norms and error metrics, pinned directly --------------------

def _op_dense(uplo, trans, diag, A):
    """op(T) as a dense matrix built explicitly from the referenced triangle."""
    k = A.shape[0]
    T = np.tril(A, -1) if uplo == "L" else np.triu(A, 1)
    T = np.nan_to_num(T, nan=0.0)
    T = T + (np.eye(k) if diag == "U" else np.diag(np.diag(A)))
    return T.T if trans in ("T", "C") else T


@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("trans", ["N", "T", "C"])
@pytest.mark.parametrize("diag", ["N", "U"])
def test_op_norms_match_numpy_on_the_built_triangle(uplo, trans, diag):
    rng = np.random.default_rng(41)
    k = 9
    A = rng.uniform(-3, 3, (k, k))
    # the unreferenced triangle (and the diagonal for 'U') is poison
    bad = np.triu(np.ones((k, k), bool), 1) if uplo == "L" else np.tril(np.ones((k, k), bool), -1)
    A[bad] = np.nan
    if diag == "U":
        A[np.arange(k), np.arange(k)] = np.nan
    A = np.asfortranarray(A)
    T = _op_dense(uplo, trans, diag, A)
    assert oracle.op_norm_inf(uplo, trans, diag, A) == pytest.approx(np.linalg.norm(T, np.inf),
                                                                      rel=1e-15)
    assert oracle.op_norm_one(uplo, trans, diag, A) == pytest.approx(np.linalg.norm(T, 1),
                                                                      rel=1e-15)


def test_forward_and_trmm_error_closed_forms():
    X_ref = np.asfortranarray(np.ones((4, 3)))
    X_hat = X_ref.copy(order="F")
    X_hat[2, :] += [0.5, -0.25, 0.0]                 # row sums of |X_ref| are 3
    assert oracle.forward_error(X_hat, X_ref) == pytest.approx(0.75 / 3.0, rel=1e-15)
    assert oracle.forward_error(X_ref, X_ref) == 0.0
    # TRMM error: ||C_hat - C_ref||_inf / (|alpha| ||op(A)||_inf ||B||_inf)
    A = np.asfortranarray(np.tril(np.full((3, 3), 2.0)))     # ||A||_inf = 6
    B = np.asfortranarray(np.ones((3, 2)))                   # ||B||_inf = 2
    C_ref = oracle.trmm("L", "L", "N", "N", -1.5, A, B)
    C_hat = C_ref.copy(order="F")
    C_hat[1, 0] += 0.9
    assert oracle.trmm_error("L", "L", "N", "N", -1.5, A, C_hat, C_ref, B) == pytest.approx(
        0.9 / (1.5 * 6.0 * 2.0), rel=1e-14)


@pytest.mark.parametrize("uplo,trans", [("L", "N"), ("U", "T"), ("L", "T")])
def test_inverse_norm_estimate_is_a_lower_bound_and_exact_when_diagonal(uplo, trans):
    rng = np.random.default_rng(7)
    for k in (1, 5, 40):
        d = 1.0 + rng.random(k) * 9.0
        D = np.asfortranarray(np.diag(d))
        exact = 1.0 / d.min()                             # ||D^-1||_1
        assert oracle.inv_norm_one_estimate(uplo, trans, "N", D) == pytest.approx(exact,
                                                                                  rel=1e-14)
        A = np.asfortranarray(np.tril(rng.uniform(-1, 1, (k, k)), -1) * 0.5 + np.diag(d))
        if uplo == "U":
            A = np.asfortranarray(A.T)
        T = _op_dense(uplo, trans, "N", A)
        true = np.linalg.norm(np.linalg.inv(T), 1)
        est = oracle.inv_norm_one_estimate(uplo, trans, "N", A)
        assert est <= true * (1 + 1e-12) and est >= true / (3.0 * k)
