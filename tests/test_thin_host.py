"""The thin solve's algebra on the host (no GPU): block forward
substitution with 64-row blocks, summed left-looking, the diagonal solve as
a product with the block's inverse and the last off-diagonal product folded
into Z = inv(M_ii) M_i,i-1:

    X_i = inv(M_ii) (alpha B_i - sum_{j < i-1} M_ij X_j) - Z_i X_i-1

replayed in FP64 against the oracle's substitution (the same exact result,
so agreement to FP64 rounding pins the reformulation the kernel computes),
for ragged orders and several right-hand sides, unit and non-unit."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2504_13821_gb300 import inputs

BR = 64


def thin_replay(M, B, alpha):
    k = M.shape[0]
    nb = -(-k // BR)
    X = np.zeros_like(B)
    for i in range(nb):
        r0, r1 = i * BR, min(k, (i + 1) * BR)
        Mii = np.tril(M[r0:r1, r0:r1])
        inv = sla.solve_triangular(Mii, np.eye(r1 - r0), lower=True)
        S = np.zeros((r1 - r0, B.shape[1]))
        for j in range(max(0, i - 1)):
            S += M[r0:r1, j * BR:(j + 1) * BR] @ X[j * BR:(j + 1) * BR]
        X[r0:r1] = inv @ (alpha * B[r0:r1] - S)
        if i > 0:
            p0, p1 = (i - 1) * BR, i * BR
            Z = inv @ M[r0:r1, p0:p1]
            X[r0:r1] -= Z @ X[p0:p1]
    return X


@pytest.mark.parametrize("k", [1, 40, 64, 65, 130, 257])
@pytest.mark.parametrize("n", [1, 5, 17])
@pytest.mark.parametrize("diag", ["N", "U"])
def test_thin_algebra_matches_substitution(k, n, diag):
    A, B = inputs.problem("L", "L", k, n, seed=7 * k + n, dtype=np.float64)
    M = np.where(np.isnan(A), 0.0, A)
    if diag == "U":
        np.fill_diagonal(M, 1.0)
    got = thin_replay(np.tril(M), B, -1.5)
    want = oracle.trsm("L", "L", "N", diag, -1.5, A, B)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_thin_leaves_then_updates():
    # thin solves as the recursion's leaves: leaves of 128 rows solved by the
    # thin algebra, the updates between them as in the recursion
    k, n, leaf = 300, 6, 128
    A, B = inputs.problem("L", "L", k, n, seed=300, dtype=np.float64)
    M = np.tril(np.where(np.isnan(A), 0.0, A))
    C = 2.0 * B.copy()
    for r0 in range(0, k, leaf):
        r1 = min(k, r0 + leaf)
        C[r0:r1] = thin_replay(M[r0:r1, r0:r1], C[r0:r1], 1.0)
        C[r1:] -= M[r1:, r0:r1] @ C[r0:r1]
    want = oracle.trsm("L", "L", "N", "N", 2.0, A, B)
    np.testing.assert_allclose(C, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())
