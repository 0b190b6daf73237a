"""Shared helpers for the GPU parity tests (device copies, tolerances)."""
import numpy as np

import oracle
from paper_2504_13821_gb300 import inputs

U = {np.float32: 2.0 ** -24, np.float64: 2.0 ** -53}
SENTINEL = 7777.0


def bound(k, dtype):
    """Normwise tolerance 8 k u of the working precision."""
    return 8 * max(int(k), 1) * U[dtype]


def to_dev(arr, device):
    """Column-major device copy of a Fortran-ordered (ld x cols) array."""
    import torch
    ld, cols = arr.shape
    t = torch.empty((cols, ld), dtype=torch.from_numpy(arr[:0, :0].copy()).dtype,
                    device=device).t()
    t.copy_(torch.from_numpy(np.asfortranarray(arr)))
    return t


def run_case(op, side, uplo, trans, diag, m, n, alpha, dtype, seed, *, lda_pad=0,
             ldb_pad=0, handle=None, device="cuda:0", check=True):
    """One library call on seeded inputs, checked against the oracle.

    Returns (metric, bound, device result as numpy)."""
    import torch
    import paper_2504_13821_gb300 as trx
    k = m if side == "L" else n
    A, B = inputs.problem(side, uplo, m, n, seed=seed, dtype=dtype,
                          poison_diag=(diag == "U"), lda=k + lda_pad, ldb=m + ldb_pad)
    B[m:, :] = SENTINEL
    At, Bt = to_dev(A, device), to_dev(B, device)
    fn = trx.trsm if op == "trsm" else trx.trmm
    fn(side, uplo, trans, diag, alpha, At[:k, :k], Bt[:m, :], handle=handle)
    torch.cuda.synchronize()
    out = Bt.cpu().numpy()
    assert np.all(out[m:, :] == SENTINEL), "write into the ldb padding"
    X = np.asfortranarray(out[:m, :])
    Ak, B0 = np.asfortranarray(A[:k, :k]), np.asfortranarray(B[:m, :])
    tol = bound(k, dtype)
    if op == "trsm":
        metric = oracle.trsm_backward_error(side, uplo, trans, diag, alpha, Ak, X, B0)["eta"]
    else:
        C_ref = oracle.trmm(side, uplo, trans, diag, alpha, Ak, B0)
        metric = oracle.trmm_error(side, uplo, trans, diag, alpha, Ak, X, C_ref, B0)
    if check:
        assert np.isfinite(metric) and metric <= tol, (
            f"{op} {side}{uplo}{trans}{diag} m={m} n={n} {np.dtype(dtype).name}: "
            f"error {metric:.3e} > {tol:.3e}")
    return metric, tol, X
