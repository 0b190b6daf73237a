"""FP64 CPU oracle for BLAS TRSM / TRMM (paper Section 2.1, Eq. 1-4).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg; never by the library itself. It
shares no code with the CUDA path. The arithmetic lives in ``trx_oracle.c``
(plain substitution / double loop over the referenced triangle, OpenMP over
independent right-hand sides); this module builds it with gcc on first use
and wraps it for numpy arrays.

Also here: the 1-norm condition estimate of a factor (Hager's method with
Higham's refinements, on the oracle's own solves) and the bisection on the
generator's off-diagonal scale that reaches a target condition number, for
the precision-form configuration.

Parity status: pinned (see ``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``trx_oracle.c`` into ``liboracle.so`` beside it (gcc, -fopenmp)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, d, c = ctypes.c_int64, ctypes.c_double, ctypes.c_char
        vp = ctypes.c_void_p
        for name in ("oracle_dtrsm", "oracle_dtrmm"):
            f = getattr(lib, name)
            f.argtypes = [c, c, c, c, i64, i64, d, vp, i64, vp, i64]
            f.restype = ctypes.c_int
        f = lib.oracle_trsm_backward_error
        f.argtypes = [c, c, c, c, i64, i64, d, vp, i64, vp, i64, vp, i64, vp]
        f.restype = ctypes.c_int
        lib.oracle_op_norm_inf.argtypes = [c, c, c, i64, vp, i64]
        lib.oracle_op_norm_inf.restype = d
        lib.oracle_nthreads.argtypes = []
        lib.oracle_nthreads.restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(x: np.ndarray) -> np.ndarray:
    """Column-major FP64 copy (FP32 inputs are widened exactly)."""
    return np.asfortranarray(np.asarray(x, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _ld(a: np.ndarray) -> int:
    return max(1, a.shape[0])


def _call(name, side, uplo, trans, diag, alpha, A, B):
    lib = _load()
    A = _f64(A)
    X = _f64(B).copy(order="F")
    m, n = X.shape
    info = getattr(lib, name)(side.encode(), uplo.encode(), trans.encode(),
                              diag.encode(), m, n, float(alpha), _ptr(A),
                              _ld(A), _ptr(X), _ld(X))
    if info != 0:
        raise ValueError(f"{name}: illegal argument / failure code {info}")
    return X


def trsm(side: str, uplo: str, trans: str, diag: str, alpha: float,
         A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R'), FP64."""
    return _call("oracle_dtrsm", side, uplo, trans, diag, alpha, A, B)


def trmm(side: str, uplo: str, trans: str, diag: str, alpha: float,
         A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """alpha op(A) B (side 'L') or alpha B op(A) (side 'R'), FP64."""
    return _call("oracle_dtrmm", side, uplo, trans, diag, alpha, A, B)


def raw_call(name: str, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb) -> int:
    """Call an oracle entry point with explicit sizes (argument-check tests)."""
    lib = _load()
    return getattr(lib, name)(side.encode(), uplo.encode(), trans.encode(),
                              diag.encode(), m, n, float(alpha),
                              None if A is None else _ptr(A), lda,
                              None if B is None else _ptr(B), ldb)


def trsm_backward_error(side, uplo, trans, diag, alpha, A, X, B) -> dict:
    """Normwise backward error of a computed TRSM result X for RHS B.

    eta = ||op(A) X - alpha B|| / (||op(A)|| ||X||) (side L; X op(A) for side
    R), infinity norms, residual summed in twice-working precision."""
    lib = _load()
    A, X, B = _f64(A), _f64(X), _f64(B)
    m, n = B.shape
    out = np.zeros(4)
    info = lib.oracle_trsm_backward_error(
        side.encode(), uplo.encode(), trans.encode(), diag.encode(), m, n,
        float(alpha), _ptr(A), _ld(A), _ptr(X), _ld(X), _ptr(B), _ld(B),
        out.ctypes.data_as(ctypes.c_void_p))
    if info != 0:
        raise ValueError(f"backward error: bad argument {info}")
    return {"eta": out[0], "res": out[1], "norm_a": out[2], "norm_x": out[3]}


def op_norm_inf(uplo, trans, diag, A) -> float:
    """||op(A)||_inf over the referenced triangle (unit diagonal counts 1)."""
    lib = _load()
    A = _f64(A)
    k = A.shape[0]
    return lib.oracle_op_norm_inf(uplo.encode(), trans.encode(), diag.encode(),
                                  k, _ptr(A), _ld(A))


def trmm_error(side, uplo, trans, diag, alpha, A, C_hat, C_ref, B) -> float:
    """||C_hat - C_ref||_inf / (|alpha| ||op(A)||_inf ||B||_inf)."""
    na = op_norm_inf(uplo, trans, diag, A)
    nb = np.abs(_f64(B)).sum(axis=1).max() if B.size else 0.0
    diff = np.abs(_f64(C_hat) - _f64(C_ref)).sum(axis=1).max() if B.size else 0.0
    den = abs(alpha) * na * nb
    return float(diff / den) if den > 0 else float(diff)


def forward_error(X_hat, X_ref) -> float:
    """||X_hat - X_ref||_inf / ||X_ref||_inf."""
    X_hat, X_ref = _f64(X_hat), _f64(X_ref)
    if X_ref.size == 0:
        return 0.0
    den = np.abs(X_ref).sum(axis=1).max()
    num = np.abs(X_hat - X_ref).sum(axis=1).max()
    return float(num / den) if den > 0 else float(num)


def op_norm_one(uplo, trans, diag, A) -> float:
    """||op(A)||_1 over the referenced triangle (unit diagonal counts 1):
    the infinity norm of op(A)^T."""
    t = {"N": "T", "T": "N", "C": "N"}[trans.upper()]
    return op_norm_inf(uplo, t, diag, A)


def inv_norm_one_estimate(uplo, trans, diag, A, itmax: int = 5) -> float:
    """Lower-bound estimate of ||op(A)^-1||_1 by Hager's method with Higham's
    refinements (Higham, "FORTRAN codes for estimating the one-norm of a real
    or complex matrix", ACM TOMS 14, 1988): power-like iterations on the
    convex set ||x||_1 <= 1, each one solve with op(A) and one with op(A)^T,
    then the alternating test vector; the larger of the two estimates.
    The solves are the oracle's own substitution."""
    A = _f64(A)
    k = A.shape[0]
    if k == 0:
        return 0.0
    t = {"N": "T", "T": "N", "C": "N"}[trans.upper()]

    def solve(op, v):
        return trsm("L", uplo, op, diag, 1.0, A, np.asfortranarray(v.reshape(k, 1)))[:, 0]

    x = np.full(k, 1.0 / k)
    est = 0.0
    prev_j = -1
    for it in range(itmax):
        y = solve(trans, x)                       # op(A) y = x
        est_new = float(np.abs(y).sum())
        if it > 0 and est_new <= est:
            break
        est = est_new
        xi = np.where(y >= 0, 1.0, -1.0)
        z = solve(t, xi)                          # op(A)^T z = sign(y)
        j = int(np.argmax(np.abs(z)))
        if np.abs(z).max() <= z @ x or j == prev_j:   # x is a local maximum
            break
        x = np.zeros(k)
        x[j] = 1.0
        prev_j = j
    # alternating-sign vector with linearly growing entries
    alt = np.array([(-1.0) ** i * (1.0 + i / max(k - 1, 1)) for i in range(k)])
    est_alt = 2.0 * float(np.abs(solve(trans, alt)).sum()) / (3.0 * k)
    return max(est, est_alt)


def cond_one_estimate(uplo, trans, diag, A) -> float:
    """kappa_1(op(A)) ~ ||op(A)||_1 * est ||op(A)^-1||_1 (a lower bound up to
    rounding)."""
    return op_norm_one(uplo, trans, diag, A) * inv_norm_one_estimate(uplo, trans, diag, A)


def scale_for_condition(k: int, target: float, *, seed: int, uplo: str = "L",
                        lo: float = 1e-3, hi: float = 1e4, steps: int = 40) -> float:
    """Off-diagonal scale s of the input generator (strict triangle
    uniform(-1,1) * s / k) whose factor has kappa_1 close to ``target``, by
    bisection on log s with the estimator above (kappa grows with s)."""
    from paper_2504_13821_gb300 import inputs

    def kappa(s):
        A = inputs.tri_matrix(k, uplo, seed=seed, dtype=np.float64, scale=s)
        return cond_one_estimate(uplo, "N", "N", A)

    a, b = np.log(lo), np.log(hi)
    for _ in range(steps):
        mid = 0.5 * (a + b)
        if kappa(np.exp(mid)) < target:
            a = mid
        else:
            b = mid
    return float(np.exp(0.5 * (a + b)))


def nthreads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_nthreads())
