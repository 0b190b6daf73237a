"""FP64 CPU oracle for BLAS TRSM / TRMM (paper Section 2.1, Eq. 1-4).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg; never by the library itself. It
shares no code with the CUDA path. The arithmetic lives in ``trx_oracle.c``
(plain substitution / double loop over the referenced triangle, OpenMP over
independent right-hand sides); this module builds it with gcc on first use
and wraps it for numpy arrays.

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


def nthreads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_nthreads())
