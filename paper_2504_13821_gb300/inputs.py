"""Seeded synthetic inputs for TRSM / TRMM.

This module only draws random numbers; it holds none of the arithmetic of the
method. It is the one piece both sides use: the tests and the benchmark feed
the same arrays to the CUDA library and to the CPU oracle.

Recipe (the paper measures on no dataset; every input is generated):
* triangular factor of order k: diagonal 1 + |N(0,1)|, strict referenced
  triangle uniform(-1, 1) * scale / k, the other triangle filled with NaN so
  that any read of it shows up (BLAS "not referenced" semantics). With
  ``poison_diag`` the diagonal is NaN as well (for diag = 'U' tests).
* right-hand side: N(0,1).
* draws are FP64 from ``numpy.random.default_rng(seed)`` (PCG64) in a fixed
  order (diagonal, then the strict triangle column by column, then B) and
  rounded once to the working precision.
"""
from __future__ import annotations

import numpy as np

_CHUNK_COLS = 1024


def tri_matrix(k: int, uplo: str, *, seed: int, dtype=np.float32,
               scale: float = 1.0, poison: bool = True,
               poison_diag: bool = False, lda: int | None = None,
               rng: np.random.Generator | None = None) -> np.ndarray:
    """k x k triangular factor, column-major, leading dimension ``lda``.

    Returns a Fortran-ordered (lda x k) array; the factor is its top k rows.
    Rows k..lda-1 (padding) are NaN.
    """
    lda = k if lda is None else lda
    assert lda >= max(1, k)
    rng = np.random.default_rng(seed) if rng is None else rng
    fill = np.nan if poison else 0.0
    out = np.full((lda, k), fill, dtype=dtype, order="F")
    if k == 0:
        return out
    diag = 1.0 + np.abs(rng.standard_normal(k))
    lower = uplo.upper() == "L"
    for c0 in range(0, k, _CHUNK_COLS):
        c1 = min(k, c0 + _CHUNK_COLS)
        blk = rng.uniform(-1.0, 1.0, size=(c1 - c0, k)).T * (scale / k)  # (k, cols)
        rows = np.arange(k)[:, None]
        cols = np.arange(c0, c1)[None, :]
        keep = (rows > cols) if lower else (rows < cols)
        sub = out[:k, c0:c1]
        sub[keep] = blk[keep].astype(dtype)
    idx = np.arange(k)
    out[idx, idx] = np.nan if poison_diag else diag.astype(dtype)
    return out


def rhs(m: int, n: int, *, seed: int, dtype=np.float32, ldb: int | None = None,
        rng: np.random.Generator | None = None, pad_value=np.nan) -> np.ndarray:
    """m x n N(0,1) right-hand side, Fortran-ordered (ldb x n); padding rows
    m..ldb-1 hold ``pad_value`` so a write into them can be detected."""
    ldb = m if ldb is None else ldb
    assert ldb >= max(1, m)
    rng = np.random.default_rng(seed) if rng is None else rng
    out = np.full((ldb, n), pad_value, dtype=dtype, order="F")
    for c0 in range(0, n, _CHUNK_COLS):
        c1 = min(n, c0 + _CHUNK_COLS)
        out[:m, c0:c1] = rng.standard_normal((c1 - c0, m)).T.astype(dtype)
    return out


def problem(side: str, uplo: str, m: int, n: int, *, seed: int,
            dtype=np.float32, scale: float = 1.0, poison_diag: bool = False,
            lda: int | None = None, ldb: int | None = None):
    """(A, B) for one TRSM/TRMM call: A is the k x k factor (k = m for side
    'L', n for side 'R'), drawn first from one generator, then B."""
    k = m if side.upper() == "L" else n
    rng = np.random.default_rng(seed)
    A = tri_matrix(k, uplo, seed=seed, dtype=dtype, scale=scale,
                   poison_diag=poison_diag, lda=lda, rng=rng)
    B = rhs(m, n, seed=seed, dtype=dtype, ldb=ldb, rng=rng)
    return A, B


def variant_seed(k: int, variant_index: int = 0) -> int:
    """Seed for a sized sweep: k, offset by 1e6 per variant."""
    return int(k) + 1_000_000 * int(variant_index)


VARIANTS = [(s, u, t, d) for s in "LR" for u in "LU" for t in "NT" for d in "NU"]
