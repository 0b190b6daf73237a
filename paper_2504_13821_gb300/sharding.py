"""Right-hand-side sharding across ranks, one GPU per rank.

For side L the columns of B are independent right-hand sides (the base
kernels of Section 3.3 already work column by column); for side R the rows
are. A rank runs the whole recursion of Section 3.1 on its own panel with a
read-only copy of the triangle, so the partition needs no exchange; only a
caller who wants B back on one device gathers the panels.
"""
from __future__ import annotations

from . import _binding


def panel(n: int, world: int, rank: int, quantum: int = 32) -> tuple[int, int]:
    """[j0, j1) of rank's share of n right-hand sides: contiguous panels in
    rank order, each (but the last non-empty one) a multiple of `quantum`
    wide, as equal as that allows; ranks past the end get an empty panel."""
    if n < 0 or world < 1 or not 0 <= rank < world or quantum < 1:
        raise ValueError("bad partition arguments")
    per = -(-n // world)
    per = -(-per // quantum) * quantum
    j0 = min(n, rank * per)
    return j0, min(n, j0 + per)


def solve_panel(op: str, side: str, uplo: str, trans: str, diag: str, alpha: float, A, B,
                world: int, rank: int, *, handle=None, stream=None):
    """This rank's share of op(A) X = alpha B (op 'S') or B := alpha op(A) B
    (op 'M'): the panel of B's right-hand sides (columns for side L, rows for
    side R) solved in place through the library. Returns (j0, j1)."""
    n = B.shape[1] if side.upper() == "L" else B.shape[0]
    j0, j1 = panel(n, world, rank)
    if j1 > j0:
        view = B[:, j0:j1] if side.upper() == "L" else B[j0:j1, :]
        fn = _binding.trsm if op.upper() == "S" else _binding.trmm
        fn(side, uplo, trans, diag, alpha, A, view, handle=handle, stream=stream)
    return j0, j1
