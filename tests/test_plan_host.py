"""Host logic of the recursion planner (Section 3.1), no GPU needed.

The library reports the launch sequence it would enqueue (trx_debug_plan).
These tests check its structure (the diagonal leaf blocks and the GEMM
update blocks tile the triangle exactly once; every update reads rows
already final and writes rows not yet final; tensor-core updates have K a
multiple of the K tile; alpha enters exactly once) and replay the sequence
in FP64 numpy on a canonical lower triangle, which must reproduce the
oracle's result.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2504_13821_gb300 import build, debug_plan, inputs

SIZES = [1, 2, 17, 63, 64, 65, 128, 255, 256, 300, 1000, 1024]
LEAVES = [16, 32, 64, 128]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def leaves_of(steps):
    out = []
    for s in steps:
        if s["kind"] == "leaf":
            for t in range(s["nleaves"]):
                out.append((s["r0"] + t * s["b"], s["b"]))
    return out


def coverage(k, steps):
    """Count how often each (i, l), l <= i, is covered by a leaf diagonal
    block or a GEMM block."""
    cnt = np.zeros((k, k), dtype=np.int32)
    for r, b in leaves_of(steps):
        e = min(k, r + b)
        blk = np.tril(np.ones((e - r, e - r), dtype=np.int32))
        cnt[r:e, r:e] += blk
    for s in steps:
        if s["kind"] == "gemm" and s.get("dense"):
            # a tile of a dense diagonal block: the full columns left of its
            # rows, and its own lower triangle with the diagonal
            r, e = s["rc"], min(k, s["rc"] + s["mlen"])
            cnt[r:e, s["rk"]:r] += 1
            cnt[r:e, r:e] += np.tril(np.ones((e - r, e - r), dtype=np.int32))
        elif s["kind"] == "gemm":
            cnt[s["rc"]:s["rc"] + s["mlen"], s["rk"]:s["rk"] + s["klen"]] += 1
    return cnt


@pytest.mark.parametrize("op", ["S", "M"])
@pytest.mark.parametrize("gemm", [1, 2])
@pytest.mark.parametrize("b", LEAVES + [256])
@pytest.mark.parametrize("k", SIZES + [4097])
def test_blocks_tile_the_triangle_once(op, gemm, b, k):
    steps = debug_plan(op, "L", "L", "N", "N", k, 5, 4, b, gemm)
    if op == "M":
        b = min(b, 128)          # TRMM leaves stop at 128 rows
    cnt = coverage(k, steps)
    low = np.tril(np.ones((k, k), dtype=bool))
    assert np.all(cnt[low] == 1)
    assert np.all(cnt[~low] == 0)
    for s in steps:
        if s["kind"] == "gemm" and s["dense"]:
            assert op == "M" and s["tc"] and s["beta"] == s["gamma"]
            assert s["mlen"] <= 128 and s["rk"] <= s["rc"] and (s["rc"] - s["rk"]) % 128 == 0
            top = s["rc"] + s["mlen"] - s["rk"]                 # K ends at the tile's last row
            assert s["klen"] % 32 == 0 and top <= s["klen"] < top + 32
        elif s["kind"] == "gemm":
            assert s["rk"] + s["klen"] <= s["rc"]           # strictly below
            if s["tc"]:
                assert s["klen"] % 64 == 0 and s["rk"] % 8 == 0
        if s["kind"] == "leaf":
            assert s["b"] <= (256 if op == "S" else 128)
            assert s["r0"] % min(b, max(k, 1)) == 0


@pytest.mark.parametrize("b", LEAVES + [256])
@pytest.mark.parametrize("k", SIZES)
def test_trsm_dependency_order_and_alpha(b, k):
    steps = debug_plan("S", "L", "L", "N", "N", k, 5, 4, b, 2)
    solved = np.zeros(k, dtype=bool)
    touched = np.zeros(k, dtype=bool)   # has alpha been applied to the row
    for s in steps:
        if s["kind"] == "leaf":
            r, e = s["r0"], min(k, s["r0"] + s["b"])
            assert not solved[r:e].any()
            # alpha is applied by the leaf iff no update has touched the rows
            assert (s["alpha"] == 2.0) == (not touched[r:e].any())
            assert touched[r:e].all() or not touched[r:e].any()
            solved[r:e] = touched[r:e] = True
        elif s["kind"] == "gemm":
            rc, re_ = s["rc"], s["rc"] + s["mlen"]
            assert solved[s["rk"]:s["rk"] + s["klen"]].all()       # reads final X
            assert not solved[rc:re_].any()                          # writes pending rows
            assert (s["beta"] == 2.0) == (not touched[rc:re_].any())
            assert touched[rc:re_].all() or not touched[rc:re_].any()
            touched[rc:re_] = True
    assert solved.all()


def replay(op, steps, M, C, alpha_seen=2.0):
    """Execute a plan in FP64 on the canonical lower matrix M (k x k)."""
    C = C.copy()
    k = M.shape[0]
    Y = np.full_like(C, np.nan)      # tensor-core Y planes: unset until written
    for s in steps:
        if s["kind"] == "conv_y":
            Y = C.copy()
        elif s["kind"] == "conv_y_rows":
            Y[s["r0"]:s["r0"] + s["b"]] = C[s["r0"]:s["r0"] + s["b"]]
        elif s["kind"] == "inv_diag":
            pass                     # the inverses are formed where they are used
        elif s["kind"] == "gemm" and s.get("inv"):
            # a TRSM leaf as one GEMM: X = gamma inv(M_ii) Y_i (beta = 0)
            r, e = s["rc"], min(k, s["rc"] + s["mlen"])
            assert s["beta"] == 0 and s["rk"] == r and s["klen"] == e - r
            W = sla.solve_triangular(np.tril(M[r:e, r:e]), np.eye(e - r), lower=True)
            C[r:e] = s["gamma"] * (W @ Y[r:e])
        elif s["kind"] == "leaf":
            for t in range(s["nleaves"]):
                r = s["r0"] + t * s["b"]
                e = min(k, r + s["b"])
                if r >= k:
                    continue
                L = np.tril(M[r:e, r:e])
                if s["trsm"]:
                    C[r:e] = sla.solve_triangular(L, s["alpha"] * C[r:e], lower=True)
                    Y[r:e] = C[r:e]
                else:
                    C[r:e] = s["alpha"] * (L @ C[r:e])
        elif s["kind"] == "gemm" and s["dense"]:
            # per-row beta times the diagonal on C's old value, the strictly
            # lower part of the tile's rows (columns rk .. row) from the Y planes
            r, e, rk = s["rc"], min(k, s["rc"] + s["mlen"]), s["rk"]
            d = np.diag(M[r:e, r:e])[:, None]
            C[r:e] = s["beta"] * d * C[r:e] + s["gamma"] * (
                M[r:e, rk:r] @ Y[rk:r] + np.tril(M[r:e, r:e], -1) @ Y[r:e])
        elif s["kind"] == "thin":
            # the thin solve on rows [r0, r0 + b), then (planes) their Y planes
            r, e = s["r0"], min(k, s["r0"] + s["b"])
            assert s["trsm"] == 1
            C[r:e] = sla.solve_triangular(np.tril(M[r:e, r:e]), s["alpha"] * C[r:e], lower=True)
            if s["planes"]:
                Y[r:e] = C[r:e]
        elif s["kind"] == "gemm":
            # tensor-core updates read the Y planes (X for TRSM, the original
            # right-hand side for TRMM), the CUDA-core ones C itself
            src = Y if s["tc"] else C
            rc, rk = s["rc"], s["rk"]
            C[rc:rc + s["mlen"]] = (s["beta"] * C[rc:rc + s["mlen"]] + s["gamma"] *
                                    M[rc:rc + s["mlen"], rk:rk + s["klen"]] @ src[rk:rk + s["klen"]])
        if s["kind"] == "gemm" and s.get("y1", 0) > s.get("y0", 0):
            Y[s["y0"]:s["y1"]] = C[s["y0"]:s["y1"]]      # the epilogue's planes
    return C


@pytest.mark.parametrize("op", ["S", "M"])
@pytest.mark.parametrize("gemm", [1, 2])
@pytest.mark.parametrize("b", LEAVES)
@pytest.mark.parametrize("k", [1, 17, 65, 255, 300, 513])
def test_replay_matches_oracle(op, gemm, b, k):
    n = 7
    A, B = inputs.problem("L", "L", k, n, seed=k + b, dtype=np.float64)
    M = np.where(np.isnan(A), 0.0, A)
    steps = debug_plan(op, "L", "L", "N", "N", k, n, 4, b, gemm)
    got = replay(op, steps, M, B)
    want = (oracle.trsm if op == "S" else oracle.trmm)("L", "L", "N", "N", 2.0, A, B)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


@pytest.mark.parametrize("dense", [64, 128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("k", [65, 300, 513, 1100, 2500])
@pytest.mark.parametrize("unit", ["N", "U"])
def test_trmm_dense_replay_matches_oracle(dense, k, unit):
    # TRMM leaves as dense diagonal-block GEMMs (Y planes hold the original
    # right-hand side; the diagonal term through the per-row beta)
    n = 5
    A, B = inputs.problem("L", "L", k, n, seed=k + dense, dtype=np.float64)
    M = np.where(np.isnan(A), 0.0, A)
    if unit == "U":
        np.fill_diagonal(M, 1.0)
    steps = debug_plan("M", "L", "L", "N", unit, k, n, 4, 0, 2, dense)
    assert steps[0] == {"kind": "conv_m", "diag_block": dense}
    assert any(s.get("dense") for s in steps) and not any(s["kind"] == "leaf" for s in steps)
    assert np.all(coverage(k, steps)[np.tril(np.ones((k, k), dtype=bool))] == 1)
    got = replay("M", steps, M, B)
    want = oracle.trmm("L", "L", "N", unit, 2.0, A, B)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


def test_trmm_level_batching():
    # b a multiple of the K tile on the tensor-core path: one launch for all
    # leaves, then one grouped launch per level with disjoint output rows.
    steps = debug_plan("M", "L", "L", "N", "N", 16384, 16384, 4, 64, 0, -1)
    kinds = [s["kind"] for s in steps]
    assert kinds[:3] == ["conv_m", "conv_y", "leaf"] and steps[2]["nleaves"] == 256
    gemms = [s for s in steps if s["kind"] == "gemm"]
    assert len(gemms) == 255
    groups, cur = [], []
    for s in gemms:
        if s["member"] == 0 and cur:
            groups.append(cur)
            cur = []
        cur.append(s)
    groups.append(cur)
    assert [len(g) for g in groups] == [2 ** d for d in range(8)]
    for g in groups:
        rows = np.zeros(16384, dtype=int)
        for s in g:
            rows[s["rc"]:s["rc"] + s["mlen"]] += 1
        assert rows.max() == 1


def test_trmm_dense_diagonal_blocks_by_default():
    # automatic at order >= 1024: 1024-row diagonal blocks in one grouped
    # launch (128-row tiles, K up to each tile's last row), then one launch
    # per level above them (node sizes 16384 .. 2048)
    steps = debug_plan("M", "L", "L", "N", "N", 16384, 16384, 4, 0, 0)
    assert steps[0] == {"kind": "conv_m", "diag_block": 1024}
    assert steps[1]["kind"] == "conv_y"
    dense = [s for s in steps if s["kind"] == "gemm" and s["dense"]]
    assert len(dense) == 128 and all(s["mlen"] == 128 and s["beta"] == 2.0 for s in dense)
    assert sorted({s["klen"] for s in dense}) == list(range(128, 1025, 128))
    assert not any(s["kind"] == "leaf" for s in steps)
    levels = [s for s in steps if s["kind"] == "gemm" and not s["dense"]]
    assert len(levels) == 15 and min(s["klen"] for s in levels) == 1024
    # below the order threshold, with an explicit leaf, or switched off: leaves
    for args in [(1000, 0, 0), (16384, 64, 0), (16384, 0, -1)]:
        k, leaf, dense_opt = args
        steps = debug_plan("M", "L", "L", "N", "N", k, 64, 4, leaf, 0, dense_opt)
        assert steps[0]["diag_block"] == 0 and any(s["kind"] == "leaf" for s in steps)
    # TRSM never uses it
    steps = debug_plan("S", "L", "L", "N", "N", 16384, 64, 4, 0, 0, 256)
    assert steps[0]["diag_block"] == 0 and not any(s.get("dense") for s in steps)


def test_trsm_block_leaves_on_request():
    # cutoff 256 (TRSM block leaves) only when asked for; TRMM stops at 128
    leaves = [s for s in debug_plan("S", "L", "L", "N", "N", 16384, 16384, 4, 256, 0)
              if s["kind"] == "leaf"]
    assert len(leaves) == 64 and all(s["b"] == 256 for s in leaves)
    # automatic: 128-row leaves for FP32 TRSM (outside the thin leaves'
    # range of right-hand sides, test_thin_leaf_automatic_rule), 64-row
    # leaves for FP64
    for args in [("L", 16384, 16384), ("L", 16384, 2048), ("L", 2048, 256), ("R", 300, 3000)]:
        side, m, n = args
        leaves = [s for s in debug_plan("S", side, "L", "N", "N", m, n, 4, 0, 0)
                  if s["kind"] == "leaf"]
        k = m if side == "L" else n
        assert len(leaves) == -(-k // 128) and leaves[0]["b"] == 128, args
    leaves = [s for s in debug_plan("S", "L", "L", "N", "N", 16384, 16384, 8, 0, 0)
              if s["kind"] == "leaf"]
    assert all(s["b"] == 64 for s in leaves)
    leaves = [s for s in debug_plan("M", "L", "L", "N", "N", 16384, 16384, 4, 256, 0)
              if s["kind"] == "leaf"]
    assert leaves[0]["b"] == 128


def test_fp64_and_small_orders_use_cuda_cores():
    assert all(not s.get("tc", 0) for s in debug_plan("S", "L", "L", "N", "N", 4096, 8, 8, 0, 0))
    assert all(s["kind"] not in ("conv_m", "conv_y")
               for s in debug_plan("S", "L", "L", "N", "N", 200, 8, 4, 0, 0))
    assert any(s.get("tc", 0) for s in debug_plan("S", "L", "L", "N", "N", 256, 8, 4, 0, 0))
    # one leaf covering the whole order: no update, so no operand planes
    assert not any(s["kind"] in ("conv_m", "conv_y") or s.get("tc", 0)
                   for s in debug_plan("S", "L", "L", "N", "N", 100, 8, 4, 0, 0))


@pytest.mark.parametrize("k", [256, 300, 1024, 1100, 2049])
@pytest.mark.parametrize("leaf", [0, 64, 128])
def test_trsm_tensor_core_leaves_replay_and_feeding(k, leaf):
    """TRX_OPT_TRSM_TC_LEAF: every full leaf becomes an inverse GEMM whose
    input planes were written just before it (by the preceding update's
    epilogue, or a conversion for the first leaf); a ragged last leaf stays
    a substitution leaf. Replayed in FP64 (unset planes are NaN) it solves
    the system."""
    steps = debug_plan("S", "L", "L", "N", "N", k, 7, 4, leaf, 0, 0, 1)
    b = 128 if leaf == 0 else leaf
    assert steps[0]["kind"] == "conv_m" and steps[1] == {"kind": "inv_diag", "b": b}
    inv = [i for i, s in enumerate(steps) if s["kind"] == "gemm" and s["inv"]]
    assert len(inv) == k // b
    for n_, i in enumerate(inv):
        g, prev = steps[i], steps[i - 1]
        assert g["mlen"] == b and g["rc"] % b == 0 and (g["y0"], g["y1"]) == (g["rc"], g["rc"] + b)
        if n_ == 0:
            assert prev == {"kind": "conv_y_rows", "r0": g["rc"], "b": b}
        else:
            assert prev["kind"] == "gemm" and not prev["inv"] and prev["rc"] == g["rc"]
            assert (prev["y0"], prev["y1"]) == (g["rc"], g["rc"] + b)
    leaves = [s for s in steps if s["kind"] == "leaf"]
    assert [s["b"] for s in leaves] == ([k % b] if k % b else [])
    rng = np.random.default_rng(k + leaf)
    M = np.tril(rng.uniform(-1, 1, (k, k)) / k) + np.diag(1 + rng.random(k))
    C = rng.standard_normal((k, 7))
    X = replay("S", steps, M, C)
    np.testing.assert_allclose(M @ X, 2.0 * C, atol=1e-9)


def test_trsm_tensor_core_leaves_only_when_asked():
    for args in [dict(trsm_tc_leaf=0), dict(trsm_tc_leaf=-1), dict(trsm_tc_leaf=1, elem=8),
                 dict(trsm_tc_leaf=1, gemm=1), dict(trsm_tc_leaf=1, leaf=32)]:
        steps = debug_plan("S", "L", "L", "N", "N", 1024, 7, args.get("elem", 4),
                           args.get("leaf", 0), args.get("gemm", 0), 0, args["trsm_tc_leaf"])
        assert not any(s["kind"] in ("inv_diag", "conv_y_rows") or s.get("inv") for s in steps)
    # TRMM is untouched by the option
    a = debug_plan("M", "L", "L", "N", "N", 1024, 7, 4, 0, 0, 0, 1)
    b = debug_plan("M", "L", "L", "N", "N", 1024, 7, 4, 0, 0, 0, 0)
    assert a == b


@pytest.mark.parametrize("gemm", [1, 2])
@pytest.mark.parametrize("tl", [256, 512, 1024])
@pytest.mark.parametrize("k", [300, 1100, 2500])
def test_thin_leaf_plan_replay_matches_oracle(gemm, tl, k):
    # TRSM leaves of tl rows as thin solves (TRX_OPT_THIN_LEAF), tensor-core
    # path only: the leaves tile the order in sequence, alpha enters the
    # first, every leaf but none of the updates' inputs lacks its Y planes
    n = 7
    A, B = inputs.problem("L", "L", k, n, seed=k + tl, dtype=np.float64)
    M = np.where(np.isnan(A), 0.0, A)
    steps = debug_plan("S", "L", "L", "N", "N", k, n, 4, 0, gemm, 0, 0, tl)
    thin = [s for s in steps if s["kind"] == "thin"]
    if gemm == 1 or k <= tl:
        assert not thin
    else:
        assert not any(s["kind"] == "leaf" for s in steps)
        assert [s["r0"] for s in thin] == sorted(s["r0"] for s in thin)
        assert thin[0]["r0"] == 0 and all(
            a["r0"] + a["b"] == b["r0"] for a, b in zip(thin, thin[1:]))
        assert thin[-1]["r0"] + thin[-1]["b"] == k and all(s["b"] <= tl for s in thin)
        assert thin[0]["alpha"] == 2.0 and all(s["alpha"] == 1.0 for s in thin[1:])
        assert all(s["planes"] == 1 for s in thin)
    got = replay("S", steps, M, B)
    want = oracle.trsm("L", "L", "N", "N", 2.0, A, B)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


@pytest.mark.parametrize("k,n,leaf,want", [
    (8192, 256, 0, 2048), (16384, 128, 0, 2048), (16384, 512, 0, 1024), (4096, 1024, 0, 1024),
    (4096, 128, 0, 0), (4096, 256, 0, 2048), (16384, 64, 0, 0), (16384, 2048, 0, 0),
    (2048, 256, 0, 0), (8192, 256, 128, 0)])
def test_thin_leaf_automatic_rule(k, n, leaf, want):
    # the automatic thin leaves: order from 4096, 65..1024 right-hand sides
    # (129.. below order 8192), 2048 rows up to 256, 1024 above; off when
    # the leaf size is set explicitly
    steps = debug_plan("S", "L", "L", "N", "N", k, n, 4, leaf, 0)
    sizes = {s["b"] for s in steps if s["kind"] == "thin"}
    assert sizes == ({want} if want else set())
