"""CUDA path against the FP64 CPU oracle, element by element through the
normwise criteria of the problem statement: TRSM backward error
||op(A) X - alpha B|| / (||op(A)|| ||X||) <= 8 k u, TRMM
||C - C_oracle|| / (|alpha| ||op(A)|| ||B||) <= 8 k u (u of the working
precision, k the order of A, infinity norms). Inputs are the seeded
generator of paper_2504_13821_gb300.inputs (unreferenced triangle and, for
unit diagonals, the diagonal filled with NaN; ldb padding with a sentinel).
"""
import numpy as np
import pytest

from helpers import SENTINEL, bound, run_case, to_dev
import oracle
from paper_2504_13821_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = inputs.VARIANTS
SHAPES = [(1, 5), (17, 3), (64, 64), (129, 40), (300, 257)]


@pytest.fixture(scope="module")
def trx():
    import paper_2504_13821_gb300 as trx
    return trx


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("op", ["trsm", "trmm"])
@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_all_variants(trx, op, side, uplo, trans, diag, dtype):
    for i, (m, n) in enumerate(SHAPES):
        run_case(op, side, uplo, trans, diag, m, n, 1.5, dtype,
                 seed=inputs.variant_seed(m * 1000 + n, VARIANTS.index((side, uplo, trans, diag))))


@pytest.mark.parametrize("op", ["trsm", "trmm"])
@pytest.mark.parametrize("engine", [1, 2], ids=["cuda_cores", "tensor_cores"])
@pytest.mark.parametrize("leaf", [16, 32, 64, 128, 256])
@pytest.mark.parametrize("variant", [("L", "L", "N", "N"), ("R", "U", "T", "U"),
                                     ("L", "U", "N", "U"), ("R", "L", "N", "N")])
def test_leaf_and_engine_sweep(trx, op, engine, leaf, variant):
    h = trx.Handle(0)
    h.set_option(trx.OPT_LEAF, leaf)
    h.set_option(trx.OPT_GEMM, engine)
    side = variant[0]
    m, n = (1000, 300) if side == "L" else (300, 1000)
    run_case(op, *variant, m, n, -2.0, np.float32, seed=leaf + engine, handle=h)
    h.close()


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_trmm_dense_diagonal_blocks_all_variants(trx, side, uplo, trans, diag):
    """FP32 TRMM at order 1100 on a default handle: 256-row dense diagonal
    blocks on the tensor cores (automatic from order 1024), a ragged last
    block of 76 rows; unit diagonals poisoned with NaN in A."""
    m, n = (1100, 300) if side == "L" else (300, 1100)
    run_case("trmm", side, uplo, trans, diag, m, n, 1.5, np.float32,
             seed=inputs.variant_seed(1100, VARIANTS.index((side, uplo, trans, diag))))


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_factor_calls_all_variants(trx, side, uplo, trans, diag):
    """Prepared factor (planes made once): TRSM and TRMM through it equal the
    plain calls bitwise, match the oracle, and follow A after an in-place
    change and update()."""
    k, nrhs = 1100, 300
    m, n = (k, nrhs) if side == "L" else (nrhs, k)
    vi = VARIANTS.index((side, uplo, trans, diag))
    A, B = inputs.problem(side, uplo, m, n, seed=inputs.variant_seed(k, vi), dtype=np.float32,
                          poison_diag=(diag == "U"))
    dev = torch.device("cuda", 0)
    At = to_dev(A, dev)
    f = trx.Factor(side, uplo, trans, diag, At)
    for op in ("trsm", "trmm"):
        plain, via = to_dev(B, dev), to_dev(B, dev)
        getattr(trx, op)(side, uplo, trans, diag, 0.75, At, plain)
        getattr(f, op)(0.75, via)
        torch.cuda.synchronize()
        assert torch.equal(plain, via), op
    # A changes in place: after update() the factor uses the new values
    A2, _ = inputs.problem(side, uplo, m, n, seed=inputs.variant_seed(k + 1, vi),
                           dtype=np.float32, poison_diag=(diag == "U"))
    At.copy_(to_dev(A2, dev))
    f.update()
    X = to_dev(B, dev)
    f.trsm(0.75, X)
    torch.cuda.synchronize()
    eta = oracle.trsm_backward_error(side, uplo, trans, diag, 0.75, A2,
                                     np.asfortranarray(X.cpu().numpy()), B)["eta"]
    assert eta <= bound(k, np.float32)
    f.close()


@pytest.mark.parametrize("op", ["trsm", "trmm"])
@pytest.mark.parametrize("side", ["L", "R"])
def test_two_panels_equal_one_call(trx, op, side):
    """Right-hand-side sharding (one panel per rank) run as two calls on one
    GPU: the gathered panels equal the single call (same plan choices:
    cutoff fixed, sizes under the automatic thresholds), bitwise."""
    from paper_2504_13821_gb300.sharding import solve_panel
    m, n = (2048, 4000) if side == "L" else (4000, 2048)
    A, B = inputs.problem(side, "U", m, n, seed=4000, dtype=np.float32)
    At = to_dev(A, "cuda:0")
    whole, parts = to_dev(B, "cuda:0"), to_dev(B, "cuda:0")
    h = trx.Handle(0)
    h.set_option(trx.OPT_LEAF, 64)
    fn = trx.trsm if op == "trsm" else trx.trmm
    fn(side, "U", "T", "N", 1.25, At, whole, handle=h)
    covered = []
    for rank in range(2):
        covered.append(solve_panel("S" if op == "trsm" else "M", side, "U", "T", "N", 1.25, At,
                                   parts, 2, rank, handle=h))
    torch.cuda.synchronize()
    assert covered[0][0] == 0 and covered[0][1] == covered[1][0] and covered[1][1] == 4000
    assert torch.equal(whole, parts)
    h.close()


@pytest.mark.parametrize("engine", [1, 2], ids=["cuda_cores", "tensor_cores"])
@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_wide_leaves_all_variants(trx, side, uplo, trans, diag, engine):
    """FP32 TRSM with 128-row leaves and many right-hand sides (the wide
    leaf kernel): k = 600 leaves a ragged last leaf of 88 rows, 4200
    right-hand sides a ragged last 32-column panel."""
    h = trx.Handle(0)
    h.set_option(trx.OPT_LEAF, 128)
    h.set_option(trx.OPT_GEMM, engine)
    m, n = (600, 4200) if side == "L" else (4200, 600)
    run_case("trsm", side, uplo, trans, diag, m, n, 1.5, np.float32,
             seed=inputs.variant_seed(600 + engine, VARIANTS.index((side, uplo, trans, diag))),
             handle=h, ldb_pad=3)
    h.close()


@pytest.mark.parametrize("k", [1, 15, 100, 128])
def test_wide_leaf_single(trx, k):
    # one leaf of k <= 128 rows over 2050 right-hand sides, alpha applied once
    h = trx.Handle(0)
    h.set_option(trx.OPT_LEAF, 128)
    run_case("trsm", "L", "L", "N", "N", k, 2050, -0.5, np.float32, seed=k, handle=h)
    run_case("trsm", "R", "U", "T", "U", 2050, k, 3.0, np.float32, seed=k + 1, handle=h)
    h.close()


@pytest.mark.parametrize("dense", [-1, 64, 128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("variant", [("L", "L", "N", "N"), ("R", "U", "T", "U")])
def test_trmm_dense_sizes(trx, dense, variant):
    h = trx.Handle(0)
    h.set_option(trx.OPT_GEMM, 2)
    h.set_option(trx.OPT_TRMM_DENSE, dense)
    m, n = (700, 200) if variant[0] == "L" else (200, 700)
    run_case("trmm", *variant, m, n, -0.75, np.float32, seed=700 + dense, handle=h, ldb_pad=5)
    h.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_block_leaves_all_variants(trx, side, uplo, trans, diag, dtype):
    """TRSM with the 256-row block leaves (cutoff 256; a ragged last leaf:
    k = 600), many right-hand sides."""
    h = trx.Handle(0)
    h.set_option(trx.OPT_LEAF, 256)
    m, n = (600, 4200) if side == "L" else (4200, 600)
    run_case("trsm", side, uplo, trans, diag, m, n, 1.5, dtype, handle=h,
             seed=inputs.variant_seed(600, VARIANTS.index((side, uplo, trans, diag))))
    h.close()


@pytest.mark.parametrize("op", ["trsm", "trmm"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_padded_leading_dimensions(trx, op, dtype):
    for side, uplo, trans, diag in (("L", "U", "T", "N"), ("R", "L", "N", "U")):
        run_case(op, side, uplo, trans, diag, 333, 270, 0.5, dtype, seed=3,
                 lda_pad=13, ldb_pad=5)


@pytest.mark.parametrize("op", ["trsm", "trmm"])
def test_alpha_zero_reads_no_a(trx, op):
    dev = torch.device("cuda", 0)
    A = trx.to_colmajor(torch.full((300, 300), float("nan"), device=dev))
    B = torch.randn(300, 40, device=dev).t().contiguous().t()
    getattr(trx, op)("L", "L", "N", "N", 0.0, A, B)
    torch.cuda.synchronize()
    assert torch.count_nonzero(B).item() == 0


def test_empty_problems(trx):
    dev = torch.device("cuda", 0)
    trx.trsm("L", "L", "N", "N", 1.0, torch.zeros(0, 0, device=dev), torch.zeros(0, 5, device=dev))
    trx.trmm("R", "L", "N", "N", 1.0, torch.zeros(0, 0, device=dev), torch.zeros(4, 0, device=dev))


def test_config1_exact(trx):
    """1024 x 256 FP32 TRSM (L, L, N, N), alpha = 1, seed 0."""
    eta, tol, _ = run_case("trsm", "L", "L", "N", "N", 1024, 256, 1.0, np.float32, seed=0)
    assert eta <= tol


@pytest.mark.parametrize("op", ["trsm", "trmm"])
def test_deterministic_and_graph_equals_direct(trx, op):
    outs = []
    for graph in (1, 1, 0):
        h = trx.Handle(0)
        h.set_option(trx.OPT_GRAPH, graph)
        _, _, X = run_case(op, "R", "U", "N", "N", 700, 900, 1.5, np.float32, seed=9, handle=h)
        outs.append(X)
        h.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("variant", [("L", "L", "N", "N"), ("R", "U", "T", "N")])
def test_column_panel_branches(trx, variant):
    """A TRSM split into column-panel branches (forked streams in one graph)
    gives the single-chain result."""
    outs = []
    for panels in (1, 3, 4):
        h = trx.Handle(0)
        h.set_option(trx.OPT_PANELS, panels)
        m, n = (1000, 3000) if variant[0] == "L" else (3000, 1000)
        _, _, X = run_case("trsm", *variant, m, n, 1.5, np.float32, seed=17, handle=h)
        outs.append(X.astype(np.float64))
        h.close()
    for X in outs[1:]:
        diff = np.abs(X - outs[0]).max() / np.abs(outs[0]).max()
        assert diff <= bound(1000, np.float32)


def test_profile_counts_launches(trx):
    h = trx.Handle(0)
    h.set_option(trx.OPT_PROFILE, 1)
    h.set_option(trx.OPT_LEAF, 64)
    run_case("trsm", "L", "L", "N", "N", 1024, 512, 1.0, np.float32, seed=1, handle=h)
    p = h.profile(reset=True)
    assert p["gemm_tc"]["launches"] == 15 and p["leaf_trsm"]["launches"] == 16
    assert p["gemm_tc"]["ms"] > 0 and p["gemm_tc"]["flops"] > 0
    assert h.profile()["gemm_tc"]["launches"] == 0
    # automatic cutoff for FP32 TRSM: 128-row leaves
    h.set_option(trx.OPT_LEAF, 0)
    run_case("trsm", "L", "L", "N", "N", 1024, 512, 1.0, np.float32, seed=1, handle=h)
    p = h.profile(reset=True)
    assert p["leaf_trsm"]["launches"] == 8 and p["gemm_tc"]["launches"] == 7
    h.close()


def sampled_case(op, side, k, nrhs, cols, dtype, seed, handle=None):
    """Full-size call, oracle on a sample of independent right-hand sides
    (columns for side L, rows for side R)."""
    import paper_2504_13821_gb300 as trx
    m, n = (k, nrhs) if side == "L" else (nrhs, k)
    A, B = inputs.problem(side, "L", m, n, seed=seed, dtype=dtype)
    dev = torch.device("cuda", 0)
    At, Bt = to_dev(A, dev), to_dev(B, dev)
    getattr(trx, op)(side, "L", "N", "N", 1.5, At, Bt, handle=handle)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(nrhs, size=min(cols, nrhs), replace=False))
    idx_t = torch.from_numpy(idx).to(dev)
    if side == "L":
        X = np.asfortranarray(Bt.index_select(1, idx_t).cpu().numpy())
        B0 = np.asfortranarray(B[:, idx])
    else:
        X = np.asfortranarray(Bt.index_select(0, idx_t).cpu().numpy())
        B0 = np.asfortranarray(B[idx, :])
    del Bt
    if op == "trsm":
        metric = oracle.trsm_backward_error(side, "L", "N", "N", 1.5, A, X, B0)["eta"]
    else:
        ref = oracle.trmm(side, "L", "N", "N", 1.5, A, B0)
        metric = oracle.trmm_error(side, "L", "N", "N", 1.5, A, X, ref, B0)
    assert metric <= bound(k, dtype), f"{op} k={k}: {metric:.3e}"
    return metric


@pytest.mark.slow
@pytest.mark.parametrize("op", ["trsm", "trmm"])
def test_large_sampled_4096(trx, op):
    sampled_case(op, "L", 4096, 4096, 64, np.float32, seed=4096)
    sampled_case(op, "R", 4096, 1024, 32, np.float64, seed=4097)


@pytest.mark.slow
@pytest.mark.parametrize("op", ["trsm", "trmm"])
def test_ragged_large_sampled(trx, op):
    # order and right-hand-side count off every tile and leaf boundary
    sampled_case(op, "L", 4099, 16383, 32, np.float32, seed=4099)
    sampled_case(op, "R", 3001, 9999, 32, np.float32, seed=3001)


@pytest.mark.slow
@pytest.mark.parametrize("op", ["trsm", "trmm"])
def test_bench_size_16384_sampled(trx, op):
    """The benchmark's workload (m = n = 16384, FP32, L L N N, alpha 1.5,
    default handle: tensor cores, cached graph), 32 sampled columns."""
    sampled_case(op, "L", 16384, 16384, 32, np.float32, seed=16384)


@pytest.mark.parametrize("side,uplo,trans,diag", VARIANTS)
def test_trsm_tensor_core_leaves_all_variants(trx, side, uplo, trans, diag):
    """TRX_OPT_TRSM_TC_LEAF: the full 128-row leaves of an order-1100 FP32
    TRSM as inverse GEMMs (input planes from the preceding update's
    epilogue), the ragged 76-row last leaf by substitution; unit diagonals
    poisoned with NaN in A."""
    h = trx.Handle(0)
    h.set_option(trx.OPT_TRSM_TC_LEAF, 1)
    m, n = (1100, 300) if side == "L" else (300, 1100)
    run_case("trsm", side, uplo, trans, diag, m, n, 1.5, np.float32,
             seed=inputs.variant_seed(1101, VARIANTS.index((side, uplo, trans, diag))), handle=h)
    h.close()


@pytest.mark.parametrize("leaf,panels,nrhs", [(64, 0, 700), (128, 0, 2100), (128, 2, 2100)])
def test_trsm_tensor_core_leaves_sizes(trx, leaf, panels, nrhs):
    """64- and 128-row inverse-GEMM leaves, many right-hand sides, and two
    column-panel branches (each with its own planes window)."""
    h = trx.Handle(0)
    h.set_option(trx.OPT_TRSM_TC_LEAF, 1)
    h.set_option(trx.OPT_LEAF, leaf)
    if panels:
        h.set_option(trx.OPT_PANELS, panels)
    for variant in [("L", "L", "N", "N"), ("R", "U", "T", "U")]:
        m, n = (2048, nrhs) if variant[0] == "L" else (nrhs, 2048)
        run_case("trsm", *variant, m, n, -0.5, np.float32, seed=leaf + nrhs, handle=h)
    h.close()


def test_trsm_tensor_core_leaves_factor_equals_plain(trx):
    """A prepared factor made while the option is on carries the inverted
    diagonal blocks: its TRSM equals the plain call bitwise, its TRMM is the
    plain TRMM (the option does not touch TRMM)."""
    dev = torch.device("cuda", 0)
    h = trx.Handle(dev)
    h.set_option(trx.OPT_TRSM_TC_LEAF, 1)
    k, nrhs = 1536, 1000
    A, B = inputs.problem("L", "U", k, nrhs, seed=31, dtype=np.float32)
    At = to_dev(A, dev)
    f = trx.Factor("L", "U", "T", "N", At, handle=h)
    out = {}
    for op in ("trsm", "trmm"):
        plain, via = to_dev(B, dev), to_dev(B, dev)
        getattr(trx, op)("L", "U", "T", "N", 2.0, At, plain, handle=h)
        getattr(f, op)(2.0, via, handle=h)
        torch.cuda.synchronize()
        assert torch.equal(plain, via), op
        out[op] = np.asfortranarray(via.cpu().numpy())
    f.close()
    h.close()
    Ak = np.asfortranarray(A[:k, :k])
    eta = oracle.trsm_backward_error("L", "U", "T", "N", 2.0, Ak, out["trsm"], B)["eta"]
    assert eta <= bound(k, np.float32), eta


@pytest.mark.parametrize("op", ["trsm", "trmm"])
def test_checked_plans_and_nvtx_ranges(trx, op):
    """TRX_OPT_CHECKED validates every launch plan before enqueueing it and
    TRX_OPT_NVTX wraps each launch step in an NVTX range (direct launches):
    results unchanged, parity holds."""
    h = trx.Handle(0)
    h.set_option(trx.OPT_CHECKED, 1)
    h.set_option(trx.OPT_NVTX, 1)
    h.set_option(trx.OPT_GRAPH, 0)
    for variant, (m, n) in ((("L", "L", "N", "N"), (1100, 300)), (("R", "U", "T", "U"), (90, 700))):
        run_case(op, *variant, m, n, 1.5, np.float32, seed=m + n, handle=h)
    h.close()
