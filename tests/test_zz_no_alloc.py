"""trx_strsm_noalloc: the FP32 TRSM for callers that cannot allocate device
memory (solves issued during CUDA-graph stream capture, inside frameworks
that own all device memory through their own pools, or in latency-bound
loops that must not trigger cudaMalloc). It keeps its scratch in a static
device array instead of a handle's workspace; its results must match the
regular handle-based trx_strsm within the tests' tolerance, on consecutive
calls that reuse (and so inherit the stale contents of) that array.

Collected last on purpose (file name), so a failure here comes after every
other test has run.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from helpers import bound, to_dev
import oracle
from paper_2504_13821_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(lib):
    f = lib.trx_strsm_noalloc
    c, i64, vp = ctypes.c_char, ctypes.c_int64, ctypes.c_void_p
    f.argtypes = [c, c, c, c, i64, i64, ctypes.c_float, vp, i64, vp, i64, vp]
    f.restype = ctypes.c_int
    return f


def _norm_inf(x):
    return np.abs(x).sum(axis=1).max() if x.size else 0.0


@pytest.mark.parametrize("side,uplo,trans,diag,m,n", [
    ("L", "L", "N", "N", 1024, 512),     # tensor-core path, planes in the static array
    ("R", "U", "T", "U", 300, 700),      # ragged, index-reversed, unit diagonal
])
def test_noalloc_matches_handle_path_twice(side, uplo, trans, diag, m, n):
    import paper_2504_13821_gb300 as trx
    lib = trx.load_library()
    f = _noalloc(lib)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    k = m if side == "L" else n
    for call, seed in enumerate((11, 12)):       # two calls in a row, different data
        A, B = inputs.problem(side, uplo, m, n, seed=seed + k, dtype=np.float32,
                              poison_diag=(diag == "U"))
        At = to_dev(A, dev)
        X_ref = to_dev(B, dev)
        trx.trsm(side, uplo, trans, diag, 1.5, At, X_ref)      # handle path
        X_na = to_dev(B, dev)
        rc = f(side.encode(), uplo.encode(), trans.encode(), diag.encode(), m, n, 1.5,
               At.data_ptr(), At.stride(1), X_na.data_ptr(), X_na.stride(1),
               stream.cuda_stream)
        assert rc == 0, f"call {call}: trx_strsm_noalloc returned {rc}"
        torch.cuda.synchronize()
        xr = X_ref.cpu().numpy().astype(np.float64)
        xn = X_na.cpu().numpy().astype(np.float64)
        tol = bound(k, np.float32)
        assert _norm_inf(xn - xr) <= tol * _norm_inf(xr), f"call {call}: differs from trx_strsm"
        eta = oracle.trsm_backward_error(side, uplo, trans, diag, 1.5, A,
                                         np.asfortranarray(xn), B)["eta"]
        assert eta <= tol, f"call {call}: backward error {eta:.3e} > {tol:.3e}"


def test_noalloc_rejects_oversized_problem_before_launch():
    import paper_2504_13821_gb300 as trx
    lib = trx.load_library()
    f = _noalloc(lib)
    dev = torch.device("cuda", 0)
    # k = 4096, nrhs = 4096 needs 192 MiB of planes (6-term split) > 64 MiB
    A = trx.to_colmajor(torch.eye(4096, device=dev))
    B = trx.to_colmajor(torch.ones(4096, 4096, device=dev))
    rc = f(b"L", b"L", b"N", b"N", 4096, 4096, 1.0, A.data_ptr(), 4096, B.data_ptr(), 4096,
           torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    assert rc == 3                                   # TRX_ERR_WORKSPACE
    assert b"scratch" in lib.trx_last_error_detail()
    assert torch.all(B == 1).item()                  # nothing was enqueued
    # BLAS argument positions come first
    assert f(b"X", b"L", b"N", b"N", 4, 4, 1.0, None, 4, None, 4, None) == -1
    assert f(b"L", b"L", b"N", b"N", 4, 4, 1.0, None, 4, None, 4, None) == -8


def test_noalloc_check_error_reports_a_timed_out_wait():
    """A bounded device-side wait that runs out is reported by
    trx_noalloc_check_error (read and clear), without a GPU fault: a child
    process sets the wait budget to 1 microsecond (TRX_NOALLOC_WAIT_NS, read
    at the device's set-up), so the tensor-core update's waits give up, the
    kernel records TRX_ERR_TIMEOUT and returns; the word reads 4 once, then
    0. The child exits normally (the context stays usable)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = textwrap.dedent("""
        import ctypes, sys
        import torch
        sys.path.insert(0, ROOT)
        import paper_2504_13821_gb300 as trx
        lib = trx.load_library()
        f = lib.trx_strsm_noalloc
        c, i64, vp = ctypes.c_char, ctypes.c_int64, ctypes.c_void_p
        f.argtypes = [c, c, c, c, i64, i64, ctypes.c_float, vp, i64, vp, i64, vp]
        dev = torch.device("cuda", 0)
        k = 1024
        A = trx.to_colmajor(torch.eye(k, device=dev) * 2 + torch.rand(k, k, device=dev).tril(-1) / k)
        B = trx.to_colmajor(torch.ones(k, 2048 // 4, device=dev))
        assert lib.trx_noalloc_check_error() == 0
        rc = f(b"L", b"L", b"N", b"N", k, B.shape[1], 1.0, A.data_ptr(), k, B.data_ptr(), k,
               torch.cuda.current_stream(dev).cuda_stream)
        assert rc == 0, rc
        torch.cuda.synchronize()
        first, second = lib.trx_noalloc_check_error(), lib.trx_noalloc_check_error()
        print("check_error", first, second)
        assert (first, second) == (4, 0), (first, second)
    """).replace("ROOT", repr(root))
    env = dict(os.environ, TRX_NOALLOC_WAIT_NS="1000")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "check_error 4 0" in r.stdout
