"""The C ABI without a GPU: the library loads, exports every function
include/trx.h declares, and checks its arguments (BLAS positions) before it
touches a handle or the device."""
import ctypes

import pytest
import torch

from paper_2504_13821_gb300 import _binding, build

ALL = ("trx_strsm", "trx_dtrsm", "trx_strmm", "trx_dtrmm")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _binding.load_library()


def test_exports_every_declared_function(lib):
    names = _binding.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def call(lib, name, side="L", uplo="L", trans="N", diag="N", m=4, n=3, A=1, lda=4, B=1, ldb=4,
         handle=None):
    return getattr(lib, name)(handle, side.encode(), uplo.encode(), trans.encode(),
                              diag.encode(), m, n, 1.0, A, lda, B, ldb, None)


@pytest.mark.parametrize("name", ALL)
def test_argument_positions(lib, name):
    assert call(lib, name, side="X") == -1
    assert call(lib, name, uplo="X") == -2
    assert call(lib, name, trans="X") == -3
    assert call(lib, name, diag="X") == -4
    assert call(lib, name, m=-1) == -5
    assert call(lib, name, n=-1) == -6
    assert call(lib, name, A=None) == -8
    assert call(lib, name, lda=3) == -9
    assert call(lib, name, side="R", lda=2) == -9
    assert call(lib, name, side="R", lda=3) == 1          # valid args, no handle
    assert call(lib, name, B=None) == -10
    assert call(lib, name, ldb=3) == -11
    # case-insensitive flags, 'C' accepted; then the missing handle is reported
    assert call(lib, name, side="l", uplo="u", trans="c", diag="u") == 1
    # empty problems skip the pointer checks but still need a handle
    assert call(lib, name, m=0, A=None, B=None, lda=1, ldb=1) == 1


def test_gemm_update_argument_positions(lib):
    f = lib.trx_sgemm_update
    ok = dict(M=4, N=3, K=64, A=1, lda=4, Y=1, ldy=64, C=1, ldc=4, engine=2)

    def g(**kw):
        a = dict(ok, **kw)
        return f(None, a["M"], a["N"], a["K"], 1.0, 1.0, a["A"], a["lda"], a["Y"], a["ldy"],
                 a["C"], a["ldc"], a["engine"], None)
    assert g(M=-1) == -2 and g(N=-1) == -3 and g(K=-1) == -4
    assert g(A=None) == -7 and g(lda=3) == -8 and g(Y=None) == -9 and g(ldy=63) == -10
    assert g(C=None) == -11 and g(ldc=3) == -12 and g(engine=0) == -13
    assert g() == 1


def test_error_strings(lib):
    assert lib.trx_error_string(0) == b"success"
    assert b"uplo" in lib.trx_error_string(-2)
    assert b"ldb" in lib.trx_error_string(-11)
    for code in range(1, 8):
        assert lib.trx_error_string(code) not in (b"", b"unknown error")
    assert lib.trx_error_string(99) == b"unknown error"
    assert lib.trx_version() >= 100


def test_handle_calls_reject_null(lib):
    assert lib.trx_set_option(None, 1, 64) == 1
    assert lib.trx_destroy(None) == 0
    assert lib.trx_check_device_error(None) == 1
    out = ctypes.c_size_t()
    assert lib.trx_workspace_size(None, b"S", b"L", 4, 4, 4, ctypes.byref(out)) == 1


def test_factor_calls_reject_bad_arguments(lib):
    import ctypes
    out = ctypes.c_void_p(1)
    # argument checks come before the handle: bad side (position 2), order (6)
    assert lib.trx_sfactor_create(None, b"X", b"L", b"N", b"N", 4, 1, 4, None,
                                  ctypes.byref(out)) == -2
    assert not out.value
    assert lib.trx_sfactor_create(None, b"L", b"L", b"N", b"N", -1, 1, 4, None,
                                  ctypes.byref(out)) == -6
    assert lib.trx_sfactor_create(None, b"L", b"L", b"N", b"N", 4, 1, 2, None,
                                  ctypes.byref(out)) == -8
    assert lib.trx_sfactor_create(None, b"L", b"L", b"N", b"N", 4, 1, 4, None,
                                  ctypes.byref(out)) == 1                  # TRX_ERR_HANDLE
    assert lib.trx_strsm_factor(None, None, 4, 1.0, None, 4, None) == 7    # TRX_ERR_INVALID_VALUE
    assert lib.trx_sfactor_update(None, None, None, None) == 1
    assert lib.trx_factor_destroy(None) == 0


def test_prepared_batch_calls_reject_null(lib):
    import ctypes
    out = ctypes.c_void_p(1)
    assert lib.trx_batch_create(None, 4, 0, None, ctypes.byref(out)) == 1    # TRX_ERR_HANDLE
    assert not out.value                                                      # cleared
    assert lib.trx_batch_run(None, None, None) == 1
    assert lib.trx_batch_destroy(None) == 0


@pytest.mark.skipif(torch.cuda.is_available(), reason="host without a GPU only")
def test_create_fails_cleanly_without_gpu(lib):
    h = ctypes.c_void_p()
    rc = lib.trx_create(ctypes.byref(h), 0, 0)
    assert rc != 0 and not h.value


def test_binding_rejects_bad_tensors():
    import paper_2504_13821_gb300 as trx
    A = torch.zeros(4, 4)
    with pytest.raises((TypeError, ValueError)):
        trx.trsm("L", "L", "N", "N", 1.0, A, torch.zeros(4, 3))   # CPU tensors
    with pytest.raises(TypeError):
        trx.trsm("L", "L", "N", "N", 1.0, A, torch.zeros(4, 3, dtype=torch.float64))


def test_refined_argument_positions(lib):
    import ctypes

    def r(side="L", m=4, n=3, A=1, lda=4, B=1, ldb=4, X=1, ldx=4, max_iter=3, tol=1e-12,
          uplo="L"):
        return lib.trx_strsm_refined(None, side.encode(), uplo.encode(), b"N", b"N", m, n, 1.0,
                                     A, lda, B, ldb, X, ldx, max_iter, tol, None, None)
    # the BLAS positions shifted by one (the handle comes first)
    assert r(side="X") == -2 and r(uplo="X") == -3 and r(m=-1) == -6 and r(n=-1) == -7
    assert r(A=None) == -9 and r(lda=3) == -10 and r(B=None) == -11 and r(ldb=3) == -12
    assert r(X=None) == -13 and r(ldx=3) == -14 and r(max_iter=-1) == -15
    assert r(tol=-1.0) == -16 and r(tol=float("nan")) == -16
    assert r() == 1                                            # valid, no handle
    assert r(m=0, A=None, B=None, X=None, lda=1, ldb=1, ldx=1) == 1
    info = _binding.RefineInfo(5, 1.0, 1.0, 1.0)
    lib.trx_strsm_refined(None, b"L", b"L", b"N", b"N", 4, 3, 1.0, 1, 4, 1, 4, 1, 4, 3, 0.0,
                          ctypes.byref(info), None)
    assert info.iterations == 5          # untouched when the handle is rejected


def test_server_calls_reject_bad_arguments(lib):
    import ctypes
    fid = ctypes.c_int(-7)
    r = lib.trx_server_register_factor
    assert r(None, b"X", b"N", b"N", 4, 4, 1, 4, ctypes.byref(fid)) == -2
    assert r(None, b"L", b"X", b"N", 4, 4, 1, 4, ctypes.byref(fid)) == -3
    assert r(None, b"L", b"N", b"X", 4, 4, 1, 4, ctypes.byref(fid)) == -4
    assert r(None, b"L", b"N", b"N", -1, 4, 1, 4, ctypes.byref(fid)) == -5
    assert r(None, b"L", b"N", b"N", 4, 2, 1, 4, ctypes.byref(fid)) == -6
    assert r(None, b"L", b"N", b"N", 4, 4, None, 4, ctypes.byref(fid)) == -7
    assert r(None, b"L", b"N", b"N", 4, 4, 1, 3, ctypes.byref(fid)) == -8
    assert r(None, b"L", b"N", b"N", 4, 4, 1, 4, None) == -9
    assert r(None, b"L", b"N", b"N", 4, 4, 1, 4, ctypes.byref(fid)) == 1     # TRX_ERR_HANDLE
    assert fid.value == -7
    rid = ctypes.c_int64()
    assert lib.trx_server_submit(None, 0, b"S", b"L", 1.0, 1, 4, 4, 4, None,
                                 ctypes.byref(rid)) == 1
    cnt = ctypes.c_int()
    assert lib.trx_server_poll(None, None, None, 0, ctypes.byref(cnt)) == 1
    assert lib.trx_server_pending(None, None, None, None) == 1
    assert lib.trx_server_wait(None) == 1
    assert lib.trx_server_release_factor(None, 0) == 1
    assert lib.trx_server_destroy(None) == 0


@pytest.mark.skipif(torch.cuda.is_available(), reason="host without a GPU only")
def test_server_create_fails_cleanly_without_gpu(lib):
    import ctypes
    s = ctypes.c_void_p(1)
    assert lib.trx_server_create(0, None, ctypes.byref(s)) != 0 and not s.value
    cfg = _binding.ServerConfig(0, 512, 16, 1 << 20, 0, 1)      # zero streams
    assert lib.trx_server_create(0, ctypes.byref(cfg), ctypes.byref(s)) == 7


def test_typed_batched_calls_check_the_operation(lib):
    import ctypes
    probs = (_binding.Problem * 2)()
    for p, op in zip(probs, (b"S", b"M")):
        p.op, p.side, p.uplo, p.transa, p.diag = op, b"L", b"L", b"N", b"N"
    # a mixed batch is refused by every typed entry point before the handle
    for name in ("trx_strsm_batched", "trx_dtrsm_batched", "trx_strmm_batched",
                 "trx_dtrmm_batched"):
        assert getattr(lib, name)(None, 2, probs, None) == 7
        assert getattr(lib, name)(None, -1, probs, None) == 7
    # a uniform batch passes the checks; then the missing handle is reported
    assert lib.trx_strsm_batched(None, 1, probs, None) == 1
    assert lib.trx_strmm_batched(None, 1, probs, None) == 7
    assert lib.trx_dtrmm_batched(None, 0, None, None) == 1


def test_copy_triangle_argument_positions(lib):
    f = lib.trx_copy_triangle_h2d

    def up(uplo="L", k=4, elem=4, host=1, ldh=4, dev=1, ldd=4):
        return f(uplo.encode(), k, elem, host, ldh, dev, ldd, None)

    assert up(uplo="X") == -1
    assert up(k=-1) == -2
    assert up(elem=2) == -3
    assert up(host=None) == -4
    assert up(ldh=3) == -5
    assert up(dev=None) == -6
    assert up(ldd=3) == -7
    # an empty triangle copies nothing and needs no pointers
    assert up(k=0, host=None, dev=None, ldh=1, ldd=1) == 0
    assert up(uplo="u", k=0, host=None, dev=None, ldh=1, ldd=1) == 0
