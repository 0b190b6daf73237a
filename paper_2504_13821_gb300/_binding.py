"""Thin ctypes binding over the trx C ABI (include/trx.h).

Argument marshalling only: torch tensors supply device pointers, leading
dimensions and the current CUDA stream; every step of TRSM/TRMM runs in the
library's own CUDA kernels. There is no fallback of any kind: if libtrx.so is
missing or the device is not a GB300 (sm_103), calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtrx.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "trx.h")

# Option and kernel-class codes (mirrors include/trx.h).
OPT_LEAF, OPT_GEMM, OPT_GRAPH, OPT_PROFILE, OPT_WAIT_LIMIT, OPT_PDL, OPT_PANELS = 1, 2, 3, 4, 5, 6, 7
OPT_TRMM_DENSE = 8
OPT_RESIDUAL = 9
OPT_TRSM_TC_LEAF = 10
OPT_SPLIT = 11          # tensor-core split: 1, 3 or 6 product terms (0: automatic, 6)
OPT_FP64_TRSM = 12      # trx_dtrsm: 0 DFMA recursion; n: FP32 solve + n float-float corrections
OPT_CHECKED = 13        # 1: validate every launch plan before enqueueing
OPT_NVTX = 14           # 1: NVTX range per launch step
OPT_TRSM_DAG = 15       # FP32 TRSM: 1 device-scheduled, -1 recursive chain, 0 automatic
OPT_FP64_TRMM = 16      # trx_dtrmm: 0 DFMA recursion; 1 one float-float pass (order >= 64)
OPT_THIN = 17           # FP32 TRSM, few right-hand sides: 1 one persistent launch, -1 recursion, 0 auto
OPT_TEST_WITHHOLD = 18  # test hook: the thin TRSM withholds its first block (waits run out)
OPT_THIN_LEAF = 19      # FP32 TRSM, tensor-core path: leaves of this many rows as thin solves (-1 off, 0 auto)
RESIDUAL_AUTO, RESIDUAL_FP64, RESIDUAL_FLOAT_FLOAT, RESIDUAL_TC = 0, 1, 2, 3
GEMM_AUTO, GEMM_SIMT, GEMM_TC = 0, 1, 2
KERNEL_CLASSES = ("leaf_trsm", "leaf_trmm", "gemm_tc", "gemm_simt", "convert", "other")
ERR_TIMEOUT = 4

_lock = threading.Lock()
_lib = None


class TrxError(RuntimeError):
    """A trx call returned a non-zero status."""

    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: trx error {code}"
        if _lib is not None:
            msg += f" ({_lib.trx_error_string(code).decode()})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class Problem(ctypes.Structure):
    """trx_problem_t: one entry of a batched call."""
    _fields_ = [("op", ctypes.c_char), ("side", ctypes.c_char), ("uplo", ctypes.c_char),
                ("transa", ctypes.c_char), ("diag", ctypes.c_char),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("alpha", ctypes.c_double),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64)]


class RefineInfo(ctypes.Structure):
    """trx_refine_info_t."""
    _fields_ = [("iterations", ctypes.c_int), ("residual_norm", ctypes.c_double),
                ("backward_error", ctypes.c_double),
                ("initial_backward_error", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    """trx_server_config_t."""
    _fields_ = [("streams", ctypes.c_int), ("small_k", ctypes.c_int),
                ("max_inflight", ctypes.c_int64), ("budget_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("graphs", ctypes.c_int),
                ("refine_corrections", ctypes.c_int), ("fp64_corrections", ctypes.c_int),
                ("fp64_trmm", ctypes.c_int)]


class _Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 6), ("flops", ctypes.c_double * 6),
                ("bytes", ctypes.c_double * 6), ("launches", ctypes.c_int64 * 6)]


def load_library() -> ctypes.CDLL:
    """Load libtrx.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"trx CUDA library not built ({LIB_PATH} missing): run "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, c = ctypes.c_void_p, ctypes.c_int64, ctypes.c_char
        lib.trx_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t]
        lib.trx_destroy.argtypes = [vp]
        lib.trx_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
        lib.trx_workspace_size.argtypes = [vp, c, c, i64, i64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_size_t)]
        for name, real in (("trx_strsm", ctypes.c_float), ("trx_strmm", ctypes.c_float),
                           ("trx_dtrsm", ctypes.c_double), ("trx_dtrmm", ctypes.c_double)):
            getattr(lib, name).argtypes = [vp, c, c, c, c, i64, i64, real, vp, i64, vp, i64, vp]
        lib.trx_set_option.argtypes = [vp, ctypes.c_int, i64]
        lib.trx_get_option.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i64)]
        lib.trx_get_profile.argtypes = [vp, ctypes.POINTER(_Profile), ctypes.c_int]
        lib.trx_check_device_error.argtypes = [vp]
        lib.trx_error_string.argtypes = [ctypes.c_int]
        lib.trx_error_string.restype = ctypes.c_char_p
        lib.trx_last_error_detail.argtypes = []
        lib.trx_last_error_detail.restype = ctypes.c_char_p
        lib.trx_debug_plan.argtypes = [c, c, c, c, c, i64, i64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_char_p, ctypes.c_size_t]
        lib.trx_sgemm_update.argtypes = [vp, i64, i64, i64, ctypes.c_float, ctypes.c_float,
                                         vp, i64, vp, i64, vp, i64, ctypes.c_int, vp]
        lib.trx_batched.argtypes = [vp, ctypes.c_int, i64, ctypes.POINTER(Problem), vp]
        for name in ("trx_strsm_batched", "trx_dtrsm_batched", "trx_strmm_batched",
                     "trx_dtrmm_batched"):
            getattr(lib, name).argtypes = [vp, i64, ctypes.POINTER(Problem), vp]
        lib.trx_batch_create.argtypes = [vp, ctypes.c_int, i64, ctypes.POINTER(Problem),
                                         ctypes.POINTER(vp)]
        lib.trx_sfactor_create.argtypes = [vp, c, c, c, c, i64, vp, i64, vp, ctypes.POINTER(vp)]
        lib.trx_sfactor_update.argtypes = [vp, vp, vp, vp]
        lib.trx_strsm_factor.argtypes = [vp, vp, i64, ctypes.c_float, vp, i64, vp]
        lib.trx_strmm_factor.argtypes = [vp, vp, i64, ctypes.c_float, vp, i64, vp]
        lib.trx_factor_destroy.argtypes = [vp]
        lib.trx_batch_run.argtypes = [vp, vp, vp]
        lib.trx_batch_destroy.argtypes = [vp]
        lib.trx_batched_autotune.argtypes = [vp, ctypes.c_int, i64, ctypes.POINTER(Problem), vp,
                                             ctypes.c_char_p, ctypes.c_size_t]
        lib.trx_strsm_refined.argtypes = [vp, c, c, c, c, i64, i64, ctypes.c_float, vp, i64, vp,
                                          i64, vp, i64, ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(RefineInfo), vp]
        lib.trx_strsm_refined_async.argtypes = [vp, c, c, c, c, i64, i64, ctypes.c_float, vp,
                                                i64, vp, i64, vp, i64, ctypes.c_int, vp]
        lib.trx_server_create.argtypes = [ctypes.c_int, ctypes.POINTER(ServerConfig),
                                          ctypes.POINTER(vp)]
        lib.trx_server_destroy.argtypes = [vp]
        lib.trx_server_register_factor.argtypes = [vp, c, c, c, i64, ctypes.c_int, vp, i64,
                                                   ctypes.POINTER(ctypes.c_int)]
        lib.trx_server_release_factor.argtypes = [vp, ctypes.c_int]
        lib.trx_server_submit.argtypes = [vp, ctypes.c_int, c, c, ctypes.c_double, vp, i64, i64,
                                          i64, vp, ctypes.POINTER(i64)]
        lib.trx_server_submit_refined.argtypes = [vp, ctypes.c_int, c, ctypes.c_double, vp, i64,
                                                  i64, i64, vp, i64, vp, ctypes.POINTER(i64)]
        lib.trx_server_poll.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int),
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.trx_server_pending.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                           ctypes.POINTER(i64)]
        lib.trx_server_wait.argtypes = [vp]
        lib.trx_version.argtypes = []
        lib.trx_batched_get_tuning.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.c_int]
        lib.trx_batched_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.c_int]
        lib.trx_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, i64,
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
        lib.trx_noalloc_check_error.argtypes = []
        lib.trx_copy_triangle_h2d.argtypes = [c, i64, ctypes.c_int, vp, i64, vp, i64, vp]
        _lib = lib
        return lib


def header_functions() -> list[str]:
    """Names of the functions include/trx.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(trx_[a-z0-9_]+)\s*\(", text)))


def _check(code: int, where: str):
    if code != 0:
        detail = _lib.trx_last_error_detail().decode() if code > 0 else ""
        raise TrxError(code, where, detail)


def _char(x: str) -> bytes:
    if not isinstance(x, str) or len(x) != 1:
        raise ValueError(f"expected a one-character flag, got {x!r}")
    return x.encode()


class Handle:
    """A trx handle on one CUDA device, with a torch-allocated workspace."""

    def __init__(self, device=None):
        import torch
        lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device()
                                   if device is None else torch.device(device).index or 0)
        self._h = ctypes.c_void_p()
        _check(lib.trx_create(ctypes.byref(self._h), self.device.index, 0), "trx_create")
        self._ws = None
        self._ws_bytes = 0

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            load_library().trx_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int):
        _check(load_library().trx_set_option(self._h, option, int(value)), "trx_set_option")

    def get_option(self, option: int) -> int:
        v = ctypes.c_int64()
        _check(load_library().trx_get_option(self._h, option, ctypes.byref(v)), "trx_get_option")
        return v.value

    def workspace_size(self, op: str, side: str, m: int, n: int, elem_bytes: int) -> int:
        out = ctypes.c_size_t()
        _check(load_library().trx_workspace_size(self._h, _char(op), _char(side), m, n,
                                                 elem_bytes, ctypes.byref(out)),
               "trx_workspace_size")
        return out.value

    def ensure_workspace(self, nbytes: int):
        """Grow the torch-owned workspace to at least nbytes."""
        import torch
        if nbytes <= self._ws_bytes:
            return
        ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        _check(load_library().trx_set_workspace(self._h, ws.data_ptr(), nbytes),
               "trx_set_workspace")
        self._ws, self._ws_bytes = ws, nbytes

    def profile(self, reset: bool = False) -> dict:
        p = _Profile()
        _check(load_library().trx_get_profile(self._h, ctypes.byref(p), int(reset)),
               "trx_get_profile")
        return {name: {"ms": p.ms[i], "flops": p.flops[i], "bytes": p.bytes[i],
                       "launches": p.launches[i]} for i, name in enumerate(KERNEL_CLASSES)}

    def check_device_error(self) -> int:
        """0, or the error code a bounded device-side wait left behind."""
        code = load_library().trx_check_device_error(self._h)
        if code not in (0, ERR_TIMEOUT):
            _check(code, "trx_check_device_error")
        return code


_handles: dict = {}


def default_handle(device=None) -> Handle:
    import torch
    idx = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    h = _handles.get(idx)
    if h is None:
        h = _handles[idx] = Handle(idx)
        # a persisted batched tuning table (save_tuning) named by the
        # environment is loaded into every default handle
        path = os.environ.get("TRX_TUNING_FILE")
        if path:
            load_tuning(path, handle=h)
    return h


def _colmajor(t, name: str):
    """(pointer, leading dimension) of a column-major 2-D tensor view."""
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D, got shape {tuple(t.shape)}")
    rows, cols = t.shape
    if rows > 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); "
                         f"use a transposed contiguous tensor, e.g. x.t().contiguous().t()")
    ld = t.stride(1) if cols > 1 else max(1, rows)
    if ld < max(1, rows):
        raise ValueError(f"{name}: leading dimension {ld} < rows {rows}")
    return t.data_ptr(), ld


def _call(op: str, side, uplo, trans, diag, alpha, A, B, handle=None, stream=None):
    import torch
    lib = load_library()
    if not (isinstance(A, torch.Tensor) and isinstance(B, torch.Tensor)):
        raise TypeError("A and B must be torch tensors")
    if A.dtype != B.dtype or A.dtype not in (torch.float32, torch.float64):
        raise TypeError(f"A and B must both be float32 or both float64 "
                        f"(got {A.dtype}, {B.dtype})")
    if not (A.is_cuda and B.is_cuda) or A.device != B.device:
        raise ValueError("A and B must be CUDA tensors on one device")
    m, n = B.shape
    k = m if side.upper() == "L" else n
    if tuple(A.shape) != (k, k):
        raise ValueError(f"A must be {k}x{k} for side {side!r} and B {m}x{n}")
    a_ptr, lda = _colmajor(A, "A")
    b_ptr, ldb = _colmajor(B, "B")
    h = handle if handle is not None else default_handle(B.device)
    elem = B.element_size()
    h.ensure_workspace(h.workspace_size("S" if op == "trsm" else "M", side, m, n, elem))
    if stream is None:
        stream = torch.cuda.current_stream(B.device)
    s_ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    fn = getattr(lib, ("trx_s" if elem == 4 else "trx_d") + op)
    rc = fn(h.ptr, _char(side), _char(uplo), _char(trans), _char(diag), m, n, float(alpha),
            a_ptr, lda, b_ptr, ldb, s_ptr)
    _check(rc, fn.__name__)
    return B


def trsm(side: str, uplo: str, trans: str, diag: str, alpha: float, A, B, *,
         handle: Handle | None = None, stream=None):
    """Solve op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R') in
    place: B (column-major CUDA tensor) is overwritten by X. Paper Eq. 3-4."""
    return _call("trsm", side, uplo, trans, diag, alpha, A, B, handle, stream)


def trmm(side: str, uplo: str, trans: str, diag: str, alpha: float, A, B, *,
         handle: Handle | None = None, stream=None):
    """B := alpha op(A) B (side 'L') or alpha B op(A) (side 'R') in place.
    Paper Eq. 1-2."""
    return _call("trmm", side, uplo, trans, diag, alpha, A, B, handle, stream)


def trsm_refined(side: str, uplo: str, trans: str, diag: str, alpha: float, A, B, *,
                 out=None, max_iter: int = 10, tol: float | None = None,
                 handle: Handle | None = None, stream=None):
    """FP32 solve of op(A) X = alpha B (or X op(A) = alpha B) refined in FP64.

    A and B are float32 CUDA tensors (B is not modified); the result is a
    float64 column-major tensor (``out`` if given). Each step forms the
    residual alpha B - op(A) X in FP64, solves for the correction in FP32 on
    the recursive path (Section 3.1) and adds it in FP64. ``tol`` bounds the
    normwise backward error ||R|| / (||op(A)|| ||X||) (infinity norms);
    by default sqrt(k) * 2**-53. The residual's arithmetic is the handle's
    OPT_RESIDUAL (float-float on the FP32 pipes unless set to RESIDUAL_FP64 or
    RESIDUAL_TC, the FP32-grade tensor-core residual for targets down to about
    1e-7). Returns (X, info) with info a dict:
    iterations, residual_norm, backward_error, initial_backward_error.
    """
    import torch
    lib = load_library()
    if not (isinstance(A, torch.Tensor) and isinstance(B, torch.Tensor)):
        raise TypeError("A and B must be torch tensors")
    if A.dtype != torch.float32 or B.dtype != torch.float32:
        raise TypeError(f"A and B must be float32 (got {A.dtype}, {B.dtype})")
    if not (A.is_cuda and B.is_cuda) or A.device != B.device:
        raise ValueError("A and B must be CUDA tensors on one device")
    m, n = B.shape
    k = m if side.upper() == "L" else n
    if tuple(A.shape) != (k, k):
        raise ValueError(f"A must be {k}x{k} for side {side!r} and B {m}x{n}")
    if out is None:
        out = torch.empty((n, m), dtype=torch.float64, device=B.device).t()
    if out.dtype != torch.float64 or tuple(out.shape) != (m, n) or out.device != B.device:
        raise ValueError(f"out must be a float64 {m}x{n} tensor on {B.device}")
    a_ptr, lda = _colmajor(A, "A")
    b_ptr, ldb = _colmajor(B, "B")
    x_ptr, ldx = _colmajor(out, "out")
    if tol is None:
        tol = max(k, 1) ** 0.5 * 2.0 ** -53
    h = handle if handle is not None else default_handle(B.device)
    need = h.workspace_size("S", side, m, n, 4)
    if h.get_option(OPT_RESIDUAL) == RESIDUAL_TC:
        # the tensor-core residual's TRMM uses the 6-term planes
        terms = h.get_option(OPT_SPLIT)
        h.set_option(OPT_SPLIT, 6)
        need = max(need, h.workspace_size("M", side, m, n, 4))
        h.set_option(OPT_SPLIT, terms)
    h.ensure_workspace(need)
    info = RefineInfo()
    rc = lib.trx_strsm_refined(h.ptr, _char(side), _char(uplo), _char(trans), _char(diag), m, n,
                               float(alpha), a_ptr, lda, b_ptr, ldb, x_ptr, ldx, int(max_iter),
                               float(tol), ctypes.byref(info), _stream_ptr(stream, B.device))
    _check(rc, "trx_strsm_refined")
    return out, {"iterations": info.iterations, "residual_norm": info.residual_norm,
                 "backward_error": info.backward_error,
                 "initial_backward_error": info.initial_backward_error}


def trsm_refined_async(side: str, uplo: str, trans: str, diag: str, alpha: float, A, B, *,
                       corrections: int = 2, out=None, handle: Handle | None = None,
                       stream=None):
    """FP32 solve plus a fixed number of float-float corrections, enqueued
    without any host read-back (trx_strsm_refined_async). A, B float32 CUDA
    tensors (B unchanged); returns the float64 result tensor (``out`` if
    given)."""
    import torch
    lib = load_library()
    if A.dtype != torch.float32 or B.dtype != torch.float32:
        raise TypeError(f"A and B must be float32 (got {A.dtype}, {B.dtype})")
    if not (A.is_cuda and B.is_cuda) or A.device != B.device:
        raise ValueError("A and B must be CUDA tensors on one device")
    m, n = B.shape
    k = m if side.upper() == "L" else n
    if tuple(A.shape) != (k, k):
        raise ValueError(f"A must be {k}x{k} for side {side!r} and B {m}x{n}")
    if out is None:
        out = torch.empty((n, m), dtype=torch.float64, device=B.device).t()
    a_ptr, lda = _colmajor(A, "A")
    b_ptr, ldb = _colmajor(B, "B")
    x_ptr, ldx = _colmajor(out, "out")
    h = handle if handle is not None else default_handle(B.device)
    h.ensure_workspace(h.workspace_size("S", side, m, n, 4))
    rc = lib.trx_strsm_refined_async(h.ptr, _char(side), _char(uplo), _char(trans), _char(diag),
                                     m, n, float(alpha), a_ptr, lda, b_ptr, ldb, x_ptr, ldx,
                                     int(corrections), _stream_ptr(stream, B.device))
    _check(rc, "trx_strsm_refined_async")
    return out


def debug_plan(op: str, side, uplo, trans, diag, m, n, elem_bytes=4, leaf=0, gemm=0,
               trmm_dense=0, trsm_tc_leaf=0, thin_leaf=0) -> list:
    """The launch sequence the library would enqueue, parsed (host only, no
    GPU needed): a list of dicts with the step kind and its row ranges."""
    lib = load_library()
    buf = ctypes.create_string_buffer(1 << 22)
    rc = lib.trx_debug_plan(_char(op), _char(side), _char(uplo), _char(trans), _char(diag),
                            m, n, elem_bytes, leaf, gemm, trmm_dense, trsm_tc_leaf, thin_leaf,
                            buf, len(buf))
    _check(rc, "trx_debug_plan")
    steps = []
    for line in buf.value.decode().splitlines():
        kind, *kv = line.split()
        d = {"kind": kind}
        for item in kv:
            key, val = item.split("=")
            d[key] = float(val) if "." in val or "e" in val else int(val)
        steps.append(d)
    return steps


def gemm_update(beta: float, gamma: float, A, Y, C, *, engine: int = GEMM_TC,
                handle: Handle | None = None, stream=None):
    """C := beta C + gamma A Y (FP32, column-major CUDA tensors): the
    recursion's off-diagonal update alone (Section 3.1)."""
    import torch
    lib = load_library()
    for t in (A, Y, C):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
            raise TypeError("A, Y, C must be float32 CUDA tensors")
    M, K = A.shape
    K2, N = Y.shape
    if K2 != K or tuple(C.shape) != (M, N):
        raise ValueError("shape mismatch")
    a, lda = _colmajor(A, "A")
    y, ldy = _colmajor(Y, "Y")
    c, ldc = _colmajor(C, "C")
    h = handle if handle is not None else default_handle(C.device)
    if engine == GEMM_TC:
        h.ensure_workspace(h.workspace_size("G", "L", M + K, N, 4))
    if stream is None:
        stream = torch.cuda.current_stream(C.device)
    s_ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(lib.trx_sgemm_update(h.ptr, M, N, K, float(beta), float(gamma), a, lda, y, ldy,
                                c, ldc, engine, s_ptr), "trx_sgemm_update")
    return C


class Factor:
    """A prepared FP32 triangle (trx_sfactor_create): its operand planes are
    made once (and again by update()), every trsm()/trmm() on it skips the
    conversion. A is a column-major CUDA tensor that must stay alive."""

    def __init__(self, side, uplo, trans, diag, A, *, handle: Handle | None = None,
                 stream=None):
        import torch
        if not (isinstance(A, torch.Tensor) and A.is_cuda and A.dtype == torch.float32):
            raise TypeError("A must be a float32 CUDA tensor")
        if A.shape[0] != A.shape[1]:
            raise ValueError("A must be square")
        self.side = side
        self.k = A.shape[0]
        self.A = A
        a, lda = _colmajor(A, "A")
        self.handle = handle if handle is not None else default_handle(A.device)
        self._f = ctypes.c_void_p()
        _check(load_library().trx_sfactor_create(self.handle.ptr, _char(side), _char(uplo),
                                                 _char(trans), _char(diag), self.k, a, lda,
                                                 _stream_ptr(stream, A.device),
                                                 ctypes.byref(self._f)), "trx_sfactor_create")

    def update(self, A=None, *, stream=None):
        """Re-make the planes from A (default: the current tensor, e.g. after
        its contents changed in place)."""
        if A is not None:
            self.A = A
        a, _ = _colmajor(self.A, "A")
        _check(load_library().trx_sfactor_update(self.handle.ptr, self._f, a,
                                                 _stream_ptr(stream, self.A.device)),
               "trx_sfactor_update")

    def _call(self, fn, alpha, B, handle, stream):
        import torch
        if not (isinstance(B, torch.Tensor) and B.is_cuda and B.dtype == torch.float32):
            raise TypeError("B must be a float32 CUDA tensor")
        b, ldb = _colmajor(B, "B")
        nrhs = B.shape[1] if self.side.upper() == "L" else B.shape[0]
        m, n = B.shape
        h = handle if handle is not None else self.handle
        h.ensure_workspace(h.workspace_size("Y", self.side, m, n, 4))
        _check(fn(h.ptr, self._f, nrhs, float(alpha), b, ldb, _stream_ptr(stream, B.device)),
               fn.__name__)
        return B

    def trsm(self, alpha, B, *, handle: Handle | None = None, stream=None):
        """B := X with op(A) X = alpha B (side L) or X op(A) = alpha B (side
        R); any handle on the factor's device may run it."""
        return self._call(load_library().trx_strsm_factor, alpha, B, handle, stream)

    def trmm(self, alpha, B, *, handle: Handle | None = None, stream=None):
        """B := alpha op(A) B (side L) or alpha B op(A) (side R)."""
        return self._call(load_library().trx_strmm_factor, alpha, B, handle, stream)

    def close(self):
        if self._f:
            load_library().trx_factor_destroy(self._f)
            self._f = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def copy_triangle_h2d(uplo: str, A_host, A_dev, *, stream=None):
    """Upload the triangle `uplo` (diagonal included) of the column-major
    k x k host tensor A_host into the column-major CUDA tensor A_dev
    (trx_copy_triangle_h2d): about half of A's bytes. Pinned A_host makes the
    copy asynchronous on `stream`."""
    import torch
    if A_host.device.type != "cpu" or A_dev.device.type != "cuda":
        raise ValueError("copy_triangle_h2d: A_host must be a CPU tensor and A_dev a CUDA one")
    if A_host.dtype != A_dev.dtype or A_host.dtype not in (torch.float32, torch.float64):
        raise TypeError("copy_triangle_h2d: A_host and A_dev must both be float32 or float64")
    if tuple(A_host.shape) != tuple(A_dev.shape) or A_host.shape[0] != A_host.shape[1]:
        raise ValueError("copy_triangle_h2d: A_host and A_dev must be the same square shape")
    hp, hld = _colmajor(A_host, "A_host")
    dp, dld = _colmajor(A_dev, "A_dev")
    _check(load_library().trx_copy_triangle_h2d(
        uplo.encode(), A_host.shape[0], A_host.element_size(), hp, hld, dp, dld,
        _stream_ptr(stream, A_dev.device)), "trx_copy_triangle_h2d")


def _stream_ptr(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _problem_array(problems):
    """ctypes array of trx_problem_t from (op, side, uplo, trans, diag, alpha,
    A, B) tuples of column-major CUDA tensors; also returns the element size."""
    import torch
    arr = (Problem * max(1, len(problems)))()
    elem = None
    for i, (op, side, uplo, trans, diag, alpha, A, B) in enumerate(problems):
        if A.dtype != B.dtype or A.dtype not in (torch.float32, torch.float64):
            raise TypeError(f"problem {i}: A and B must share float32/float64")
        if elem is None:
            elem = A.element_size()
        elif A.element_size() != elem:
            raise TypeError("all problems of a batch share one element type")
        a, lda = _colmajor(A, "A")
        b, ldb = _colmajor(B, "B")
        m, n = B.shape
        arr[i] = Problem(_char(op), _char(side), _char(uplo), _char(trans), _char(diag),
                         m, n, float(alpha), a, lda, b, ldb)
    return arr, (elem or 4)


class Batch:
    """A batch of (op, side, uplo, trans, diag, alpha, A, B) problems,
    prepared once on a handle (trx_batch_create: checked, canonicalised,
    cost-sorted, descriptors kept on the device); run() can be called
    repeatedly and does no host work (the tensors are referenced, not
    copied: their contents may change between runs, their storage not)."""

    def __init__(self, problems, *, handle: Handle | None = None):
        self.problems = list(problems)
        self.array, self.elem = _problem_array(self.problems)
        self.device = self.problems[0][7].device if self.problems else None
        self.handle = None
        self._b = ctypes.c_void_p()
        if self.problems:
            self.handle = handle if handle is not None else default_handle(self.device)
            _check(load_library().trx_batch_create(self.handle.ptr, self.elem, len(self.problems),
                                                   self.array, ctypes.byref(self._b)),
                   "trx_batch_create")

    def __len__(self):
        return len(self.problems)

    def run(self, *, handle: Handle | None = None, stream=None):
        import torch
        if not self.problems:
            return
        if handle is not None and handle is not self.handle:
            raise ValueError("a prepared batch runs on the handle it was created with")
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        s_ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(load_library().trx_batch_run(self.handle.ptr, self._b, s_ptr), "trx_batch_run")

    def close(self):
        if self._b:
            load_library().trx_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batched(problems, *, handle: Handle | None = None, stream=None):
    """Run many small TRSM ('S') / TRMM ('M') problems in one persistent
    launch. problems: list of (op, side, uplo, trans, diag, alpha, A, B)
    (checked and sorted on the host for this call: trx_batched), or a
    prepared Batch (no host work: trx_batch_run)."""
    import torch
    if isinstance(problems, Batch):
        problems.run(handle=handle, stream=stream)
        return
    problems = list(problems)
    if not problems:
        return
    arr, elem = _problem_array(problems)
    dev = problems[0][7].device
    h = handle if handle is not None else default_handle(dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    s_ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(load_library().trx_batched(h.ptr, elem, len(problems), arr, s_ptr), "trx_batched")


def batched_autotune(problems, *, handle: Handle | None = None, stream=None) -> dict:
    """Tune the batched kernel's sub-block height per order bucket on these
    problems (their B arrays are overwritten) and return the table."""
    import json
    import torch
    lib = load_library()
    arr, elem = _problem_array(problems)
    dev = problems[0][7].device
    h = handle if handle is not None else default_handle(dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    s_ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    buf = ctypes.create_string_buffer(16384)
    _check(lib.trx_batched_autotune(h.ptr, elem, len(problems), arr, s_ptr, buf, len(buf)),
           "trx_batched_autotune")
    return json.loads(buf.value.decode())


TUNE_ENTRIES = 4 * 3      # TRX_TUNE_K_BUCKETS * TRX_TUNE_N_BUCKETS


def save_tuning(path: str, *, handle: Handle | None = None):
    """Write the handle's batched tuning tables (both element types) as JSON."""
    import json
    lib = load_library()
    h = handle if handle is not None else default_handle()
    out = {}
    for name, elem in (("f32", 4), ("f64", 8)):
        t = (ctypes.c_int * TUNE_ENTRIES)()
        _check(lib.trx_batched_get_tuning(h.ptr, elem, t, TUNE_ENTRIES), "trx_batched_get_tuning")
        out[name] = list(t)
    out["layout"] = "order buckets k<=64,128,256,512 x right-hand-side buckets <=8,24,more"
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def load_tuning(path: str, *, handle: Handle | None = None):
    """Restore tables written by save_tuning into the handle."""
    import json
    lib = load_library()
    h = handle if handle is not None else default_handle()
    with open(path) as f:
        d = json.load(f)
    for name, elem in (("f32", 4), ("f64", 8)):
        if name in d:
            t = (ctypes.c_int * TUNE_ENTRIES)(*d[name])
            _check(lib.trx_batched_set_tuning(h.ptr, elem, t, TUNE_ENTRIES),
                   "trx_batched_set_tuning")


PEAK_KINDS = {"ffma": 0, "dfma": 1, "dmma": 2, "tc_tf32": 3, "tc_bf16": 4}


def peak_probe(kind: str, iters: int, device: int = 0) -> tuple[float, float]:
    """One launch of the library's peak-rate probe ``kind`` (PEAK_KINDS):
    (dense TFLOP/s, milliseconds)."""
    lib = load_library()
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.trx_peak_probe(int(device), PEAK_KINDS[kind], int(iters), ctypes.byref(t),
                              ctypes.byref(ms)), "trx_peak_probe")
    return t.value, ms.value


def to_colmajor(x):
    """Column-major copy of a 2-D tensor (same shape)."""
    return x.t().contiguous().t()
