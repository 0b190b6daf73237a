"""Binding of the library's request server (trx_server_* in include/trx.h).

The scheduling (admission by slots and device-memory budget, small problems
batched per tick, large ones on the least-loaded of parallel streams, completion
by events) runs in the C library; this class marshals arguments and keeps
the tensors the device is still using alive: a right-hand side until its
request has completed, a factor until it is released and its last request
has completed.
"""
from __future__ import annotations

import collections
import ctypes

from . import _binding


class Server:
    """trx_server_t over torch tensors (column-major CUDA views)."""

    def __init__(self, device=0, streams: int = 4, budget_bytes: int = 150 << 30,
                 max_inflight: int = 4096, small_k: int = 512, workspace_bytes: int = 0,
                 graphs: bool = True, refine_corrections: int = 2, fp64_corrections: int = 0,
                 fp64_trmm: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device if isinstance(device, int) else
                                   torch.device(device).index or 0)
        lib = _binding.load_library()
        cfg = _binding.ServerConfig(streams, small_k, max_inflight, budget_bytes,
                                    workspace_bytes, int(graphs), refine_corrections,
                                    fp64_corrections, fp64_trmm)
        h = ctypes.c_void_p()
        _binding._check(lib.trx_server_create(self.device.index, ctypes.byref(cfg),
                                              ctypes.byref(h)), "trx_server_create")
        self._s = h
        self._factors = {}                     # id -> A (kept alive)
        self._released = set()
        self._outstanding = collections.Counter()
        self._requests = {}                    # id -> (factor id, B)
        self._cap = 4096
        self._ids = (ctypes.c_int64 * self._cap)()
        self._status = (ctypes.c_int * self._cap)()

    def register(self, A, uplo: str, trans: str = "N", diag: str = "N") -> int:
        """Keep a factor resident; returns its id."""
        ptr, lda = _binding._colmajor(A, "A")
        if A.shape[0] != A.shape[1]:
            raise ValueError("A must be square")
        fid = ctypes.c_int()
        _binding._check(_binding.load_library().trx_server_register_factor(
            self._s, _binding._char(uplo), _binding._char(trans), _binding._char(diag),
            A.shape[0], A.element_size(), ptr, lda, ctypes.byref(fid)),
            "trx_server_register_factor")
        self._factors[fid.value] = A
        return fid.value

    def release(self, fid: int):
        """No new requests for the factor; dropped after its last request."""
        _binding._check(_binding.load_library().trx_server_release_factor(self._s, fid),
                        "trx_server_release_factor")
        self._released.add(fid)
        self._drop(fid)

    def _drop(self, fid):
        if fid in self._released and self._outstanding[fid] == 0:
            self._factors.pop(fid, None)
            self._released.discard(fid)
            del self._outstanding[fid]

    def submit(self, fid: int, op: str, side: str, alpha: float, B, stream=None) -> int:
        """Queue B := op's result (in place); returns the request id. The
        request's launch waits for work already enqueued on `stream` (the
        current stream by default)."""
        A = self._factors[fid]
        if B.dtype != A.dtype or B.device != A.device:
            raise TypeError("B must match the factor's dtype and device")
        ptr, ldb = _binding._colmajor(B, "B")
        m, n = B.shape
        rid = ctypes.c_int64()
        _binding._check(_binding.load_library().trx_server_submit(
            self._s, fid, _binding._char(op), _binding._char(side), float(alpha), ptr, m, n, ldb,
            _binding._stream_ptr(stream, B.device), ctypes.byref(rid)), "trx_server_submit")
        self._requests[rid.value] = (fid, B)
        self._outstanding[fid] += 1
        return rid.value

    def submit_refined(self, fid: int, side: str, alpha: float, B, X, stream=None) -> int:
        """Queue a refined FP32 TRSM: X (float64) := the solution of
        op(A) X = alpha B (side 'L') or X op(A) = alpha B, B float32 (not
        modified); returns the request id."""
        torch = self.torch
        A = self._factors[fid]
        if A.dtype != torch.float32 or B.dtype != torch.float32 or X.dtype != torch.float64:
            raise TypeError("refined requests: float32 factor and B, float64 X")
        if tuple(X.shape) != tuple(B.shape):
            raise ValueError("X must have B's shape")
        bptr, ldb = _binding._colmajor(B, "B")
        xptr, ldx = _binding._colmajor(X, "X")
        m, n = B.shape
        rid = ctypes.c_int64()
        _binding._check(_binding.load_library().trx_server_submit_refined(
            self._s, fid, _binding._char(side), float(alpha), bptr, m, n, ldb, xptr, ldx,
            _binding._stream_ptr(stream, B.device), ctypes.byref(rid)),
            "trx_server_submit_refined")
        self._requests[rid.value] = (fid, (B, X))
        self._outstanding[fid] += 1
        return rid.value

    def poll(self) -> list[tuple[int, int]]:
        """One scheduling tick; returns the (request id, status) pairs that
        completed."""
        lib = _binding.load_library()
        out = []
        while True:
            cnt = ctypes.c_int()
            rc = lib.trx_server_poll(self._s, self._ids, self._status, self._cap,
                                     ctypes.byref(cnt))
            for i in range(cnt.value):
                rid = self._ids[i]
                fid, _ = self._requests.pop(rid)
                self._outstanding[fid] -= 1
                self._drop(fid)
                out.append((rid, self._status[i]))
            _binding._check(rc, "trx_server_poll")
            if cnt.value < self._cap:
                return out

    def pending(self) -> tuple[int, int, int]:
        """(queued, in flight, completed but not yet reported)."""
        w, f, u = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _binding._check(_binding.load_library().trx_server_pending(
            self._s, ctypes.byref(w), ctypes.byref(f), ctypes.byref(u)), "trx_server_pending")
        return w.value, f.value, u.value

    def wait(self):
        """Block until the oldest launch group in flight has finished."""
        _binding._check(_binding.load_library().trx_server_wait(self._s), "trx_server_wait")

    def drain(self) -> list[tuple[int, int]]:
        """Tick until nothing is queued or in flight; returns completions."""
        out = self.poll()
        while any(self.pending()):
            self.wait()
            out += self.poll()
        return out

    def close(self):
        if self._s:
            _binding.load_library().trx_server_destroy(self._s)
            self._s = None
            self._requests.clear()
            self._factors.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
