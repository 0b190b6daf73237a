"""Continuous-batching request loop for triangular solves and multiplies.

Factors (triangular matrices) are registered once and stay resident on the
device; requests name a factor, an operation (TRSM 'S' / TRMM 'M'), a side,
alpha and a right-hand side. The loop runs in ticks:

* admission: arrived requests are admitted while the device-memory budget
  (their right-hand sides plus the library workspace they need) and the
  in-flight slot count allow; the rest wait, and are admitted in a later
  tick as earlier work completes and frees budget and slots (continuous
  batching: admission does not wait for the GPU to drain);
* small problems (order <= TRX_BATCH_MAX_K) admitted in one tick go out as
  one persistent batched launch (trx_batched); larger ones go one call each
  to the recursive path, spread round-robin over parallel streams (one
  handle, and so one workspace, per stream);
* completion: every launch records a CUDA event; a request completes when
  its event has fired, and its latency is completion time minus arrival
  time (host clock).

The plan each request gets depends only on its own problem (size, element
type, variant), never on what else is in flight, so a result is the same
alone and in the mix.
"""
from __future__ import annotations

import collections
import dataclasses
import time

from . import _binding

SMALL_K = 512


@dataclasses.dataclass
class Factor:
    A: object              # column-major CUDA tensor (k x k)
    uplo: str
    trans: str
    diag: str


@dataclasses.dataclass
class Request:
    rid: int
    factor: int
    op: str                # 'S' or 'M'
    side: str
    alpha: float
    B: object              # column-major CUDA tensor, overwritten by the result
    arrival: float         # host clock (perf_counter seconds)
    admitted: float = 0.0
    done: float = 0.0


class Server:
    """Single-threaded scheduler over the trx C ABI."""

    def __init__(self, device=0, streams: int = 4, budget_bytes: int = 150 << 30,
                 max_inflight: int = 4096, keep_results: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self.handles = [_binding.Handle(self.device) for _ in range(streams)]
        self.batch_handle = _binding.Handle(self.device)
        self.batch_stream = torch.cuda.Stream(self.device)
        self.budget = budget_bytes
        self.max_inflight = max_inflight
        self.factors: list[Factor] = []
        self.waiting: collections.deque[Request] = collections.deque()
        self.inflight: list[tuple[object, list[Request], int]] = []  # (event, reqs, bytes)
        self.inflight_bytes = 0
        self.inflight_reqs = 0
        self.completed: list[Request] = []
        self._rr = 0
        self.outstanding = collections.Counter()   # factor id -> requests not done
        self.to_release: set[int] = set()
        self.keep_results = keep_results

    # -- registry ---------------------------------------------------------
    def register(self, A, uplo: str, trans: str = "N", diag: str = "N") -> int:
        """Keep a factor resident; returns its id."""
        self.factors.append(Factor(A, uplo, trans, diag))
        return len(self.factors) - 1

    def release(self, fid: int):
        """Drop a factor once the requests already submitted for it are done."""
        self.to_release.add(fid)
        self._maybe_release(fid)

    def _maybe_release(self, fid: int):
        if fid in self.to_release and self.outstanding[fid] == 0:
            self.factors[fid] = None
            self.to_release.discard(fid)

    def submit(self, req: Request):
        self.outstanding[req.factor] += 1
        self.waiting.append(req)

    # -- one scheduling tick ----------------------------------------------
    def _cost_bytes(self, req: Request) -> int:
        f = self.factors[req.factor]
        b = req.B.numel() * req.B.element_size()
        k = f.A.shape[0]
        if k > SMALL_K and req.B.element_size() == 4:
            b += 4 * k * (k + (req.B.shape[1] if req.side == "L" else req.B.shape[0]))
        return b

    def tick(self, now: float | None = None):
        """Retire finished work, admit what fits, launch it."""
        now = time.perf_counter() if now is None else now
        self._retire()
        small, large = [], []
        while self.waiting:
            req = self.waiting[0]
            if req.arrival > now:
                break
            cost = self._cost_bytes(req)
            if (self.inflight_reqs + len(small) + len(large) >= self.max_inflight or
                    self.inflight_bytes + cost > self.budget):
                break
            self.waiting.popleft()
            req.admitted = now
            self.inflight_bytes += cost
            (small if self.factors[req.factor].A.shape[0] <= SMALL_K else large).append((req, cost))
        if small:
            self._launch_small(small)
        for req, cost in large:
            self._launch_large(req, cost)

    def _launch_small(self, items):
        by_elem = collections.defaultdict(list)
        for req, cost in items:
            by_elem[req.B.element_size()].append((req, cost))
        for elem, group in by_elem.items():
            probs = []
            for req, _ in group:
                f = self.factors[req.factor]
                probs.append((req.op, req.side, f.uplo, f.trans, f.diag, req.alpha, f.A, req.B))
            # inputs were written on the submitting (current) stream
            self.batch_stream.wait_stream(self.torch.cuda.current_stream(self.device))
            _binding.batched(probs, handle=self.batch_handle, stream=self.batch_stream)
            ev = self.torch.cuda.Event()
            ev.record(self.batch_stream)
            nbytes = sum(c for _, c in group)
            self.inflight.append((ev, [r for r, _ in group], nbytes))
            self.inflight_reqs += len(group)

    def _launch_large(self, req: Request, cost: int):
        i = self._rr % len(self.streams)
        self._rr += 1
        f = self.factors[req.factor]
        fn = _binding.trsm if req.op == "S" else _binding.trmm
        self.streams[i].wait_stream(self.torch.cuda.current_stream(self.device))
        fn(req.side, f.uplo, f.trans, f.diag, req.alpha, f.A, req.B,
           handle=self.handles[i], stream=self.streams[i])
        ev = self.torch.cuda.Event()
        ev.record(self.streams[i])
        self.inflight.append((ev, [req], cost))
        self.inflight_reqs += 1

    def _retire(self):
        still = []
        now = time.perf_counter()
        for ev, reqs, nbytes in self.inflight:
            if ev.query():
                for r in reqs:
                    r.done = now
                    if not self.keep_results:
                        r.B = None          # its work has finished: safe to free
                    self.completed.append(r)
                    self.outstanding[r.factor] -= 1
                    self._maybe_release(r.factor)
                self.inflight_bytes -= nbytes
                self.inflight_reqs -= len(reqs)
            else:
                still.append((ev, reqs, nbytes))
        self.inflight = still

    def drain(self):
        while self.waiting or self.inflight:
            self.tick()

    def close(self):
        self.torch.cuda.synchronize(self.device)
        for h in self.handles + [self.batch_handle]:
            h.close()


def latency_stats(reqs) -> dict:
    """p50 / p99 latency (ms) and completions per second over a run."""
    import numpy as np
    if not reqs:
        return {"count": 0}
    lat = np.array([(r.done - r.arrival) * 1e3 for r in reqs])
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"count": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "solves_per_s": len(reqs) / span if span > 0 else None}
