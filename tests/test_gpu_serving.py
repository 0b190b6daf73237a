"""Serving loop: requests of mixed sizes, element types and operations
arrive while others are on the GPU and are admitted as budget and slots
free up (small ones batched per tick, large ones on parallel streams).
Every result must match the FP64 oracle within 8 k u, and be bit-identical
to the same request served alone."""
import time

import numpy as np
import pytest

from helpers import bound, to_dev
import oracle
from paper_2504_13821_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def build(server, dev, seed):
    rng = np.random.default_rng(seed)
    facs = []
    for i, (k, dtype) in enumerate([(90, np.float32), (300, np.float64), (700, np.float32),
                                    (1500, np.float32), (600, np.float64)]):
        uplo, trans, diag = rng.choice(["L", "U"]), rng.choice(["N", "T"]), rng.choice(["N", "U"])
        A = inputs.tri_matrix(k, uplo, seed=seed + i, dtype=dtype, poison_diag=(diag == "U"))
        fid = server.register(to_dev(A, dev), uplo, trans, diag) if server else None
        facs.append((fid, A, uplo, trans, diag, dtype))
    reqs = []
    for r in range(80):
        fi = int(rng.integers(len(facs)))
        fid, A, uplo, trans, diag, dtype = facs[fi]
        k = A.shape[0]
        op = "S" if rng.random() < 0.7 else "M"
        side = str(rng.choice(["L", "R"]))
        nrhs = int(rng.integers(1, 200))
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        B = inputs.rhs(m, n, seed=seed * 1000 + r, dtype=dtype)
        reqs.append((fi, op, side, float(rng.choice([1.5, -1.0])), B))
    return facs, reqs


def serve(reqs, facs, dev, spread_s):
    from paper_2504_13821_gb300 import serving
    srv = serving.Server(0, streams=3, budget_bytes=1 << 30, max_inflight=64)
    ids = [srv.register(to_dev(A, dev), u, t, d) for (_, A, u, t, d, _) in facs]
    t0 = time.perf_counter()
    out = []
    for i, (fi, op, side, alpha, B) in enumerate(reqs):
        Bt = to_dev(B, dev)
        req = serving.Request(i, ids[fi], op, side, alpha, Bt, t0 + spread_s * i / len(reqs))
        srv.submit(req)
        out.append(req)
    srv.drain()
    torch.cuda.synchronize()
    stats = serving.latency_stats(srv.completed)
    srv.close()
    return [r.B.cpu().numpy() for r in out], stats


def test_serving_mix_matches_oracle_and_solo():
    dev = torch.device("cuda", 0)
    facs, reqs = build(None, dev, seed=3)
    mixed, stats = serve(reqs, facs, dev, spread_s=0.05)
    assert stats["count"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    for i, (fi, op, side, alpha, B) in enumerate(reqs):
        _, A, uplo, trans, diag, dtype = facs[fi]
        X = np.asfortranarray(mixed[i])
        if op == "S":
            e = oracle.trsm_backward_error(side, uplo, trans, diag, alpha, A, X, B)["eta"]
        else:
            e = oracle.trmm_error(side, uplo, trans, diag, alpha, A, X,
                                  oracle.trmm(side, uplo, trans, diag, alpha, A, B), B)
        assert e <= bound(A.shape[0], dtype), (i, op, side, A.shape[0], e)
    for i in range(0, len(reqs), 9):                   # a sample served alone
        solo, _ = serve([reqs[i]], facs, dev, spread_s=0.0)
        assert np.array_equal(solo[0], mixed[i]), f"request {i} differs alone vs in the mix"
