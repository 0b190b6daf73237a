"""Request server (trx_server_*): requests of mixed sizes, element types
and operations arrive while others are on the GPU and are admitted as budget
and slots free up (small ones batched per tick, large ones on parallel
streams).
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


def serve(reqs, facs, dev, spread_s, graphs=True):
    """Submit the requests spread over spread_s seconds, polling the
    server between arrivals, then drain it."""
    from paper_2504_13821_gb300 import serving
    srv = serving.Server(0, streams=3, budget_bytes=1 << 30, max_inflight=64, graphs=graphs)
    ids = [srv.register(to_dev(A, dev), u, t, d) for (_, A, u, t, d, _) in facs]
    t0 = time.perf_counter()
    outs, status = [], {}
    for i, (fi, op, side, alpha, B) in enumerate(reqs):
        Bt = to_dev(B, dev)
        while time.perf_counter() < t0 + spread_s * i / len(reqs):
            status.update(srv.poll())
        rid = srv.submit(ids[fi], op, side, alpha, Bt)
        outs.append((rid, Bt))
    status.update(srv.drain())
    torch.cuda.synchronize()
    srv.close()
    assert sorted(status) == sorted(r for r, _ in outs)
    assert all(v == 0 for v in status.values()), status
    return [Bt.cpu().numpy() for _, Bt in outs]


@pytest.mark.parametrize("graphs", [True, False], ids=["graphs", "direct"])
def test_serving_mix_matches_oracle_and_solo(graphs):
    dev = torch.device("cuda", 0)
    facs, reqs = build(None, dev, seed=3)
    mixed = serve(reqs, facs, dev, spread_s=0.05, graphs=graphs)
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
        solo = serve([reqs[i]], facs, dev, spread_s=0.0, graphs=graphs)
        assert np.array_equal(solo[0], mixed[i]), f"request {i} differs alone vs in the mix"


def test_server_budget_and_release():
    """A budget that fits one request at a time still serves every request
    (one admitted per tick, the oversized one alone), and a released
    factor takes no new requests."""
    from paper_2504_13821_gb300 import serving
    dev = torch.device("cuda", 0)
    A = inputs.tri_matrix(600, "L", seed=8, dtype=np.float32)
    srv = serving.Server(0, streams=2, budget_bytes=600 * 40 * 4, max_inflight=8)
    fid = srv.register(to_dev(A, dev), "L")
    Bs = [to_dev(inputs.rhs(600, n, seed=n, dtype=np.float32), dev) for n in (40, 30, 90)]
    rids = [srv.submit(fid, "S", "L", 1.0, B) for B in Bs]
    srv.release(fid)
    with pytest.raises(Exception):
        srv.submit(fid, "S", "L", 1.0, Bs[0].clone())
    got = dict(srv.drain())
    torch.cuda.synchronize()
    assert sorted(got) == sorted(rids) and not any(got.values())
    assert srv.pending() == (0, 0, 0)
    for n, B in zip((40, 30, 90), Bs):
        B0 = inputs.rhs(600, n, seed=n, dtype=np.float32)
        X = np.asfortranarray(B.cpu().numpy())
        e = oracle.trsm_backward_error("L", "L", "N", "N", 1.0, A, X, B0)["eta"]
        assert e <= bound(600, np.float32)
    srv.close()


@pytest.mark.parametrize("refine_corr,fp64_corr,fp64_trmm", [(2, 3, 0), (1, 2, 1)])
def test_serving_refined_and_mixed_fp64_kinds(refine_corr, fp64_corr, fp64_trmm):
    """Refined FP32 TRSM requests (FP64 result, float-float corrections) and
    FP64 TRSM on the mixed engine (FP32 solve + corrections) in one mix with
    FP32 TRMM and FP64 TRMM (DFMA, or one float-float pass): every refined
    result has the backward error of an FP64 solve (8 k 2^-53 against the
    oracle), every FP64 TRSM too, every TRMM is inside 8 k u, and each
    result is bit-identical to the same request served alone; with two /
    three corrections and DFMA TRMM, and with the one / two corrections and
    float-float TRMM the serving benchmark uses."""
    from paper_2504_13821_gb300 import serving
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(41)
    facs = []
    for i, (k, dtype) in enumerate([(120, np.float32), (700, np.float32), (400, np.float64),
                                    (1100, np.float64)]):
        uplo, trans = str(rng.choice(["L", "U"])), str(rng.choice(["N", "T"]))
        A = inputs.tri_matrix(k, uplo, seed=500 + i, dtype=dtype)
        facs.append((A, uplo, trans, dtype))
    reqs = []
    for r in range(40):
        fi = int(rng.integers(len(facs)))
        A, uplo, trans, dtype = facs[fi]
        k = A.shape[0]
        op = "S" if rng.random() < 0.7 else "M"
        side = str(rng.choice(["L", "R"]))
        nrhs = int(rng.integers(1, 150))
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        reqs.append((fi, op, side, inputs.rhs(m, n, seed=9000 + r, dtype=dtype)))

    def run(sel, spread):
        srv = serving.Server(0, streams=3, budget_bytes=1 << 30, max_inflight=64,
                             refine_corrections=refine_corr, fp64_corrections=fp64_corr,
                             fp64_trmm=fp64_trmm)
        ids = [srv.register(to_dev(A, dev), u, t, "N") for (A, u, t, _) in facs]
        outs, status = [], {}
        t0 = time.perf_counter()
        for j, i in enumerate(sel):
            fi, op, side, B = reqs[i]
            Bt = to_dev(B, dev)
            while time.perf_counter() < t0 + spread * j / len(sel):
                status.update(srv.poll())
            if op == "S" and facs[fi][3] == np.float32:
                X = torch.empty(B.shape[1], B.shape[0], device=dev, dtype=torch.float64).t()
                rid = srv.submit_refined(ids[fi], side, 1.5, Bt, X)
                outs.append((rid, X))
            else:
                rid = srv.submit(ids[fi], op, side, 1.5, Bt)
                outs.append((rid, Bt))
        status.update(srv.drain())
        torch.cuda.synchronize()
        srv.close()
        assert sorted(status) == sorted(r for r, _ in outs) and not any(status.values()), status
        return [o.cpu().numpy() for _, o in outs]

    mixed = run(range(len(reqs)), 0.05)
    for i, (fi, op, side, B) in enumerate(reqs):
        A, uplo, trans, dtype = facs[fi]
        k = A.shape[0]
        X = np.asfortranarray(mixed[i].astype(np.float64))
        A64, B64 = A.astype(np.float64), B.astype(np.float64)
        if op == "S":
            e = oracle.trsm_backward_error(side, uplo, trans, "N", 1.5, A64, X, B64)["eta"]
            assert e <= 8 * k * 2.0 ** -53, (i, dtype, k, e)
        else:
            e = oracle.trmm_error(side, uplo, trans, "N", 1.5, A64, X,
                                  oracle.trmm(side, uplo, trans, "N", 1.5, A64, B64), B64)
            assert e <= bound(k, dtype), (i, dtype, k, e)
    for i in range(0, len(reqs), 7):
        solo = run([i], 0.0)
        assert np.array_equal(solo[0], mixed[i]), f"request {i} differs alone vs in the mix"
