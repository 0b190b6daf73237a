"""Batched uneven problems (one persistent launch): every problem of a mixed
batch (TRSM and TRMM, all side/uplo/trans/diag, orders log-uniform 16..512,
1..64 right-hand sides, FP32 and FP64) against the FP64 oracle with the
same 8 k u criteria as the single calls."""
import numpy as np
import pytest

from helpers import bound, to_dev
import oracle
from paper_2504_13821_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_batch(count, dtype, seed, dev):
    rng = np.random.default_rng(seed)
    probs, host = [], []
    for i in range(count):
        k = int(round(np.exp(rng.uniform(np.log(16), np.log(512)))))
        nrhs = int(rng.integers(1, 65))
        side, uplo = rng.choice(["L", "R"]), rng.choice(["L", "U"])
        trans, diag = rng.choice(["N", "T"]), rng.choice(["N", "U"])
        op = "S" if rng.random() < 0.7 else "M"
        alpha = float(rng.choice([1.5, -0.5, 1.0]))
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        A, B = inputs.problem(side, uplo, m, n, seed=seed * 100000 + i, dtype=dtype,
                              poison_diag=(diag == "U"))
        At, Bt = to_dev(A, dev), to_dev(B, dev)
        probs.append((op, side, uplo, trans, diag, alpha, At, Bt))
        host.append((A, B))
    return probs, host


def check(probs, host, dtype):
    worst = 0.0
    for (op, side, uplo, trans, diag, alpha, At, Bt), (A, B) in zip(probs, host):
        X = np.asfortranarray(Bt.cpu().numpy())
        k = A.shape[0]
        if op == "S":
            e = oracle.trsm_backward_error(side, uplo, trans, diag, alpha, A, X, B)["eta"]
        else:
            ref = oracle.trmm(side, uplo, trans, diag, alpha, A, B)
            e = oracle.trmm_error(side, uplo, trans, diag, alpha, A, X, ref, B)
        assert np.isfinite(e) and e <= bound(k, dtype), (op, side, uplo, trans, diag, k, e)
        worst = max(worst, e / bound(k, dtype))
    return worst


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_batched_mixed_against_oracle(dtype):
    import paper_2504_13821_gb300 as trx
    dev = torch.device("cuda", 0)
    probs, host = make_batch(300, dtype, seed=7, dev=dev)
    trx.batched(probs)
    torch.cuda.synchronize()
    check(probs, host, dtype)


def test_batched_graph_replay_and_autotune():
    import paper_2504_13821_gb300 as trx
    dev = torch.device("cuda", 0)
    h = trx.Handle(0)
    probs, host = make_batch(120, np.float32, seed=8, dev=dev)
    table = trx.batched_autotune(probs, handle=h)     # clobbers B
    assert [b["kmax"] for b in table["buckets"]] == [k for k in (64, 128, 256, 512)
                                                     for _ in range(3)]
    assert [b["nrhs_max"] for b in table["buckets"]] == [8, 24, 64] * 4
    assert all(b["sb"] in (4, 8, 16) for b in table["buckets"])
    assert sum(b["problems"] for b in table["buckets"]) == len(probs)
    # the table persists and restores (another handle, same results bitwise)
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        path = d + "/tuning.json"
        _binding_save = trx._binding.save_tuning
        _binding_save(path, handle=h)
        h2 = trx.Handle(0)
        trx._binding.load_tuning(path, handle=h2)
        for (_, _, _, _, _, _, _, Bt), (_, B) in zip(probs, host):
            Bt.copy_(torch.from_numpy(np.asfortranarray(B)))
        trx.batched(probs, handle=h2)
        torch.cuda.synchronize()
        via_loaded = [p[7].cpu().clone() for p in probs]
        h2.close()
    outs = []
    for _ in range(2):                               # second call replays the cached graph
        for (_, _, _, _, _, _, _, Bt), (_, B) in zip(probs, host):
            Bt.copy_(torch.from_numpy(np.asfortranarray(B)))
        trx.batched(probs, handle=h)
        torch.cuda.synchronize()
        check(probs, host, np.float32)
        outs.append([p[7].cpu().clone() for p in probs])
    assert all(torch.equal(a, b) for a, b in zip(*outs))
    assert all(torch.equal(a, b) for a, b in zip(outs[0], via_loaded))
    h.close()


def test_batched_rejects_large_order_and_alpha_zero_reads_no_a():
    import paper_2504_13821_gb300 as trx
    dev = torch.device("cuda", 0)
    A = trx.to_colmajor(torch.eye(600, device=dev))
    B = trx.to_colmajor(torch.ones(600, 3, device=dev))
    with pytest.raises(trx.TrxError):
        trx.batched([("S", "L", "L", "N", "N", 1.0, A, B)])
    An = trx.to_colmajor(torch.full((40, 40), float("nan"), device=dev))
    Bz = trx.to_colmajor(torch.ones(40, 5, device=dev))
    trx.batched([("S", "L", "L", "N", "N", 0.0, An, Bz)])
    torch.cuda.synchronize()
    assert torch.count_nonzero(Bz).item() == 0


def test_prepared_batch_equals_one_shot_and_reruns():
    """trx_batch_create / trx_batch_run: the same results as trx_batched,
    bitwise, on every run (contents of B refreshed in place between runs)."""
    import paper_2504_13821_gb300 as trx
    dev = torch.device("cuda", 0)
    probs, host = make_batch(200, np.float32, seed=11, dev=dev)
    originals = [p[7].clone() for p in probs]
    one_shot = [(o, s, u, t, d, a, A, B.clone()) for (o, s, u, t, d, a, A, B) in probs]
    trx.batched(one_shot)
    h = trx.Handle(0)
    batch = trx.Batch(probs, handle=h)
    for _ in range(2):
        for p, b0 in zip(probs, originals):
            p[7].copy_(b0)
        batch.run(handle=h)
        torch.cuda.synchronize()
        for p, q in zip(probs, one_shot):
            assert torch.equal(p[7], q[7])
    check(probs, host, np.float32)
    batch.close()
    h.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_typed_batched_entry_points_equal_mixed_call(dtype):
    """trx_{s,d}{trsm,trmm}_batched on a one-operation batch give the same
    bits as trx_batched on the same problems."""
    import paper_2504_13821_gb300 as trx
    from paper_2504_13821_gb300 import _binding
    lib = _binding.load_library()
    dev = torch.device("cuda", 0)
    h = trx.Handle(dev)
    pre = "trx_s" if dtype == np.float32 else "trx_d"
    for op, name in (("S", pre + "trsm_batched"), ("M", pre + "trmm_batched")):
        probs, _ = make_batch(60, dtype, seed=11, dev=dev)
        probs = [(op,) + p[1:] for p in probs]
        twin = [p[:7] + (p[7].clone(),) for p in probs]
        arr, elem = _binding._problem_array(probs)
        s = torch.cuda.current_stream(dev).cuda_stream
        assert getattr(lib, name)(h.ptr, len(probs), arr, s) == 0
        trx.batched(twin, handle=h)
        torch.cuda.synchronize()
        for p, q in zip(probs, twin):
            assert torch.equal(p[7], q[7])
    h.close()
