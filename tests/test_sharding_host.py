"""Multi-rank host logic, no GPU: the right-hand-side partition and the
bench's rank reductions, as two gloo ranks on CPU.

Right-hand sides are independent, so ranks that each solve their panel (with
the FP64 oracle standing in for the device here) must reproduce the
single-rank result exactly once the panels are gathered.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2504_13821_gb300 import inputs
from paper_2504_13821_gb300.sharding import panel

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1000, 16384])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_panels_cover_once(n, world):
    seen = np.zeros(n, dtype=int)
    prev = 0
    for r in range(world):
        j0, j1 = panel(n, world, r)
        assert j0 == prev and j0 <= j1 <= n          # contiguous, in rank order
        if j1 < n:
            assert (j1 - j0) % 32 == 0
        seen[j0:j1] += 1
        prev = j1
    assert prev == n and np.all(seen == 1)


def test_panel_rejects_bad_arguments():
    for args in [(-1, 2, 0), (10, 0, 0), (10, 2, 2), (10, 2, -1)]:
        with pytest.raises(ValueError):
            panel(*args)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # bench's reductions: max over ranks, barrier
    got = bench.max_over_ranks(float(10 * rank + 1), world)
    bench.barrier(world)
    # each rank solves its column panel (side L) and its row panel (side R)
    out = {}
    for side in ("L", "R"):
        m, n = (70, 301) if side == "L" else (301, 70)
        A, B = inputs.problem(side, "U", m, n, seed=77, dtype=np.float64)
        nr = n if side == "L" else m
        j0, j1 = panel(nr, world, rank)
        Bp = B[:, j0:j1] if side == "L" else B[j0:j1, :]
        X = oracle.trsm(side, "U", "T", "N", 1.5, A, np.asfortranarray(Bp))
        # gather the panels on every rank (padded to the largest panel)
        width = panel(nr, world, 0)[1]
        pad = np.zeros((m, width) if side == "L" else (width, n))
        if side == "L":
            pad[:, :j1 - j0] = X
        else:
            pad[:j1 - j0, :] = X
        parts = [torch.zeros(pad.shape, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(pad))
        pieces = []
        for r in range(world):
            a0, a1 = panel(nr, world, r)
            p = parts[r].numpy()
            pieces.append(p[:, :a1 - a0] if side == "L" else p[:a1 - a0, :])
        out[side] = np.concatenate(pieces, axis=1 if side == "L" else 0)
    # the same partition through the library's own host plan: each rank
    # replays (FP64, on the host) the launch sequence the library would
    # enqueue for its panel of a side-L TRSM and TRMM on the tensor-core
    # path, and the gathered panels match the oracle's single-rank result
    from test_plan_host import replay
    from paper_2504_13821_gb300 import debug_plan
    k, nr = 300, 257
    A, B = inputs.problem("L", "L", k, nr, seed=78, dtype=np.float64)
    M = np.where(np.isnan(A), 0.0, A)
    j0, j1 = panel(nr, world, rank)
    width = panel(nr, world, 0)[1]
    for op in ("S", "M"):
        pad = np.zeros((k, width))
        if j1 > j0:
            steps = debug_plan(op, "L", "L", "N", "N", k, j1 - j0, 4, 0, 2)
            pad[:, :j1 - j0] = replay(op, steps, M, B[:, j0:j1])
        parts = [torch.zeros(pad.shape, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(pad))
        out["plan_" + op] = np.concatenate(
            [parts[r].numpy()[:, :panel(nr, world, r)[1] - panel(nr, world, r)[0]]
             for r in range(world)], axis=1)
    dist.destroy_process_group()
    np.savez(os.path.join(outdir, f"rank{rank}.npz"), maxv=got, L=out["L"], R=out["R"],
             plan_S=out["plan_S"], plan_M=out["plan_M"])


def test_two_gloo_ranks_reproduce_single_rank(tmp_path):
    oracle.build()
    world = 2
    port = _free_port()
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    for rank in range(world):
        d = np.load(tmp_path / f"rank{rank}.npz")
        assert float(d["maxv"]) == 11.0
        for side in ("L", "R"):
            m, n = (70, 301) if side == "L" else (301, 70)
            A, B = inputs.problem(side, "U", m, n, seed=77, dtype=np.float64)
            want = oracle.trsm(side, "U", "T", "N", 1.5, A, B)
            np.testing.assert_array_equal(d[side], want)
        A, B = inputs.problem("L", "L", 300, 257, seed=78, dtype=np.float64)
        for op, fn in (("S", oracle.trsm), ("M", oracle.trmm)):
            want = fn("L", "L", "N", "N", 2.0, A, B)     # the plan dump's alpha
            np.testing.assert_allclose(d["plan_" + op], want, rtol=1e-10,
                                       atol=1e-10 * np.abs(want).max())
