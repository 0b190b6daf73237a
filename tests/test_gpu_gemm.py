"""The GEMM update on its own (Section 3.1's off-diagonal step),
C := beta C + gamma A Y, tensor-core and CUDA-core engines, against an FP64
product on tile-edge shapes (ragged M, N; K multiples of the 64 K tile)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 64), (127, 129, 64), (128, 256, 64), (129, 257, 128), (300, 70, 192),
          (256, 512, 1024), (1000, 513, 2048)]


def colmajor(x):
    return x.t().contiguous().t()


@pytest.mark.parametrize("engine", [2, 1])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gemm_update_against_fp64(M, N, K, engine):
    import paper_2504_13821_gb300 as trx
    rng = np.random.default_rng(M * 7 + N * 13 + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    Y = rng.standard_normal((K, N)).astype(np.float32)
    C = rng.standard_normal((M, N)).astype(np.float32)
    beta, gamma = 0.75, -1.25
    dev = torch.device("cuda", 0)
    At, Yt, Ct = (colmajor(torch.from_numpy(x).to(dev)) for x in (A, Y, C))
    trx.gemm_update(beta, gamma, At, Yt, Ct, engine=engine)
    torch.cuda.synchronize()
    got = Ct.cpu().numpy().astype(np.float64)
    ref = beta * C.astype(np.float64) + gamma * (A.astype(np.float64) @ Y.astype(np.float64))
    mag = np.abs(beta * C.astype(np.float64)) + abs(gamma) * (np.abs(A).astype(np.float64) @
                                                              np.abs(Y).astype(np.float64))
    # split-BF16 products: about 3 * 2^-17 each; FP32 accumulation over K
    tol = (2.0 ** -14 + K * 2.0 ** -23) * mag + 2.0 ** -20 * np.abs(ref)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (f"{bad.sum()} of {bad.size} outside tolerance; worst "
                           f"{np.max(np.abs(got - ref) / np.maximum(mag, 1e-30)):.3e}")


def test_gemm_update_is_deterministic():
    import paper_2504_13821_gb300 as trx
    rng = np.random.default_rng(5)
    dev = torch.device("cuda", 0)
    A = colmajor(torch.from_numpy(rng.standard_normal((500, 512)).astype(np.float32)).to(dev))
    Y = colmajor(torch.from_numpy(rng.standard_normal((512, 700)).astype(np.float32)).to(dev))
    C0 = colmajor(torch.from_numpy(rng.standard_normal((500, 700)).astype(np.float32)).to(dev))
    outs = []
    for _ in range(3):
        C = C0.clone(memory_format=torch.preserve_format)
        C = colmajor(C)
        trx.gemm_update(1.0, -1.0, A, Y, C)
        outs.append(C.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
