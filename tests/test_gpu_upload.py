"""Host-to-device upload of the referenced triangle (trx_copy_triangle_h2d):
the triangle arrives exactly, the other triangle of the device array is left
alone outside the 256 x 256 diagonal blocks the copy moves whole, and a
solve on the uploaded factor matches the oracle."""
import numpy as np
import pytest

from helpers import bound, to_dev
import oracle
from paper_2504_13821_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _block_mask(k, blk=256):
    """True where (i, j) share a 256 x 256 diagonal block."""
    idx = np.arange(k) // blk
    return idx[:, None] == idx[None, :]


@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("k", [1, 255, 256, 257, 700])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_triangle_arrives_other_left(uplo, k, dtype):
    import paper_2504_13821_gb300 as trx
    rng = np.random.default_rng(k)
    ldh, ldd = k + 3, k + 5
    host_full = np.asfortranarray(rng.standard_normal((ldh, k)).astype(dtype))
    A_host = torch.from_numpy(host_full).pin_memory()[:k]
    dev_full = torch.full((k, ldd), float("nan"), dtype=A_host.dtype, device="cuda").t()
    A_dev = dev_full[:k]
    if k > 1:   # (a single column's leading dimension is not carried by its strides)
        assert A_host.stride() == (1, ldh) and A_dev.stride() == (1, ldd)
    trx.copy_triangle_h2d(uplo, A_host, A_dev)
    torch.cuda.synchronize()
    got = A_dev.cpu().numpy()
    want = host_full[:k]
    tri = np.tril(np.ones((k, k), bool)) if uplo == "L" else np.triu(np.ones((k, k), bool))
    assert np.array_equal(got[tri], want[tri])
    other = ~tri
    inside = other & _block_mask(k)
    outside = other & ~_block_mask(k)
    assert np.array_equal(got[inside], want[inside])
    assert np.isnan(got[outside]).all()
    # rows below k in the device storage are never written
    assert torch.isnan(dev_full[k:]).all()


def test_uploaded_factor_solves():
    import paper_2504_13821_gb300 as trx
    k, n = 1000, 64
    A, B = inputs.problem("L", "U", k, n, seed=5, dtype=np.float32)
    A_host = torch.from_numpy(A).pin_memory()
    A_dev = torch.full((k, k), float("nan"), device="cuda").t()
    trx.copy_triangle_h2d("U", A_host, A_dev)
    Bt = to_dev(B, "cuda:0")
    trx.trsm("L", "U", "N", "N", 1.5, A_dev, Bt)
    torch.cuda.synchronize()
    X = np.asfortranarray(Bt.cpu().numpy())
    eta = oracle.trsm_backward_error("L", "U", "N", "N", 1.5, A.astype(np.float64),
                                     X.astype(np.float64), B.astype(np.float64))["eta"]
    assert eta <= bound(k, np.float32)
