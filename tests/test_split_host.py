"""The BF16 slice arithmetic of the tensor-core FP32 path, emulated on the
host (no GPU): an FP32 value x is carried as x0 = bf16(x), x1 = bf16(x -
x0), x2 = bf16(x - x0 - x1) (round to nearest even, each difference exact
in FP32); a product takes the slice products above FP32's rounding level:
1 term (x0 y0), 3 terms (+ x0 y1 + x1 y0) or 6 terms (+ x0 y2 + x1 y1 +
x2 y0). Pinned here: the three slices reconstruct x exactly, and each
form's product error lies within its stated level (2^-8, 2^-16, a few units
of 2^-24), against the exact product in FP64."""
import numpy as np
import pytest


def bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def slices(x):
    x = np.asarray(x, dtype=np.float32)
    s0 = bf16(x)
    r = (x - s0).astype(np.float32)
    s1 = bf16(r)
    s2 = bf16((r - s1).astype(np.float32))
    return s0, s1, s2


def sample(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-60, 60, n)
    sign = rng.choice([-1.0, 1.0], n)
    return (sign * mant * 2.0 ** expo).astype(np.float32)


def test_rounding_is_nearest_even():
    # values exactly between two BF16 neighbours go to the even one
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)                   # BF16 spacing in [1, 2)
    half = np.float32(2.0 ** -8)
    assert bf16(one + half) == one                # tie: 1.0 is even
    assert bf16(one + ulp + half) == one + 2 * ulp  # tie: rounds up to even
    assert bf16(np.float32(1.0 + 2.0 ** -9)) == one
    assert bf16(np.float32(-3.0)) == np.float32(-3.0)


def test_three_slices_reconstruct_fp32_exactly():
    x = sample(200000, 1)
    s0, s1, s2 = slices(x)
    rec = s0.astype(np.float64) + s1.astype(np.float64) + s2.astype(np.float64)
    assert np.array_equal(rec, x.astype(np.float64))
    # each remainder was exact in FP32 and each slice keeps 8 significant bits
    assert np.all(np.abs(s1.astype(np.float64)) <= 2.0 ** -8 * np.abs(x.astype(np.float64)))
    assert np.all(np.abs(s2.astype(np.float64)) <= 2.0 ** -16 * np.abs(x.astype(np.float64)))


@pytest.mark.parametrize("terms,level", [(1, 2.0 ** -7), (3, 2.0 ** -15), (6, 2.0 ** -23)])
def test_product_forms_within_their_level(terms, level):
    x, y = sample(200000, 2), sample(200000, 3)
    xs = [s.astype(np.float64) for s in slices(x)]
    ys = [s.astype(np.float64) for s in slices(y)]
    pairs = [(0, 0)] + ([(0, 1), (1, 0)] if terms >= 3 else []) + \
            ([(0, 2), (1, 1), (2, 0)] if terms == 6 else [])
    approx = sum(xs[i] * ys[j] for i, j in pairs)   # each product exact in FP64
    exact = x.astype(np.float64) * y.astype(np.float64)
    rel = np.abs(approx - exact) / np.abs(exact)
    assert rel.max() <= level
