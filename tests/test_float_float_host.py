"""The float-float accumulation of the refined TRSM's residual, emulated on
the host in IEEE FP32 step by step (no GPU), against exact sums.

Per term a * x with a FP32 and x = xh + xl (two floats): p = fl(a xh) and
e = a xh - p exactly (one FMA), p enters hi by Knuth's two-sum, the
two-sum's error, e and a xl enter lo; every 32 terms lo moves into a second
pair (mid, lo2) by another two-sum; the result is hi + (mid + (lo + lo2))
in FP64. Measured here: 2^-46 of sum |a x| per output or better on random
rows, 2^-44 or better with cancelling terms, magnitudes spread over 2^80 and
a dominant term; one FP32 dot product gives about 2^-24.
"""
import math

import numpy as np

F = np.float32


def two_sum(s, b):
    """s + b = t + err exactly (FP32 arrays), Knuth."""
    t = F(s + b)
    bp = F(t - s)
    err = F(F(s - F(t - bp)) + F(b - bp))
    return t, err


def emulate(a, xh, xl, fold=32):
    """Rows of the kernel's accumulation; a, xh, xl: (terms, rows) FP32."""
    rows = a.shape[1]
    hi = np.zeros(rows, F)
    lo = np.zeros(rows, F)
    mid = np.zeros(rows, F)
    lo2 = np.zeros(rows, F)
    for t in range(a.shape[0]):
        ax = a[t].astype(np.float64) * xh[t].astype(np.float64)     # exact (24 x 24 bits)
        p = ax.astype(F)
        e = (ax - p.astype(np.float64)).astype(F)                    # exact: the FMA's result
        hi, err = two_sum(hi, p)
        s = F(lo + F(err + e))
        # fma(a, xl, s): a xl is exact in FP64, one rounding to FP32 after
        lo = (a[t].astype(np.float64) * xl[t].astype(np.float64) + s.astype(np.float64)).astype(F)
        if (t + 1) % fold == 0:
            mid, err2 = two_sum(mid, lo)
            lo2 = F(lo2 + err2)
            lo = np.zeros(rows, F)
    return hi.astype(np.float64) + (mid.astype(np.float64) +
                                    (lo.astype(np.float64) + lo2.astype(np.float64)))


def exact(a, xh, xl):
    """Exact sums of a xh + a xl per row (every product exact in FP64)."""
    out = []
    for r in range(a.shape[1]):
        terms = np.concatenate([a[:, r].astype(np.float64) * xh[:, r].astype(np.float64),
                                a[:, r].astype(np.float64) * xl[:, r].astype(np.float64)])
        out.append(math.fsum(terms))
    return np.array(out)


def split(x):
    xh = x.astype(F)
    xl = (x - xh.astype(np.float64)).astype(F)
    return xh, xl


def check(a, x, bound_bits):
    xh, xl = split(x)
    got = emulate(a, xh, xl)
    ref = exact(a, xh, xl)
    scale = np.sum(np.abs(a.astype(np.float64) * x), axis=0)
    rel = np.abs(got - ref) / scale
    assert np.all(rel <= 2.0 ** -bound_bits), (rel.max(), np.log2(rel.max()))
    return rel.max()


def test_random_rows_keep_46_bits():
    rng = np.random.default_rng(1)
    K, R = 4096, 48
    a = rng.uniform(-1, 1, (K, R)).astype(F)
    x = rng.standard_normal((K, R))
    worst = check(a, x, 46)
    # one FP32 dot product of the same data is some 20 bits worse
    naive = np.zeros(R, F)
    for t in range(K):
        naive = F(naive + F(a[t] * split(x)[0][t]))
    ref = exact(a, *split(x))
    scale = np.sum(np.abs(a.astype(np.float64) * x), axis=0)
    assert np.max(np.abs(naive - ref) / scale) > 2.0 ** 20 * worst


def test_cancelling_and_spread_magnitudes():
    """Adversarial rows: terms that cancel to a tiny sum, magnitudes spread
    over 2^-20 .. 2^20 in both factors, and a dominant first term that keeps
    the running sum large (measured 2^-44.6)."""
    rng = np.random.default_rng(2)
    K, R = 2048, 24
    a = (rng.uniform(-1, 1, (K, R)) * 2.0 ** rng.integers(-20, 21, (K, R))).astype(F)
    x = rng.standard_normal((K, R)) * 2.0 ** rng.integers(-20, 21, (K, R))
    x[K // 2:] = -x[:K // 2] * (a[:K // 2] / np.where(a[K // 2:] == 0, 1, a[K // 2:]))
    a[0] = F(2.0 ** 30)
    check(a, x, 44)


def test_split_of_x_keeps_48_bits():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(10000) * 2.0 ** rng.integers(-30, 31, 10000)
    xh, xl = split(x)
    rel = np.abs(x - (xh.astype(np.float64) + xl.astype(np.float64))) / np.abs(x)
    assert rel.max() <= 2.0 ** -47


def emulate_pair(ah, al, xh, xl, fold=32):
    """The FP64-data mode: a = ah + al as well. Per term p = fl(ah xh) and
    e = ah xh - p exactly; p two-summed into hi; err + e, then ah xl and
    al xh (two FMAs, in that order) into lo; folds as above."""
    rows = ah.shape[1]
    hi = np.zeros(rows, F)
    lo = np.zeros(rows, F)
    mid = np.zeros(rows, F)
    lo2 = np.zeros(rows, F)
    d = np.float64
    for t in range(ah.shape[0]):
        ax = ah[t].astype(d) * xh[t].astype(d)
        p = ax.astype(F)
        e = (ax - p.astype(d)).astype(F)
        hi, err = two_sum(hi, p)
        s = F(lo + F(err + e))
        s = (ah[t].astype(d) * xl[t].astype(d) + s.astype(d)).astype(F)
        lo = (al[t].astype(d) * xh[t].astype(d) + s.astype(d)).astype(F)
        if (t + 1) % fold == 0:
            mid, err2 = two_sum(mid, lo)
            lo2 = F(lo2 + err2)
            lo = np.zeros(rows, F)
    return hi.astype(d) + (mid.astype(d) + (lo.astype(d) + lo2.astype(d)))


def test_pair_mode_fp64_data_keeps_44_bits():
    """A and X both FP64 data, each carried as two floats: the residual of
    an FP64 system on the FP32 pipes. Against the exact sum of the FP64
    products a x (math.fsum of products split exactly), the error stays
    below 2^-44 of sum |a x| on random and on cancelling rows (the dropped
    al xl term alone is about 2^-48)."""
    rng = np.random.default_rng(4)
    K, R = 2048, 32
    a = rng.uniform(-1, 1, (K, R)) * 2.0 ** rng.integers(-10, 11, (K, R))
    x = rng.standard_normal((K, R))
    x[K // 2:] = -x[:K // 2] * a[:K // 2] / a[K // 2:]    # pairs that cancel
    ah, al = split(a)
    xh, xl = split(x)
    got = emulate_pair(ah, al, xh, xl)
    ref = []
    for r in range(R):
        terms = []
        for t in range(K):
            # a x exactly as a sum of FP64 pieces: (ah + al)(xh + xl)
            for u in (ah[t, r], al[t, r]):
                for v in (xh[t, r], xl[t, r]):
                    terms.append(float(u) * float(v))      # exact: 24 x 24 bits
        ref.append(math.fsum(terms))
    ref = np.array(ref)
    scale = np.sum(np.abs(a * x), axis=0)
    rel = np.abs(got - ref) / scale
    assert rel.max() <= 2.0 ** -44, np.log2(rel.max())
    # the same data with A rounded to one float (mode 0) is ~2^-24 off
    coarse = emulate(ah, xh, xl)
    assert np.max(np.abs(coarse - ref) / scale) > 2.0 ** 16 * rel.max()
