"""The double-float accumulation of the FP64-grade products of mixed-precision
solves (block_gemm_df), emulated step by step in NumPy float32 and checked
against exact rational sums: the error bound that the design relies on
(~1e-14 relative to sum |a b| per output, for k up to a few hundred)."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _fma32(a, b, c):
    # a*b + c rounded once to FP32: the product of two FP32 values is exact in
    # FP64, and so is its sum with an FP32 c at these magnitudes
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _df_dot(a, b):
    """sum_k a_k b_k as the kernel forms one output: b split into hi + lo,
    exact a*b_hi by FMA, TwoSum into (hi, lo), renormalised every 16 terms."""
    hi, lo = f32(0), f32(0)
    for k, (x, y) in enumerate(zip(a, b)):
        bh = f32(y)
        bl = f32(y - np.float64(bh))
        p = f32(x * bh)
        e = _fma32(x, bh, -p)
        e = _fma32(x, bl, e)
        s = f32(hi + p)
        bb = f32(s - hi)
        err = f32(f32(hi - f32(s - bb)) + f32(p - bb))
        hi = s
        lo = f32(lo + f32(err + e))
        if k % 16 == 15:
            s = f32(hi + lo)
            lo = f32(lo - f32(s - hi))
            hi = s
    return np.float64(hi) + np.float64(lo)


def test_double_float_products_reach_fp64_grade_accuracy():
    rng = np.random.default_rng(7)
    worst = 0.0
    for k in (16, 152, 348):
        for _ in range(20):
            a = (rng.standard_normal(k) * 0.3).astype(f32)          # exact FP32 rows
            b = rng.standard_normal(k) * 0.5                        # FP64 matrix entries
            exact = float(sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)))
            scale = float(np.sum(np.abs(a.astype(np.float64) * b)))
            worst = max(worst, abs(_df_dot(a, b) - exact) / scale)
    assert worst < 2e-14
    # plain FP32 accumulation misses by orders of magnitude more
    a = (rng.standard_normal(152) * 0.3).astype(f32)
    b = rng.standard_normal(152) * 0.5
    exact = float(sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)))
    plain = f32(0)
    for x, y in zip(a, b):
        plain = _fma32(x, f32(y), plain)
    assert abs(float(plain) - exact) / float(np.sum(np.abs(a * b))) > 1e-9
