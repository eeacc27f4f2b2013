"""Error bound of the split-TF32 product used by the tensor-core gather (CPU).

The 2-D FP32 interpolation forms each weight x field product on the tensor
cores from TF32 operands: x = hi + lo with hi = x cut to TF32 (its 13 low
mantissa bits cleared) and lo = x - hi exact in FP32, of which the tensor
core reads only the TF32 part; the product is hi_x hi_y + hi_x lo_y + lo_x hi_y.
Its error is below 3 * 2^-20 of |x y| (the dropped lo_x lo_y and the two cuts
of lo), which keeps a w^2-term gather well inside the 1e-5 bar of the FP32
path.  This models the split on FP32 bit patterns with numpy and checks the
bound over operands spanning many binades; the products and the
three-term sum are taken exactly in FP64 (each product of two 11-bit
significands is exact in FP32, too).
"""
import numpy as np

MASK = np.uint32(0xFFFFE000)


def cut_tf32(v):
    return (np.asarray(v, dtype=np.float32).view(np.uint32) & MASK).view(np.float32)


def split(v):
    v = np.asarray(v, dtype=np.float32)
    hi = cut_tf32(v)
    lo = (v - hi).astype(np.float32)            # exact in FP32
    return hi, cut_tf32(lo)                     # the tensor core reads lo's TF32 part


def test_split_product_error_is_below_3_times_2_to_the_minus_20():
    rng = np.random.default_rng(20)
    n = 400_000
    x = (rng.random(n) + 0.5) * np.exp2(rng.integers(-40, 40, n))
    y = (rng.standard_normal(n)) * np.exp2(rng.integers(-40, 40, n))
    x = x.astype(np.float32)
    y = y.astype(np.float32)
    hx, lx = split(x)
    hy, ly = split(y)
    # the remainder before its cut is exact and small
    lo_exact = x.astype(np.float64) - hx.astype(np.float64)
    assert np.all(np.abs(lo_exact) < np.exp2(-10.0) * np.abs(x.astype(np.float64)))
    got = (hx.astype(np.float64) * hy + hx.astype(np.float64) * ly
           + lx.astype(np.float64) * hy)
    ref = x.astype(np.float64) * y.astype(np.float64)
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() < 3 * np.exp2(-20.0)
    # and a plain TF32 product (no split) is about 2^-10 off: the split matters
    plain = hx.astype(np.float64) * hy.astype(np.float64)
    assert (np.abs(plain - ref) / np.abs(ref)).max() > np.exp2(-12.0)


def test_split_dot_product_error_against_the_sum_of_magnitudes():
    # a 7 x 7 window of positive weights against fields of both signs: the
    # error of the split sum relative to sum |w f| stays below 3 * 2^-20
    rng = np.random.default_rng(21)
    w = rng.random((20_000, 49)).astype(np.float32) * np.float32(0.3)
    f = rng.standard_normal((20_000, 49)).astype(np.float32)
    hw, lw = split(w)
    hf, lf = split(f)
    got = np.sum(hw.astype(np.float64) * hf + hw.astype(np.float64) * lf
                 + lw.astype(np.float64) * hf, axis=1)
    ref = np.sum(w.astype(np.float64) * f.astype(np.float64), axis=1)
    mag = np.sum(np.abs(w.astype(np.float64) * f.astype(np.float64)), axis=1)
    assert (np.abs(got - ref) / mag).max() < 3 * np.exp2(-20.0)
