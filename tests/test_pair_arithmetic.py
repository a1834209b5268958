"""The FP32-pair arithmetic of the Krylov operator, checked on the host (no GPU).

The CG operator products of the FP32-cycle solve are formed from float pairs: a value
a = hi + lo with hi = fl32(a), lo = fl32(a - hi); a product a x is hi_a hi_x taken
exactly (its rounded value p plus the error fma(hi_a, hi_x, -p)) plus the cross terms
hi_a lo_x + lo_a hi_x, and lo_a lo_x is dropped; the rounded products are summed with
Knuth's TwoSum and every error term goes to a second float.  This restates those steps
in numpy float32 (an FMA is emulated through float64, where a product of two floats is
exact) and checks the claim the kernels rely on: a row sum S + s lies within a small
multiple of 2^-48 of sum |a_j x_j| from the exact sum (computed in rationals), for
random rows, for rows whose sum cancels to far below its terms, and for values far
from 1 -- about 2^24 times closer than plain float32 summation.
"""
from fractions import Fraction

import numpy as np

F = np.float32


def split(v):
    hi = F(v)
    return hi, F(v - float(hi))


def fma32(a, b, c):
    # float32 FMA: the product of two floats is exact in float64, so only the sum rounds
    # (then to float32); the double rounding this leaves is far below the bound tested
    return F(float(a) * float(b) + float(c))


def two_sum(a, b):
    t = F(a + b)
    bp = F(t - a)
    return t, F(F(a - F(t - bp)) + F(b - bp))


def pair_row_sum(avals, xvals):
    S, s = F(0), F(0)
    for a, x in zip(avals, xvals):
        ah, al = split(a)
        xh, xl = split(x)
        p = F(ah * xh)
        e = fma32(ah, xh, -p)
        e = fma32(ah, xl, e)
        e = fma32(al, xh, e)
        S, err = two_sum(S, p)
        s = F(s + F(err + e))
    return float(S) + float(s)


def exact_row_sum(avals, xvals):
    return float(sum(Fraction(a) * Fraction(x) for a, x in zip(avals, xvals)))


def test_pair_row_sum_is_accurate_to_2_pow_minus_48():
    rng = np.random.default_rng(0)
    worst = 0.0
    for trial in range(300):
        m = int(rng.integers(9, 120))         # 3 x (3..40 blocks) terms of a row
        scale = 10.0 ** rng.uniform(-25, 25)
        a = rng.standard_normal(m) * 10.0 ** rng.uniform(-3, 1)
        x = rng.standard_normal(m) * scale
        if trial % 3 == 0:                    # a row sum that cancels: append its negative
            a = np.concatenate([a, [-1.0]])
            x = np.concatenate([x, [float(np.dot(a[:-1], x))]])
        got = pair_row_sum(a, x)
        want = exact_row_sum(a, x)
        bound = float(np.sum(np.abs(a * x)))
        worst = max(worst, abs(got - want) / bound)
    assert worst <= 8 * 2.0 ** -48, worst


def test_plain_float32_sum_is_far_worse():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(81)
    x = rng.standard_normal(81)
    bound = float(np.sum(np.abs(a * x)))
    want = exact_row_sum(a, x)
    f32 = float(np.sum(a.astype(F) * x.astype(F), dtype=F))
    pair = pair_row_sum(a, x)
    assert abs(pair - want) * 2.0 ** 20 <= abs(f32 - want) + 2.0 ** -70 * bound


def _split_error(v):
    hi, lo = split(v)
    return abs((Fraction(float(hi)) + Fraction(float(lo))) - Fraction(v)) / abs(Fraction(v))


def test_split_is_exact_to_2_pow_minus_48_in_its_range():
    """hi + lo carries v to 2^-48 while lo is a normal float or exact: for |v| from
    about 2^-102 (2e-31; below, lo's last bits fall under FP32's subnormal spacing
    2^-149) up to FP32's largest finite value."""
    rng = np.random.default_rng(2)
    mags = 10.0 ** rng.uniform(-30, 38, 1000)        # |v| from 1e-30 to 1e38
    for v in mags * rng.choice([-1.0, 1.0], 1000):
        assert _split_error(v) <= Fraction(2) ** -48
    assert _split_error(1.1389453937858296e-31) > Fraction(2) ** -48   # the range's edge
