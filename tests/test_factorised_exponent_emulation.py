"""The exponent of the factorised pass (lse_fact.cu), restated with exact
rational arithmetic for the FP32 fused multiply-adds:

    x = fma(-b_hi, p_hi, c_hi) + fma(-b_lo, p_hi, fma(-b_hi, p_lo, c_lo)),

with (c_hi, c_lo), (b_hi, b_lo), (p_hi, p_lo) the FP32 pairs of the FP64
values c = (f + log N - a) log2(e), b' = b log2(e) and phi. Pinned against
the exact c - b' phi on tempering magnitudes (|c|, |b' phi| ~ 1e3 and more,
cancelling to |x| of a few hundred): the error stays within two FP32 ulps
of x itself (measured: under one), while one FP32 product and difference
lose the ulps of the operands (measured: ~45 ulps of x)."""
from fractions import Fraction

import numpy as np


def f32(x) -> np.float32:
    return np.float32(float(x))


def fma32(a, b, c) -> np.float32:
    return f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def pair(x: float):
    hi = np.float32(x)
    return hi, np.float32(x - float(hi))


def ulp32(x: float) -> float:
    return float(np.spacing(np.float32(abs(x))))


def test_exponent_is_within_a_few_ulps_of_itself():
    g = np.random.default_rng(5)
    s2 = 2000.0
    log2e = 1.4426950408889634
    worst, worst_naive = 0.0, 0.0
    for _ in range(3000):
        bk = g.uniform(0.5, 1.0)
        bp = g.uniform(0.5, 1.0)                      # the sample's own state
        phi = -bp * s2 + np.sqrt(s2) * g.standard_normal()
        f = -bk * bk * s2 / 2 + g.normal() * 3        # near the solution
        c = (f + np.log(4000.0)) * log2e
        b = bk * log2e
        ch, cl = pair(c)
        bh, bl = pair(b)
        ph, pl = pair(phi)
        x = f32(float(fma32(-bh, ph, ch)) + float(fma32(-bl, ph, fma32(-bh, pl, cl))))
        exact = Fraction(c) - Fraction(b) * Fraction(float(phi))
        err = abs(float(Fraction(float(x)) - exact))
        worst = max(worst, err / ulp32(float(exact)))
        naive = f32(float(ch) - float(f32(float(bh) * float(ph))))
        worst_naive = max(worst_naive, abs(float(Fraction(float(naive)) - exact)) / ulp32(float(exact)))
    assert worst <= 2.0
    assert worst_naive > 10.0 * worst
