"""The exponent of the factorised pass (lse_fact.cu), restated with exact
rational arithmetic for each FP32 add and fused multiply-add. Where the
exponents can exceed 2^12 in magnitude, every sample is taken relative to a
reference state r near its largest exponent (below that the pass forms x_kp
itself; the second test):

    x_k - x_r = fma(-(b_hi,k - b_hi,r), p_hi, c_hi,k - c_hi,r) + (lo_k - lo_r),
    lo_k      = fma(-b_lo,k, p_hi, fma(-b_hi,k, p_lo, c_lo,k)),

with (c_hi, c_lo), (b_hi, b_lo), (p_hi, p_lo) the FP32 pairs of the FP64
values c = (f + log N - a) log2(e), b' = b log2(e) and phi. The two hi
differences are exact where c_k, c_r (b'_k, b'_r) lie within a factor of two
(Sterbenz), else they round at their own magnitude; so the error is bounded
by a few FP32 ulps of x_k - x_r, c_k - c_r and (b'_k - b'_r) phi, not of
x_k. Pinned on replica-ladder magnitudes (u = beta_k E, beta = 1 + D k up to
~520, so c and b' phi reach ~1e5 and cancel to x ~ 1e5, while the states
that carry weight differ by a few units): within two of those ulps; the
absolute form x_k = fma(-b_hi, p_hi, c_hi) + ..., rounded at the magnitude
of x_k, misses the difference by hundreds of them on the upper rungs."""
from fractions import Fraction

import numpy as np

LOG2E = 1.4426950408889634


def f32(x) -> np.float32:
    return np.float32(float(x))


def add32(a, b) -> np.float32:
    return f32(Fraction(float(a)) + Fraction(float(b)))


def fma32(a, b, c) -> np.float32:
    return f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def pair(x: float):
    hi = np.float32(x)
    return hi, np.float32(x - float(hi))


def ulp32(x: float) -> float:
    return float(np.spacing(np.float32(max(abs(x), 2.0 ** -24))))


def lo_part(cl, bh, bl, ph, pl):
    return fma32(-bl, ph, fma32(-bh, pl, cl))


def relative_exponent(k, r, ph, pl):
    """The kernel's x_k - x_r from the pairs of states k and r."""
    (chk, clk, bhk, blk), (chr_, clr, bhr, blr) = k, r
    dch = add32(chk, -chr_)
    ndb = add32(-bhk, bhr)
    xh = fma32(ndb, ph, dch)
    return add32(xh, add32(lo_part(clk, bhk, blk, ph, pl), -lo_part(clr, bhr, blr, ph, pl)))


def absolute_exponent(k, ph, pl):
    ch, cl, bh, bl = k
    return add32(fma32(-bh, ph, ch), lo_part(cl, bh, bl, ph, pl))


def test_relative_exponent_is_within_a_few_ulps_of_the_difference():
    g = np.random.default_rng(5)
    D = 0.5066942062715996          # Sec. IV spacing at 80 % neighbour overlap
    worst, worst_abs = 0.0, 0.0
    for _ in range(1500):
        j = int(g.integers(0, 1024))
        beta = lambda k: 1.0 + D * k
        E = -beta(j) + g.standard_normal()
        f = lambda k: -beta(k) ** 2 / 2 + g.normal() * 1e-3
        consts = {}
        for k in range(max(0, j - 4), j + 5):
            c = (f(k) + np.log(20000.0)) * LOG2E
            b = beta(k) * LOG2E
            consts[k] = (*pair(c), *pair(b))
        ph, pl = pair(E)
        # reference: the largest exponent among the sample's neighbours
        xs = {k: Fraction(float(consts[k][0])) + Fraction(float(consts[k][1]))
              - (Fraction(float(consts[k][2])) + Fraction(float(consts[k][3]))) * Fraction(float(E))
              for k in consts}
        r = max(xs, key=lambda k: xs[k])
        for k in consts:
            exact = float(xs[k] - xs[r])
            if exact < -30.0:       # weight below 2^-30 of the sample's largest
                continue
            dc = float(consts[k][0]) - float(consts[r][0])
            dbp = (float(consts[k][2]) - float(consts[r][2])) * float(E)
            scale = ulp32(exact) + ulp32(dc) + ulp32(dbp)
            if max(abs(float(consts[k][0])), abs(float(consts[r][0]))) >= 1e3:
                # large rungs: the hi differences are exact (Sterbenz)
                assert Fraction(float(add32(consts[k][0], -consts[r][0]))) == \
                    Fraction(float(consts[k][0])) - Fraction(float(consts[r][0]))
                assert Fraction(float(add32(-consts[k][2], consts[r][2]))) == \
                    Fraction(float(consts[r][2])) - Fraction(float(consts[k][2]))
            rel = relative_exponent(consts[k], consts[r], ph, pl)
            worst = max(worst, abs(float(rel) - exact) / scale)
            if j > 200:
                absd = float(absolute_exponent(consts[k], ph, pl)) - float(absolute_exponent(consts[r], ph, pl))
                worst_abs = max(worst_abs, abs(absd - exact) / scale)
    assert worst <= 2.0
    assert worst_abs > 100.0 * worst


def test_absolute_exponent_is_within_a_few_ulps_of_itself():
    """Below the 2^12 switch the pass forms x_kp itself: fma(-b_hi, p_hi,
    c_hi) + lo_k, rounded once where c and b' phi cancel. Pinned on
    tempering magnitudes (|c|, |b' phi| ~ 1e3, |x| a few hundred): within
    two FP32 ulps of x, while a plain FP32 product and difference lose the
    operands' ulps (tens of ulps of x)."""
    g = np.random.default_rng(5)
    s2 = 2000.0
    worst, worst_naive = 0.0, 0.0
    for _ in range(3000):
        bk = g.uniform(0.5, 1.0)
        bp = g.uniform(0.5, 1.0)                      # the sample's own state
        phi = -bp * s2 + np.sqrt(s2) * g.standard_normal()
        f = -bk * bk * s2 / 2 + g.normal() * 3        # near the solution
        c = (f + np.log(4000.0)) * LOG2E
        b = bk * LOG2E
        k = (*pair(c), *pair(b))
        ph, pl = pair(phi)
        x = absolute_exponent(k, ph, pl)
        exact = Fraction(c) - Fraction(b) * Fraction(float(phi))
        assert abs(float(exact)) < 4096.0               # the absolute form's range
        worst = max(worst, abs(float(Fraction(float(x)) - exact)) / ulp32(float(exact)))
        naive = f32(float(k[0]) - float(f32(float(k[2]) * float(ph))))
        worst_naive = max(worst_naive, abs(float(Fraction(float(naive)) - exact)) / ulp32(float(exact)))
    assert worst <= 2.0
    assert worst_naive > 10.0 * worst
