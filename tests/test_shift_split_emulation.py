"""The FP32 per-sample shift of the mixed-precision store (prep.cu):
v = (uh - mh) + (ul - ml) from integer hi/lo splits of u and of the column
minimum m (hi = the value truncated toward zero to 24 significant bits, lo =
the dropped 29 fraction bits rounded once to FP32), restated in Python
integers and numpy float32 arithmetic. Pinned against the exact u - m:
within 1.5 units in the last place of fl32(u - m) plus 2^-46 max(|u|, |m|)
(the binary32 rounding of the residuals), exact when the difference is
exactly representable in FP32, never negative. The round-to-nearest split
of the factorised pass (common.cuh split_f64) is pinned separately."""
import struct

import numpy as np


def split(x: float):
    d = struct.unpack("<Q", struct.pack("<d", x))[0]
    dh, dl = d >> 32, d & 0xFFFFFFFF
    E = (dh >> 20) & 0x7FF
    e, s = E - 1023 + 127, E - 1075
    if e <= 0 or e >= 254 or s < -126:
        return None
    sign = dh & 0x80000000
    mant = ((dh & 0xFFFFF) << 3) | (dl >> 29)
    rest = dl & 0x1FFFFFFF
    up = 1 if (rest > 0x10000000 or (rest == 0x10000000 and (mant & 1))) else 0
    hi = struct.unpack("<f", struct.pack("<I", sign | (((e << 23) | mant) + up)))[0]
    r = rest - (up << 29)
    scale = struct.unpack("<f", struct.pack("<I", (s + 127) << 23))[0]
    lo = np.float32(np.float32(r) * np.float32(scale))
    if sign:
        lo = -lo
    return np.float32(hi), np.float32(lo)


def split_trunc(x: float):
    """prep.cu split_f64_trunc: hi = x truncated to 24 significant bits,
    lo = RN32 of the 29 dropped fraction bits; None outside the normal range
    of hi and of lo's scale (|x| outside [2^-74, 2^128))."""
    d = struct.unpack("<Q", struct.pack("<d", x))[0]
    dh, dl = d >> 32, d & 0xFFFFFFFF
    E = (dh >> 20) & 0x7FF
    if not (949 <= E <= 1150):
        return None
    sign = dh & 0x80000000
    hi_bits = sign | ((((dh & 0x7FFFFFFF) - 0x38000000) << 3) & 0xFFFFFFFF) | (dl >> 29)
    hi = struct.unpack("<f", struct.pack("<I", hi_bits))[0]
    scale = struct.unpack("<f", struct.pack("<I", (E - 948) << 23))[0]
    lo = np.float32(np.float32(dl & 0x1FFFFFFF) * np.float32(scale))
    if sign:
        lo = -lo
    return np.float32(hi), np.float32(lo)


def shifted(u: float, m: float) -> np.float32:
    mu = split_trunc(m) if m != 0.0 else (np.float32(0), np.float32(0))
    su = split_trunc(u)
    if mu is None or su is None:
        return np.float32(u - m)
    return np.float32(np.float32(su[0] - mu[0]) + np.float32(su[1] - mu[1]))


def within_bound(v: np.float32, u: float, m: float) -> bool:
    exact = u - m
    ref = np.float32(exact)
    bound = 1.5 * float(np.spacing(np.float32(max(abs(float(ref)), 1e-38)))) + 2.0 ** -46 * max(abs(u), abs(m))
    return abs(float(v) - exact) <= bound


def test_alchemical_like_columns():
    g = np.random.default_rng(0)
    for _ in range(300):
        m = -1e4 + 100 * g.standard_normal()
        for du in np.abs(20 * g.standard_t(4, size=30)) * g.uniform(0, 1, size=30):
            u = m + du
            v = shifted(u, m)
            assert v >= 0.0
            assert within_bound(v, u, m), (u, m, v)


def test_wide_magnitudes_and_the_minimum_itself():
    g = np.random.default_rng(1)
    for _ in range(3000):
        m = g.standard_normal() * 10.0 ** g.integers(-6, 8)
        u = m + abs(g.standard_normal()) * 10.0 ** g.integers(-8, 8)
        v = shifted(u, m)
        assert v >= 0.0
        assert within_bound(v, u, m), (u, m, v)
        assert shifted(m, m) == 0.0


def test_truncating_split_is_exact_in_its_pair():
    """hi + lo reproduces x to within the one rounding of lo: hi is x with
    its low 29 fraction bits cleared (so |hi| <= |x|, same sign) and
    |hi + lo - x| <= 2^-48 |x|."""
    g = np.random.default_rng(5)
    xs = np.concatenate([g.standard_normal(3000) * 10.0 ** g.integers(-20, 30, 3000), [1.0, -1.0, 3.0e5]])
    for x in xs:
        r = split_trunc(float(x))
        if r is None:
            continue
        hi, lo = r
        assert abs(float(hi)) <= abs(float(x)) and np.signbit(hi) == np.signbit(x)
        assert abs(float(hi) + float(lo) - float(x)) <= 2.0 ** -48 * abs(float(x))


def test_binade_boundaries_stay_non_negative():
    """u just above m across powers of two (where truncated hi parts step to
    the next exponent) never gives a negative shifted value."""
    for e in range(-30, 40):
        for m0 in (2.0 ** e, -(2.0 ** e)):
            for k in range(1, 40):
                m = np.nextafter(m0, -np.inf) if k % 2 else m0
                u = float(m)
                for _ in range(k):
                    u = float(np.nextafter(u, np.inf))
                v = shifted(u, float(m))
                assert v >= 0.0
                assert within_bound(v, u, float(m)), (u, m, v)


def test_exact_when_the_difference_is_a_float():
    for m in [-1e4, -12345.678, 3.25, 1e-3]:
        for du in [0.0, 0.5, 1.25, 7.0, 1024.0]:
            assert shifted(m + du, m) == np.float32((m + du) - m)


def test_split_is_round_to_nearest_pair():
    """The same split on the per-sample coordinate of the factorised pass
    (lse_fact.cu): hi = RN32(x) and lo = RN32(x - hi), checked against
    numpy's conversions on energies of the tempering workload's range."""
    g = np.random.default_rng(11)
    xs = np.concatenate([-2000.0 + 45.0 * g.standard_normal(2000), g.uniform(-1e6, 1e6, 2000),
                         g.uniform(-1e-3, 1e-3, 200), [1.0, -1.5, 3.0e5, 2.0**-100]])
    for x in xs:
        r = split(float(x))
        if r is None:           # the kernel takes its FP64 route there
            assert abs(x) < 2.0**-60
            continue
        hi, lo = r
        assert hi == np.float32(x)
        assert lo == np.float32(float(x) - float(hi))


def widen(x: np.float32) -> float:
    """binary32 -> binary64 by integer fields (f32_to_f64_bits in common.cuh)."""
    u = struct.unpack("<I", struct.pack("<f", x))[0]
    sign, e, m = u & 0x80000000, (u >> 23) & 0xFF, u & 0x7FFFFF
    if e == 0:
        if m:
            return float(x)
        hi = sign
    elif e == 0xFF:
        hi = sign | 0x7FF00000 | (m >> 3)
    else:
        hi = sign | ((e + 896) << 20) | (m >> 3)
    bits = (hi << 32) | (m << 29)
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def test_widen_matches_the_conversion():
    g = np.random.default_rng(12)
    xs = np.concatenate([g.standard_normal(3000) * 10.0 ** g.integers(-30, 30, 3000),
                         [0.0, -0.0, 1.0, -2.5, 3.4028235e38, -1.1754944e-38, np.inf, -np.inf]]).astype(np.float32)
    for x in xs:
        w = widen(x)
        assert w == float(x) and np.signbit(w) == np.signbit(x)
    assert np.isnan(widen(np.float32(np.nan)))
