"""The integer binary64 -> binary32 round-to-nearest-even of the FP32 shift
(prep.cu, f64_to_f32_rn), restated step by step in Python integers and
checked against numpy's IEEE conversion on random, tie, carry and edge
values. The CUDA function performs the same integer steps."""
import struct

import numpy as np


def f64_to_f32_bits(x: float) -> int | None:
    d = struct.unpack("<Q", struct.pack("<d", x))[0]
    hi, lo = d >> 32, d & 0xFFFFFFFF
    e = ((hi >> 20) & 0x7FF) - 1023 + 127
    if e <= 0 or e >= 255:
        return None                      # hardware conversion path
    sign = hi & 0x80000000
    mant = ((hi & 0xFFFFF) << 3) | (lo >> 29)
    rest = lo & 0x1FFFFFFF
    half = 0x10000000
    up = 1 if (rest > half or (rest == half and (mant & 1))) else 0
    return sign | (((e << 23) | mant) + up)


def ref_bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", np.float32(x)))[0]


def test_random_values_match_ieee():
    g = np.random.default_rng(0)
    xs = np.concatenate([g.standard_normal(20000) * 10.0 ** g.integers(-30, 30, 20000),
                         g.uniform(0, 1e4, 20000)])
    for x in xs:
        b = f64_to_f32_bits(float(x))
        if b is not None:
            assert b == ref_bits(float(x)), x


def test_ties_round_to_even_and_carries():
    for f in [1.0, 1.5, 3.0, 1234.5, 2.0 ** 20 + 1.0, 16777215.0]:
        f32 = np.float32(f)
        ulp = np.spacing(f32)
        for frac in [0.5, 0.25, 0.75, 0.5 + 2.0 ** -30, 0.5 - 2.0 ** -30]:
            x = float(f32) + frac * float(ulp)
            b = f64_to_f32_bits(x)
            assert b == ref_bits(x), (f, frac)
    x = float(np.float32(3.4e38)) * (1 + 2.0 ** -25)   # rounds within range
    assert f64_to_f32_bits(x) == ref_bits(x)
    x = 2.0 - 2.0 ** -30                               # fraction carry into the exponent
    assert f64_to_f32_bits(x) == ref_bits(x) == 0x40000000


def test_out_of_range_values_take_the_hardware_path():
    assert f64_to_f32_bits(0.0) is None
    assert f64_to_f32_bits(1e-40) is None
    assert f64_to_f32_bits(1e39) is None
