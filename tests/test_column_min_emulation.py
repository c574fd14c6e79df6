"""The per-sample minimum of the mixed-precision staging (prep.cu,
stage_tma_kernel): every binary64 u_kn is mapped to an order-preserving
64-bit integer (negative values: all bits flipped; others: the sign bit
set), each thread keeps the integer minimum of its rows, and one warp per
sample combines its 32 partials as the minimum of the high 32-bit words
followed by the minimum of the low words over the lanes that hold that
high word (two warp-wide unsigned reductions). Restated with Python
integers and pinned against numpy's minimum of the doubles, including
values that share their high word, signed zeros and both signs."""
import numpy as np

MASK64 = (1 << 64) - 1


def ordered_bits(x: float) -> int:
    b = int(np.array([x], dtype=np.float64).view(np.uint64)[0])
    return (~b & MASK64) if (b >> 63) else (b | (1 << 63))


def from_ordered(k: int) -> float:
    b = (k & ~(1 << 63)) if (k >> 63) else (~k & MASK64)
    return float(np.array([b], dtype=np.uint64).view(np.float64)[0])


def warp_min(parts: list[int]) -> int:
    """The two reductions of one warp over its 32 partial minima."""
    hi = [p >> 32 for p in parts]
    lo = [p & 0xFFFFFFFF for p in parts]
    mh = min(hi)
    ml = min(l if h == mh else 0xFFFFFFFF for h, l in zip(hi, lo))
    return (mh << 32) | ml


def column_min(col: np.ndarray, lanes: int = 32) -> float:
    """Rows k = lane, lane + 32, ... per lane, then the warp's reductions."""
    parts = []
    for lane in range(lanes):
        m = MASK64
        for x in col[lane::lanes]:
            m = min(m, ordered_bits(float(x)))
        parts.append(m)
    return from_ordered(warp_min(parts))


def test_ordered_bits_preserve_the_order_of_doubles():
    g = np.random.default_rng(3)
    x = np.concatenate([g.standard_normal(500) * 10.0 ** g.integers(-30, 30, 500),
                        [0.0, -0.0, np.finfo(np.float64).max, -np.finfo(np.float64).max,
                         np.finfo(np.float64).tiny, -np.finfo(np.float64).tiny, 5e-324, -5e-324]])
    keys = [ordered_bits(float(v)) for v in x]
    order = np.lexsort((~np.signbit(x), x))     # by value, -0.0 before +0.0
    ks = [keys[i] for i in order]
    assert all(a <= b for a, b in zip(ks, ks[1:]))
    assert all(from_ordered(k) == v for k, v in zip(keys, x))


def test_warp_minimum_equals_the_64_bit_minimum():
    g = np.random.default_rng(11)
    for _ in range(2000):
        base = int(g.integers(0, 1 << 62)) | (1 << 63)
        # partials that often share the high word and differ in the low one
        parts = [(base & ~0xFFFFFFFF) | int(g.integers(0, 1 << 32)) if g.random() < 0.5
                 else int(g.integers(0, 1 << 63)) | (int(g.integers(0, 2)) << 63) for _ in range(32)]
        assert warp_min(parts) == min(parts)


def test_column_minimum_matches_numpy_on_staged_shapes():
    g = np.random.default_rng(7)
    for K in (1, 31, 33, 500, 512):
        for _ in range(5):
            # energies of the default workload's scale, some columns shifted
            # so that entries share their exponent and high bits
            col = -1e4 + 100.0 * g.standard_normal(K) + 20.0 * g.standard_t(4, K)
            if g.random() < 0.5:
                col = np.round(col, 1)
            assert column_min(col) == float(np.min(col))
    col = np.array([0.0, -0.0, 1.0])
    assert np.signbit(column_min(col))          # -0.0 orders below +0.0
    assert column_min(np.array([-3.5, 2.0, -3.5000000000000004])) == -3.5000000000000004
