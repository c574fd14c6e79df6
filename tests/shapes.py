"""Launch-shape rules restated for the tests (no method arithmetic)."""


def lane_shape(K):
    """(lanes per sample, float4 chunks per lane) of the sample-major and
    factorised passes: as few lanes (a power of two, at most 32) as give
    each lane at most four float4 chunks of the K states rounded up to 4;
    three chunks are rounded up to four below 32 lanes."""
    q = (K + 3) // 4
    lps = 1
    while lps < 32 and lps * 4 < q:
        lps *= 2
    nk = -(-q // lps)
    if lps < 32 and nk == 3:
        nk = 4
    return lps, nk


# (K, N) cases of the stateless passes: ragged N, and every dispatched
# (lanes per sample, chunks per lane) instance for K = 1..1024
LANE_SHAPE_CASES = [(1, 7), (3, 4099), (8, 3), (12, 4099), (16, 777), (20, 3001), (37, 5001), (64, 1000),
                    (100, 1999), (130, 2049), (300, 2049), (500, 1333), (600, 1333), (700, 1111), (800, 999),
                    (1000, 777)]
