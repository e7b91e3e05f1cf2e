"""The chord scan's bit-pattern reduction, checked on the host.

The tensor-core kernels fold each row's ratio r = s / g (s >= 0) into the
walker's chord (Algorithm 2: lambda_max = min over g > 0 of r, lambda_min =
max over g < 0 of r) without selects: lambda_max is the unsigned min of the
FP32 bit patterns of all r (negative floats, NaN and the +Inf start rank
above every non-negative ratio), lambda_min the signed min (non-negative
floats and the -Inf start rank above every negative ratio; among negative
floats a smaller magnitude is a smaller signed integer).  This test restates
that reduction in numpy and compares it with the plain definition on edge
cases (s = 0, g = +-0, tiny g, huge g, both signs) and random draws.
"""
import numpy as np
import pytest

INF_BITS = np.uint32(0x7F800000)
NEG_INF_BITS = np.int32(np.uint32(0xFF800000).view(np.int32))


def clamp_slack(s):
    """The kernels' clamp: integer max over the bit pattern (negatives and -0 to +0)."""
    b = np.asarray(s, np.float32).view(np.int32)
    return np.maximum(b, 0).astype(np.int32).view(np.float32)


def bit_chord(s, g):
    """The kernels' reduction (a reciprocal then a product, as in FP32)."""
    s = clamp_slack(s)
    g = np.asarray(g, np.float32)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        r = (s * (np.float32(1.0) / g)).astype(np.float32)
    u = r.view(np.uint32)
    i = r.view(np.int32)
    hi = np.minimum(INF_BITS, u.min(initial=INF_BITS)).view(np.float32)
    lo = np.minimum(NEG_INF_BITS, i.min(initial=NEG_INF_BITS)).view(np.float32)
    return float(lo), float(hi)


def plain_chord(s, g):
    """Algorithm 2's chord from the same rounded ratios, by definition."""
    s = np.maximum(np.asarray(s, np.float32), np.float32(0.0)) + np.float32(0.0)
    g = np.asarray(g, np.float32)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        r = (s * (np.float32(1.0) / g)).astype(np.float32)
    pos = g > 0
    neg = g < 0
    # A ratio from a tiny |g| can overflow to Inf: it bounds nothing.
    hi = r[pos & np.isfinite(r)].min(initial=np.inf)
    lo = r[neg & np.isfinite(r)].max(initial=-np.inf)
    return float(lo), float(hi)


@pytest.mark.parametrize("case", [
    ([1.0, 2.0, 3.0], [1.0, -1.0, 0.5]),          # one row each side
    ([0.0, 1.0], [2.0, -3.0]),                     # s = 0, g > 0: lambda_max = +0
    ([0.0, 1.0], [-2.0, 3.0]),                     # s = 0, g < 0: lambda_min = -0
    ([1.0, 1.0], [0.0, -0.0]),                     # g = +-0: bounds nothing
    ([1.0, 1.0, 2.0], [1e-40, -1e-40, 4.0]),       # subnormal g: ratio overflows
    ([1.0, 5.0], [1e30, -1e30]),                   # huge g: ratio near 0
    ([3.0], [1.0]),                                # open below
    ([3.0], [-1.0]),                               # open above
    ([-0.0, 1.0], [2.0, -1.0]),                    # s = -0 over g > 0: lambda_max = +0
    ([-1e-7, 2.0], [-3.0, 1.0]),                   # negative slack clamps to +0
])
def test_edge_cases(case):
    s, g = case
    lo, hi = bit_chord(s, g)
    plo, phi = plain_chord(s, g)
    assert lo == plo and hi == phi
    # -0 and +0 keep their signs (the chord's end at the point itself).
    assert np.signbit(lo) == np.signbit(plo)
    assert np.signbit(hi) == np.signbit(phi)


def test_random_rows_any_order():
    rng = np.random.default_rng(0)
    for _ in range(200):
        m = int(rng.integers(1, 300))
        s = np.abs(rng.standard_normal(m)).astype(np.float32)
        s[rng.random(m) < 0.05] = 0.0
        g = rng.standard_normal(m).astype(np.float32)
        g[rng.random(m) < 0.05] = 0.0
        lo, hi = bit_chord(s, g)
        assert (lo, hi) == plain_chord(s, g)
        # Any split of the rows, reduced part by part, gives the same bits.
        cut = int(rng.integers(0, m + 1))
        a = bit_chord(s[:cut], g[:cut])
        b = bit_chord(s[cut:], g[cut:])
        assert max(a[0], b[0]) == lo and min(a[1], b[1]) == hi
        perm = rng.permutation(m)
        assert bit_chord(s[perm], g[perm]) == (lo, hi)
