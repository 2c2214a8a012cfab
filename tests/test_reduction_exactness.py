"""Exhaustive check of the claim that the split's fp32 reduction is exact
(no GPU).

The split forms, per modulus m, the quarter-integer y' = P0 + 1/4 + sum_i P_i c_i
from signed pieces of the truncated integer (13-bit pieces, |P_i| <= 8191,
at most four constants; or 12-bit pieces, at most six) and constants c_i =
2^(bits i) mod m taken nearest zero (|c_i| <= floor(m/2) <= 119). It then
takes q = rint(y' fl(1/m)) with one rounding of the exact product (an fma
against 1.5 * 2^23) and r = y' - q m - 1/4. The claim: q is the integer
nearest y'/m for every reachable y', so r is the representative of a' modulo
m nearest zero in [-floor(m/2), ceil(m/2) - 1] (Sec. "Ozaki II"). It holds
because fl(1/m) is off by at most half an ulp, which moves y'/m by less than
1/(4m), while a quarter-integer over m is at least 1/(4m) from every
half-integer.

Here every reachable y' (|y'| <= 8191 (1 + 4 * 119) + 1/4) is tried for every
modulus the INT8 plans use (the 20 of the nested max-product list up to 239),
against exact integer arithmetic. fl(1/m) is the float32 quotient 1.0f / m.
"""
import numpy as np
import pytest

import oracle

MODULI = oracle.max_product_moduli(20, 239)
Y_MAX = 8191 * (1 + 4 * 119)          # 13-bit pieces; the 12-bit case (4095 * (1 + 6 * 119)) is smaller


def test_reachable_range_covers_both_piece_widths():
    assert 4095 * (1 + 6 * 119) < Y_MAX < 2**22
    assert max(m // 2 for m in MODULI) == 119


@pytest.mark.parametrize("m", MODULI)
def test_single_rint_reduction_is_exact(m):
    k = np.arange(-Y_MAX - 1, Y_MAX + 1, dtype=np.int64)        # y' = k + 1/4
    y = k.astype(np.float64) + 0.25
    invm = float(np.float32(1.0) / np.float32(m))
    t = y * invm                                                  # exact: 24-bit by 24-bit significands
    q = np.rint(t)                                                # the fma's one rounding, ties to even
    # the integer nearest (4k + 1) / (4m); no ties, since 4k + 1 is odd
    nearest = (4 * k + 1 + 2 * m) // (4 * m)
    assert np.array_equal(q.astype(np.int64), nearest)
    r = y - q * m - 0.25                                          # exact in float64 (and in fp32: |r| < 2^8)
    assert np.array_equal(r, np.rint(r))
    ri = r.astype(np.int64)
    assert ri.min() >= -(m // 2) and ri.max() <= (m + 1) // 2 - 1
    assert np.array_equal(ri % m, k % m)                          # r = a' mod m: y' - 1/4 = k
