"""Exhaustive check of the claim that the split's fp32 reduction is exact
(no GPU).

The split forms, per modulus m, the integer y = P0 + sum_i P_i c_i from
signed pieces of the truncated integer (a first piece of 22 bits,
|P0| <= 2^22 - 1, then 13-bit pieces, |P_i| <= 8191, at most four of them;
or 12-bit pieces, at most six) and constants c_i = 2^(bits below piece i)
mod m taken nearest zero (|c_i| <= floor(m/2) <= 119). It then takes
q = rint(y fl(1/m)) with one rounding of the exact product (an fma against
1.5 * 2^23) and r = y - q m, and for the even modulus maps r = +m/2 to -m/2.
The claim: r is the representative of a' modulo m nearest zero in
[-floor(m/2), ceil(m/2) - 1] for every reachable y (Sec. "Ozaki II"). It
holds because fl(1/m) is off by at most half an ulp, which moves y/m by less
than |y| 2^-24 / m < 1/(2m), while for odd m an integer over m is at least
1/(2m) from every half-integer; for even m a half-integer y/m may round
either way, and the fix takes the tie to -m/2.

Here every reachable y (|y| <= 2^22 - 1 + 4 * 8191 * 119) is tried for every
modulus the INT8 plans use (the 20 of the nested max-product list up to 239),
against exact integer arithmetic. fl(1/m) is the float32 quotient 1.0f / m.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

MODULI = oracle.max_product_moduli(20, 239)
Y_MAX = (2**22 - 1) + 4 * 8191 * 119      # 22 + 4 x 13 bits; 22 + 6 x 12 bits reaches less


def test_reachable_range_covers_both_piece_layouts():
    assert (2**22 - 1) + 6 * 4095 * 119 < Y_MAX < 2**23
    assert (2**22 - 1) + 3 * 8191 * 119 < Y_MAX
    assert max(m // 2 for m in MODULI) == 119
    # 22 + 3 x 13 = 61 bits (beta <= 61), 22 + 4 x 13 = 74, 22 + 6 x 12 = 94 (widened a' < 2^84)
    assert 22 + 3 * 13 == 61 and 22 + 4 * 13 >= 64 and 22 + 6 * 12 >= 84
    # the only even modulus is the third of the list (the split's tie fix is for index 2 only)
    assert [i for i, m in enumerate(MODULI) if m % 2 == 0] == [2]


@pytest.mark.parametrize("m", MODULI)
def test_single_rint_reduction_is_exact(m):
    invm = float(np.float32(1.0) / np.float32(m))
    step = 1 << 22
    for lo in range(-Y_MAX, Y_MAX + 1, step):
        y = np.arange(lo, min(lo + step, Y_MAX + 1), dtype=np.int64)
        q = np.rint(y.astype(np.float64) * invm)             # exact product, the fma's one rounding
        r = y - q.astype(np.int64) * m                          # exact in fp32 too: |r| <= m/2 < 2^8
        if m % 2 == 0:
            r = np.where(r == m // 2, -(m // 2), r)             # the tie fix of the even modulus
        assert r.min() >= -(m // 2) and r.max() <= (m + 1) // 2 - 1
        assert np.array_equal(r % m, y % m)


T_MAX = 1024 * 119 * 119 + 2 * 120    # a slab's sum plus the residue it lands on (and the other chain's)


@pytest.mark.parametrize("m", MODULI)
def test_slab_drain_reduction_bounds_the_residue(m):
    """The TC GEMM epilogue reduces each FP32 accumulator value t (an integer,
    |t| <= 1024 * 119^2 + 240 < 2^24) to r = t - m rint(t fl(1/m)), one fma
    rounding for the quotient. Claim: r = t mod m and |r| <= 120, so the next
    slab's sum on top of r stays below 2^24 (eq. ov-accgen) and r + 128 fits
    in a byte. Every t in range is tried."""
    assert T_MAX < 2**24
    invm = float(np.float32(1.0) / np.float32(m))
    step = 1 << 22
    for lo in range(-T_MAX, T_MAX + 1, step):
        t = np.arange(lo, min(lo + step, T_MAX + 1), dtype=np.int64)
        q = np.rint(t.astype(np.float64) * invm)              # exact product, one rounding
        r = t - q.astype(np.int64) * m
        assert np.abs(r).max() <= 120
        assert np.array_equal(r % m, t % m)


@pytest.mark.parametrize("m", MODULI)
def test_digit_step_lands_in_range(m):
    """The last slab's digit: from the balanced residue r of W (|r| <= 120),
    y = r f with f = (P/m)^-1 mod m, or f = 1 for the raw value W mod m
    (|y| <= 120 * 238 < 2^15, exact in fp32), then one floor quotient
    q = rint(fl32(y fl(1/m) + bias)), bias = fl32(-1/2 + fl(1/m) / 2), by an
    fma and the 1.5 * 2^23 rounding constant, and d = y - q m. Claim: d is
    (W mod m) f mod m in [0, m), for every r and every f below m (so for
    whatever (P/m)^-1 a plan has, and for raw). The emulation is exact: the
    fma's product and sum are exact in float64 (39 significant bits), and
    float64 -> float32 and rint both round to nearest even, as the GPU does."""
    invm = np.float32(1.0) / np.float32(m)
    bias = np.float32(0.5 * np.float64(invm) - 0.5)
    r = np.arange(-120, 121, dtype=np.int64)
    for f in range(m):
        y = r * f
        t = (y.astype(np.float64) * np.float64(invm) + np.float64(bias)).astype(np.float32)
        q = np.rint(t.astype(np.float64)).astype(np.int64)
        d = y - q * m
        assert d.min() >= 0 and d.max() < m
        assert np.array_equal(d, (r * f) % m)


@pytest.mark.parametrize("fmt", ["E4M3", "E5M2", "E2M3", "E3M2", "E2M1"])
@pytest.mark.parametrize("k_hint", [8192, 16384])
def test_float_format_fold_stays_exact(fmt, k_hint):
    """The float-format GEMM epilogue folds each GEMM's integer W of a channel
    (|W| <= K rho^2 <= 2^24, rho the largest plane value of the plan and K
    its accumulation cap k_acc, the longest inner dimension one GEMM may take,
    Sec. "Slabs") into the channel's running
    residue r, all in fp32: wm = W - m rint(W fl(1/m)), t = lambda wm + r,
    r' = t - m rint(t fl(1/m)), with 0 <= lambda < m. From the exact error of
    fl(1/m) this bounds |wm|, shows t below 2^24 (so exact), and gives a bound
    R >= |r'| that holds for every fold: R < 0.51 m, and r + 2048 fits its
    16-bit field. At the end, r is taken to [0, m) and multiplied by the CRT
    coefficient (below m^2 < 2^24), and one more quotient lands in (-m, m)."""
    import paper_2609_37693_gb300 as oz
    plan = oz.PlanFP(fmt, k_hint)
    # the premise, from the plan itself: its plane tables and its cap
    rho = max(max(abs(int(v)) for v in tab) for tab in plan.plane_values())
    K = plan.k_acc
    assert K >= plan.k_cfg
    w_max = K * rho * rho
    assert w_max <= 2**24
    for m in plan.moduli:
        assert m < 4096
        delta = abs(Fraction(float(np.float32(1.0) / np.float32(m))) - Fraction(1, m))
        wm_max = Fraction(m, 2) + m * w_max * delta
        assert wm_max < Fraction(65, 100) * m
        # R = m/2 + m delta ((m - 1) wm_max + R), the bound that reproduces itself
        R = (Fraction(m, 2) + m * delta * (m - 1) * wm_max) / (1 - m * delta)
        assert (m - 1) * wm_max + R < 2**24
        assert R < Fraction(51, 100) * m and R < 2048
        assert (m - 1) ** 2 < 2**24 and Fraction(1, 2) + (m - 1) ** 2 * delta < 1


def _groups(moduli):
    """The grouping of the byte-digit reconstruct: triples, then the last one
    or two moduli joined into a quad (product below 2^31) or pairs."""
    Q = len(moduli)
    nt, rest = Q // 3, Q % 3
    sizes = [3] * nt
    if rest == 2:
        sizes.append(2)
    elif rest == 1:
        sizes.pop()
        if math.prod(moduli[Q - 4:]) < 2**31:
            sizes.append(4)
        else:
            sizes += [2, 2]
    out, q = [], 0
    for sz in sizes:
        out.append(tuple(moduli[q:q + sz]))
        q += sz
    return out


def _group_t(grp, y):
    """t_g as the kernel forms it: sum y_q (M_g / m_q); a quad reduces each pair first."""
    if len(grp) == 4:
        ma, mb, mc, md = grp
        zab, zcd = y[0] * mb + y[1] * ma, y[2] * md + y[3] * mc
        wab, wcd = zab % (ma * mb), zcd % (mc * md)
        assert zab < 2 * ma * mb and zcd < 2 * mc * md    # one conditional subtraction reduces each
        return wab * (mc * md) + wcd * (ma * mb)
    Mg = math.prod(grp)
    return sum(yq * (Mg // mq) for yq, mq in zip(y, grp))


@pytest.mark.parametrize("Q", list(range(9, 17)))
def test_grouped_crt_sum_is_exact(Q):
    """The reconstruct of byte digits in groups of moduli (Sec. "Around the
    GEMMs", Reconstruct): every t_g fits 32 bits and the sum of their maxima
    stays below 2^32 (so each 64-bit accumulator of t_g times a 32-bit limb of
    P / M_g is exact), P / M_g fits four limbs, S = sum_g t_g (P / M_g) is
    congruent to X modulo P and below 15 P (the table of qP has 16 entries),
    and the fp32 quotient estimate sum_g fl(t_g) fl(1 / M_g) (fused
    multiply-adds, every term non-negative) is within 2^-18 of S / P, far
    inside the 2^-10 margin below which the kernel settles a tie exactly.
    Checked on the largest digits, single-digit patterns and random digits
    against Python integers."""
    import numpy as np
    mods = oracle.max_product_moduli(Q)
    P = math.prod(mods)
    assert P.bit_length() <= 125 and all(m < 256 for m in mods)
    groups = _groups(mods)
    tmax = [(2 if len(g) == 4 else len(g)) * math.prod(g) for g in groups]
    assert sum(tmax) < 2**32 and sum(t // math.prod(g) for t, g in zip(tmax, groups)) <= 15
    for g in groups:
        if len(g) == 3:
            assert all(a * b < 2**16 for a, b in ((g[1], g[2]), (g[0], g[2]), (g[0], g[1])))
        assert (P // math.prod(g)).bit_length() <= 128
    invM = [np.float32(1.0 / math.prod(g)) for g in groups]
    inv = [pow(P // m, -1, m) for m in mods]
    rng = np.random.default_rng(Q)
    cases = [[m - 1 for m in mods], [0] * Q]
    cases += [[m - 1 if i == r else 0 for i, m in enumerate(mods)] for r in range(Q)]
    cases += [[int(rng.integers(0, m)) for m in mods] for _ in range(2000)]
    for y in cases:
        acc = [0, 0, 0, 0]
        q = 0
        f = np.float32(0.0)
        for gi, g in enumerate(groups):
            t = _group_t(g, y[q:q + len(g)])
            assert 0 <= t < 2**32
            # fmaf: one rounding of fl(t) * fl(1/M) + f
            f = np.float32(Fraction(float(np.float32(t))) * Fraction(float(invM[gi])) + Fraction(float(f)))
            N = P // math.prod(g)
            for l in range(4):
                acc[l] += t * ((N >> (32 * l)) & 0xffffffff)
            q += len(g)
        assert max(acc) < 2**64
        S = acc[0] + (acc[1] << 32) + (acc[2] << 64) + (acc[3] << 96)
        X = sum(yq * (P // m) for yq, m in zip(y, mods)) % P
        assert S % P == X and S < 15 * P
        # the residues the digits encode: y_q = (X mod m_q) inv_q mod m_q
        assert all((X % m) * iv % m == yq for yq, m, iv in zip(y, mods, inv))
        assert abs(Fraction(float(f)) - Fraction(S, P)) < Fraction(1, 2**18)
