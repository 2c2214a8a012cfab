"""Pins of the oracle's float-format configuration logic against values the
paper prints (alphabets, Example ex:ov-base, Fig. 2 and Fig. 3 captions, Table
tab:moduli, Example ex:widened), plus the product planner's frozen
configurations checked against the oracle (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import forms

SLOW = os.environ.get("OZ_SLOW_TESTS") == "1"


def test_e2m1_alphabet_and_products():
    """Sec. 'Forms and Channels': S = {0, +-1, +-2, +-3, +-4, +-6, +-8, +-12} at
    e_S = 1; Example ex:ov-decoders: |S.S| = 37."""
    S, e = forms.alphabet("E2M1")
    assert e == 1 and S == [-12, -8, -6, -4, -3, -2, -1, 0, 1, 2, 3, 4, 6, 8, 12]
    assert len({a * b for a in S for b in S}) == 37


def test_plane_radius_under_fp32_accumulation():
    """Example ex:ov-equiv: r_max(1) = 32 under FP32 accumulation at K = 2^14
    (eq. rmax with Lambda = 2^24)."""
    assert forms.LAMBDA_FP32 == 2**24
    assert forms.rmax1(2**14, forms.LAMBDA_FP32) == 32
    assert forms.rmax1(2**13, forms.LAMBDA_FP32) == 45


@pytest.mark.parametrize("name,dtype", [("E4M3", "float8_e4m3fn"), ("E5M2", "float8_e5m2")])
def test_fp8_values_and_codes_match_a_library_decoder(name, dtype):
    """The OCP FP8 encodings as PyTorch decodes them: every finite code's
    value, times 2^e_S, is the oracle's code table entry, and the finite
    values are exactly the oracle's value set (E4M3 tops out at 448, its
    all-ones code being NaN; E5M2 keeps IEEE infinities and NaNs)."""
    torch = pytest.importorskip("torch")
    dt = getattr(torch, dtype, None)
    if dt is None:
        pytest.skip(f"torch without {dtype}")
    vals = torch.arange(256, dtype=torch.uint8).view(dt).to(torch.float64).tolist()
    finite = {c: v for c, v in enumerate(vals) if math.isfinite(v)}
    _, e_s = forms.alphabet(name)
    codes = forms.code_values(name)
    assert set(codes) == set(finite)
    assert all(codes[c] == finite[c] * 2**e_s for c in finite)
    from fractions import Fraction
    assert forms.float_values(name) == {Fraction(v) for v in finite.values()}


def test_fp8_fp6_alphabets_agree():
    """Example ex:ov-equiv: E4M3 agrees with E2M3 up to 60 and E5M2 with E3M2 up
    to 448; Sec. 'FP8 and FP6': within radius 32, 49 values for E4M3 and E2M3
    against 33 for E5M2 and E3M2."""
    sc = {}
    for n in ("E4M3", "E2M3", "E5M2", "E3M2"):
        vals = forms.float_values(n)
        unit = min(abs(v) for v in vals if v)
        sc[n] = sorted(v / unit for v in vals)      # in units of the smallest subnormal
    e2m3 = set(sc["E2M3"])
    assert max(e2m3) == 60 and {v for v in sc["E4M3"] if abs(v) <= 60} == e2m3
    e3m2 = set(sc["E3M2"])
    assert max(e3m2) == 448 and {v for v in sc["E5M2"] if abs(v) <= 448} == e3m2
    for n, count in (("E4M3", 49), ("E2M3", 49), ("E5M2", 33), ("E3M2", 33)):
        S, _ = forms.alphabet(n)
        assert len([s for s in S if abs(s) <= 32]) == count


def test_example_base13_limbs():
    """Example ex:ov-base and Fig. 2: at b = 13 over E2M1, 5 = -8 + 13; one limb
    covers [-4, 4], two cover [-56, 56]; past that run 58, 60, 64 are reachable
    and 57, 59, 61, 62, 63, 65 are not; channel (115, 13, 2) stores class 57 as
    (-6, -4) and has radius 8; 13 values lie within radius 8, and (169, 13, 2)
    is admissible."""
    S, _ = forms.alphabet("E2M1")
    assert 5 not in S and -8 + 13 * 1 == 5
    one = set(S)
    two = {a + 13 * b for a in S for b in S}

    def run(vals):
        X = 0
        while X + 1 in vals and -(X + 1) in vals:
            X += 1
        return X

    assert run(one) == 4 and run(two) == 56
    assert {58, 60, 64} <= two and not ({57, 59, 61, 62, 63, 65} & two)
    t = forms.tables("E2M1", 2**14, 115, "school4", 13)
    assert (t[0][57], t[1][57]) == (-6, -4)
    assert max(max(abs(t[0][c]), abs(t[1][c])) for c in range(115)) == 8
    assert len([s for s in S if abs(s) <= 8]) == 13
    t169 = forms.tables("E2M1", 2**14, 169, "school3", 13)
    assert max(max(abs(t169[0][c]), abs(t169[1][c])) for c in range(169)) <= 8


def _schoolbook_only(pool):
    rank = {}
    for m, k in pool.kind.items():
        if k == "one":
            rank[m] = 1
        elif k == "school3":
            rank[m] = 3
        else:
            rank[m] = 4        # every two-limb member admits a rank-4 schoolbook
    return rank


def test_fig3_schoolbook_pool_and_its_optimum():
    """Fig. 3 caption: E2M1's one-limb and two-limb schoolbook channels at
    K = 2^14 under FP32 accumulation: 147 channels; the least set has
    Q = 4*1 + 2*3 + 14*4 = 66 with P = 2^122.36."""
    pool = forms.Pools("E2M1", 2**14)
    assert len(pool.rank) == 147
    Q, mods = forms.least_q(_schoolbook_only(pool), 2**14)
    assert Q == 66
    assert abs(math.log2(math.prod(mods)) - 122.36) < 0.005
    counts = {}
    for m in mods:
        r = _schoolbook_only(pool)[m]
        counts[r] = counts.get(r, 0) + 1
    assert counts == {1: 4, 3: 2, 4: 14}


@pytest.mark.parametrize("K,Q", [(2**12, 58), (2**14, 59), (2**16, 61), (2**18, 62)])
def test_table_moduli_e2m1(K, Q):
    """Table tab:moduli, row 'E2M1 (ours)'."""
    pool = forms.Pools("E2M1", K)
    assert forms.least_q(pool.rank, K)[0] == Q


@pytest.mark.parametrize("K,Q", [(2**12, 49), (2**14, 50), (2**16, 51), (2**18, 52)])
def test_table_moduli_int4(K, Q):
    """Table tab:moduli, row 'INT4 (ours)' (INT32 accumulation)."""
    pool = forms.Pools("INT4", K, forms.LAMBDA_INT32)
    assert forms.least_q(pool.rank, K)[0] == Q


@pytest.mark.parametrize("d,Q", [(16, 78)])
def test_widened_e2m1(d, Q):
    """Example ex:widened: at E2M1 and K = 2^14, operands spanning 2^16 keep
    53 + 16 bits and need 78 GEMMs. (Its 134 at 2^64 needs moduli above 169,
    i.e. three-limb forms, which this candidate set does not build.)"""
    pool = forms.Pools("E2M1", 2**14)
    assert forms.least_q(pool.rank, 2**14, beta=53 + d)[0] == Q


@pytest.mark.skipif(not SLOW, reason="minutes of CPU; set OZ_SLOW_TESTS=1")
def test_table_moduli_e2m3_at_2p14():
    """Table tab:moduli, row 'E4M3, E2M3 (ours)' at K = 2^14: 30, made of 15
    one-limb channels and 5 channels of three GEMMs (Sec. 'FP8 and FP6')."""
    pool = forms.Pools("E2M3", 2**14)
    Q, mods = forms.least_q(pool.rank, 2**14)
    assert Q == 30
    assert sorted(pool.rank[m] for m in mods) == [1] * 15 + [3] * 5


@pytest.mark.parametrize("name,K,top", [("E2M1", 2**14, None), ("E4M3", 2**13, 400), ("E3M2", 2**13, 400)])
def test_form_tables_decode_and_recombine(name, K, top):
    """Sec. 'Forms and Channels' for every form kind the pools hold: each
    class c of a channel is stored as plane values of the alphabet within the
    plane radius whose limb value (a0 for one limb, a0 + b a1 for two) is c
    modulo m, and the form's GEMMs recombine with their weights into the
    product of the limb values. For the four-GEMM schoolbook this is the
    expansion of (a0 + b a1)(b0 + b b1); for Toom at 0, 1 and infinity it is
    a0 b0 (1 - b) + (a0 + a1)(b0 + b1) b + a1 b1 (b^2 - b), the same
    polynomial; both are exact integer identities. The three-GEMM schoolbook
    drops a1 b1 b^2, which is 0 modulo m because m divides b^2 (eq. qm)."""
    pool = forms.Pools(name, K, m_top=top)
    S, _ = forms.alphabet(name)
    r = forms.rmax1(K, forms.LAMBDA_FP32)
    allowed = {s for s in S if abs(s) <= r}
    by_kind = {}
    for m, kind in sorted(pool.kind.items()):
        by_kind.setdefault(kind, []).append(m)
    assert set(by_kind) >= {"one", "toom", "school3"}
    rng = np.random.default_rng(1)

    def value(planes, kind, b):
        return planes[0] if kind == "one" else planes[0] + b * planes[-1]

    for kind, ms in by_kind.items():
        for m in ms[:3] + ms[-2:]:
            b = pool.base[m]
            t = forms.tables(name, K, m, kind, b)
            if kind == "toom":
                assert all(t[1][c] == t[0][c] + t[2][c] for c in range(m))
            for c in range(m):
                planes = [t[p][c] for p in range(len(t))]
                assert all(v in allowed for v in planes), (kind, m, c)
                assert value(planes, kind, b) % m == c, (kind, m, c)
            w = forms.weights(kind, b)
            for c1, c2 in rng.integers(0, m, size=(64, 2)):
                x = [t[p][c1] for p in range(len(t))]
                y = [t[p][c2] for p in range(len(t))]
                total = sum(lam * x[pa] * y[pb] for pa, pb, lam in w)
                exact = value(x, kind, b) * value(y, kind, b)
                if kind == "school3":
                    assert (b * b) % m == 0 and total == exact - b * b * x[1] * y[1]
                else:
                    assert total == exact, (kind, m)
                assert total % m == (int(c1) * int(c2)) % m
