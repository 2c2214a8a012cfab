"""The library's frozen float-format configurations against the oracle (no
GPU): valid configurations (pairwise coprime, window, exactness), least GEMM
counts equal to the oracle's search or the paper's printed values, and plane
tables equal to the oracle's enumeration."""
import itertools
import math
import os

import pytest

import paper_2609_37693_gb300 as oz
from oracle import forms

KIND = {1: "one", 2: "school3", 3: "toom", 4: "school4"}
SLOW = os.environ.get("OZ_SLOW_TESTS") == "1"


def _plan(fmt, K):
    return oz.PlanFP(fmt, K)


@pytest.mark.parametrize("fmt", ["E4M3", "E2M3", "E3M2", "E5M2", "E2M1"])
@pytest.mark.parametrize("K,beta", [(8192, 53), (16384, 53), (65536, 53), (16384, 69)])
def test_configuration_is_valid_and_tables_match_oracle(fmt, K, beta):
    p = oz.PlanFP(fmt, K, beta if beta > 53 else 0)
    assert p.k_cfg == K and p.bits >= beta
    assert all(math.gcd(a, b) == 1 for a, b in itertools.combinations(p.moduli, 2))
    P = math.prod(p.moduli)
    assert P > 2 * K * (2**beta - 1) ** 2                      # eq. ov-crtgen at beta bits
    assert p.q == sum(len(forms.weights(KIND[f], b)) for f, b in zip(p.forms, p.bases))
    r = forms.rmax1(K, forms.LAMBDA_FP32)
    vals = p.plane_values()
    i = 0
    S = set(forms.alphabet(fmt)[0])
    for m, f, b in zip(p.moduli, p.forms, p.bases):
        ref = forms.tables(fmt, K, m, KIND[f], b)
        for plane in ref:
            assert vals[i] == plane, (fmt, m)
            assert all(v in S and abs(v) <= r for v in plane)     # eq. ov-accgen per GEMM
            i += 1
        # the form's identity eq. ov-linear, checked on every pair of classes
        for c1 in range(0, m, max(1, m // 23)):
            for c2 in range(0, m, max(1, m // 19)):
                lhs = sum(lam * ref[pa][c1] * ref[pb][c2] for pa, pb, lam in forms.weights(KIND[f], b))
                assert (lhs - c1 * c2) % m == 0
    assert i == len(vals)


@pytest.mark.parametrize("K,Q", [(8192, 59), (16384, 59), (65536, 61)])
def test_e2m1_least_q_equals_oracle(K, Q):
    """Table tab:moduli prints 59 GEMMs for E2M1 at K = 2^14; at K = 2^16 the
    window needs two more bits of P (eq. ov-crtgen) and the oracle's search
    takes two more GEMMs."""
    p = _plan("E2M1", K)
    pool = forms.Pools("E2M1", K)
    assert p.q == forms.least_q(pool.rank, K)[0] == Q


def test_widened_e2m1_takes_78_gemms():
    """Example ex:widened: at E2M1 and K = 2^14, operands spanning 2^16 more
    keep 53 + 16 bits with 78 GEMMs. The library's frozen widened configuration
    has that count, equals the oracle's least-Q search at beta = 69, and is
    what a plan asking for more bits than the base configuration holds gets;
    without such a request the base configuration (59 GEMMs) serves."""
    p = oz.PlanFP("E2M1", 16384, 69)
    pool = forms.Pools("E2M1", 16384)
    assert p.q == forms.least_q(pool.rank, 16384, beta=69)[0] == 78
    assert oz.PlanFP("E2M1", 16384).q == 59
    assert oz.PlanFP("E2M1", 16384, 60).q == 78          # 60 bits: past the base window, within the widened
    st, _ = oz.oz_plan_create_fp(oz.OZ_FMT_E2M1, 16384, 72)
    assert st == oz.OZ_ERR_K_TOO_LARGE                    # no configuration holds 72 bits at K = 2^14


@pytest.mark.skipif(not SLOW, reason="minutes of CPU; set OZ_SLOW_TESTS=1")
@pytest.mark.parametrize("fmt,Q", [("E2M3", 39), ("E3M2", 52)])
def test_widened_fp6_least_q_equals_oracle(fmt, Q):
    p = oz.PlanFP(fmt, 16384, 69)
    pool = forms.Pools(fmt, 16384)
    assert p.q == forms.least_q(pool.rank, 16384, beta=69)[0] == Q


def test_fp8_counts_match_the_paper():
    """Table tab:moduli / Sec. 'FP8 and FP6': E4M3 and E2M3 take 30 GEMMs at
    K = 2^14, 15 one-limb channels and 5 channels of three GEMMs."""
    for fmt in ("E4M3", "E2M3"):
        p = _plan(fmt, 16384)
        assert p.q == 30
        assert sorted(len(forms.weights(KIND[f], b)) for f, b in zip(p.forms, p.bases)) == [1] * 15 + [3] * 5


def test_plan_refuses_inner_dimension_above_its_configurations():
    """Configurations exist for K_cfg = 2^13, 2^14 and 2^16 (Sec. 'Solving the
    Program': each K re-searched); past 2^16 a float plan is refused."""
    assert oz.PlanFP("E4M3", 20000).k_cfg == 65536
    st, h = oz.oz_plan_create_fp(oz.OZ_FMT_E4M3, 65537, 0)
    assert st == oz.OZ_ERR_K_TOO_LARGE and h is None
    assert oz.oz_plan_create_fp(99, 1000, 0)[0] == oz.OZ_ERR_UNSUPPORTED


def test_blocked_candidates_keep_the_bits():
    """The blocked-call configurations offered for a product keep 53 bits and
    admit its K: the INT8 plan of the least Q (whole K and shorter slabs) and
    each float format whose frozen configuration's window holds, in slabs of
    its accumulation cap; past every float window only INT8 is offered."""
    cands = oz.blocked_candidates(3000, 53, slabs=(1024,))
    labels = [c[0] for c in cands]
    assert labels[0].startswith("int8 q=16") and "int8 q=16 slab=1024" in labels
    assert any(l.startswith("E4M3") for l in labels) and any(l.startswith("E2M1") for l in labels)
    for label, plan, k_slab in cands:
        assert plan.bits == 53 and 3000 <= plan.k_rec and k_slab <= plan.k_acc
    far = oz.blocked_candidates(120000, 53, slabs=(8192,))
    assert [c[0].split()[0] for c in far] == ["int8", "int8"]
