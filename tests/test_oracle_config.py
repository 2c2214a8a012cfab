"""Pins of the oracle's configuration logic (moduli, caps, bit budget) against
numbers the paper prints and against exhaustive search."""
import itertools
import json
import math
import os

import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "int8_config.json")))


def _brute_max_product(Q, m_max, m_min=2):
    best = None
    for combo in itertools.combinations(range(m_min, m_max + 1), Q):
        if all(math.gcd(a, b) == 1 for a, b in itertools.combinations(combo, 2)):
            key = (math.prod(combo), -max(combo))
            if best is None or key > best[0]:
                best = (key, sorted(combo, reverse=True))
    return best[1]


@pytest.mark.parametrize("Q,m_max", [(3, 20), (4, 30), (5, 40), (6, 36), (4, 17)])
def test_dp_matches_exhaustive_search(Q, m_max):
    assert oracle.max_product_moduli(Q, m_max) == _brute_max_product(Q, m_max)


def test_int8_set_reproduces_printed_kmax():
    mods = oracle.max_product_moduli(16, 239)
    assert len(mods) == 16 and len(set(mods)) == 16
    assert all(math.gcd(a, b) == 1 for a, b in itertools.combinations(mods, 2))
    assert max(mods) == GOLD["largest_modulus_ours"]["value"]
    assert max(oracle.radius(m) for m in mods) == GOLD["radius_ours"]["value"]
    k_rec, k_acc, k_max = oracle.caps(mods, beta=53)
    assert k_max == GOLD["k_max_ours"]["value"]
    assert k_acc == GOLD["k_max_ours"]["value"] and k_rec > k_acc   # the accumulation cap sets it
    # the window eq. ov-crt holds at K = 2^14
    assert oracle.modulus_product(mods) > 2**14 * 2**107


def test_kmax_is_largest_at_239_and_256_gives_ozii_int8():
    """Of the sets of sixteen, capping the moduli at 239 gives the largest K_max
    (Sec. 'INT4 and INT8'); at 256 the cap is OzII-INT8's 131 071."""
    best = {}
    for m_max in range(225, 257):
        mods = oracle.max_product_moduli(16, m_max)
        best[m_max] = oracle.caps(mods, beta=53)[2]
    top = max(best.values())
    assert top == GOLD["k_max_ours"]["value"]
    assert min(m for m, v in best.items() if v == top) == 239
    assert best[256] == GOLD["k_max_ozii_int8"]["value"]


def test_rmax_and_counting_bound():
    assert oracle.r_max(1, 2**14) == GOLD["r_max1_int32_k2p14"]["value"]
    assert oracle.r_max(1, 2**14, oracle.FP32_LAMBDA) == GOLD["fp32_rmax1_k2p14"]["value"]
    assert oracle.counting_bound(2**14) == GOLD["counting_bound_int8_k2p14"]["value"]
    assert oracle.INT32_LAMBDA == GOLD["int32_lambda"]["value"]
    assert oracle.FP32_LAMBDA == GOLD["fp32_lambda"]["value"]


def test_least_q_row_of_table():
    g = GOLD["least_q_int8"]
    assert [oracle.least_q(K) for K in g["K"]] == g["Q"]


def test_nested_prefix_list():
    """The max-product sets for Q = 9..20 (moduli <= 239) are prefixes of one list."""
    full = oracle.max_product_moduli(20, 239)
    for Q in range(9, 20):
        assert oracle.max_product_moduli(Q, 239) == full[:Q]


def test_beta_max_definition():
    mods = oracle.max_product_moduli(16, 239)
    P = oracle.modulus_product(mods)
    for K in (256, 1024, 8192, 16384):
        b = oracle.beta_max(mods, K)
        assert 2 * K * (2**b - 1) ** 2 < P <= 2 * K * (2**(b + 1) - 1) ** 2
    assert oracle.beta_max(mods, 8192) == 55
    assert oracle.beta_max(oracle.max_product_moduli(14, 239), 256) == 50
    # kappa_rec at beta = 53 by Q: 14 -> 4, 15 -> 836, 16 -> 159 819
    assert [oracle.caps(oracle.max_product_moduli(q, 239), 53)[0] for q in (14, 15, 16)] == [4, 836, 159819]


def test_kappa_rec_reproduces_the_least_q_row_of_table():
    """eq. caps' reconstruction cap, read against Table tab:moduli's INT8 row:
    at each printed K, with the moduli capped where their radius still meets
    eq. rmax (and at 256), the least Q whose kappa_rec reaches K is the
    printed count (16, 16, 16, 18)."""
    g = GOLD["least_q_int8"]
    got = []
    for K in g["K"]:
        rm = oracle.r_max(1, K)
        top = min(256, 2 * rm + 1)
        while top > 2 and oracle.radius(top) > rm:
            top -= 1
        got.append(next(q for q in range(1, 40) if oracle.caps(oracle.max_product_moduli(q, top), 53)[0] >= K))
    assert got == g["Q"]
