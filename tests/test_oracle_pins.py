"""Pins of the C oracle's arithmetic against exact brute force, closed forms and
invariants (no GPU)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests import brute

MODS16 = oracle.max_product_moduli(16, 239)
MODS14 = oracle.max_product_moduli(14, 239)
# 26 pairwise-coprime moduli, P about 2^154.5: the channel moduli of the widened
# E2M1 configuration (Example ex:widened, beta = 53 + 16 at K = 2^14)
MODS26 = [169, 157, 151, 149, 139, 137, 131, 127, 113, 89, 85, 83, 79, 73, 71, 67, 61, 59, 53, 47, 43, 41, 11, 9,
          8, 7]


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


@pytest.mark.parametrize("seed,phi,beta,mods", [(0, 0.5, 53, MODS16), (1, 2.0, 55, MODS16), (2, 1.0, 50, MODS14),
                                                (3, 4.0, 53, MODS16), (4, 4.0, 69, MODS26), (5, 1.0, 71, MODS26)])
def test_oracle_equals_exact_definition(seed, phi, beta, mods):
    """C, X = A'B' and every W mod m equal the exact big-integer evaluation of
    eq. convert and C = fl(mu^-1 A'B' nu^-1)."""
    M, N, K = 5, 4, 7
    A, B = synth.phi_pair(M, N, K, phi, seed)
    C_ref, X_ref, s_ref, t_ref = brute.emulated(A, B, beta)
    C, W, s, t = oracle.dgemm(A, B, mods, beta, want_residues=True)
    assert list(s) == s_ref and list(t) == t_ref
    assert np.array_equal(_bits(C), _bits(C_ref))
    for k, m in enumerate(mods):
        assert all(int(W[k, i, j]) == X_ref[i][j] % m for i in range(M) for j in range(N))
    rows, cols = np.divmod(np.arange(M * N), N)
    Ce, Xe = oracle.dgemm_entries(A, B, mods, beta, rows, cols, want_x=True)
    assert np.array_equal(_bits(Ce), _bits(C.ravel()))
    assert Xe == [X_ref[i][j] for i, j in zip(rows, cols)]


def test_planes_are_balanced_residues_of_truncation():
    A, _ = synth.phi_pair(6, 1, 9, 1.0, 5)
    s = oracle.scale(A, 53, axis=1)
    U = oracle.planes(A, s, MODS16, axis=1)
    for i in range(6):
        assert s[i] == brute.shift(A[i], 53)
        for h in range(9):
            a = brute.trunc_scaled(A[i, h], s[i])
            assert abs(a) < 2**53
            for k, m in enumerate(MODS16):
                r = int(U[k, i, h])
                assert r == brute.balanced(a, m)
                assert -(m // 2) <= r <= (m + 1) // 2 - 1
    # ties of the even modulus (236) go to -m/2: the representative nearest
    # zero (Sec. "Ozaki II") taken in [-m/2, m/2 - 1], which is two's
    # complement at m = 256; a row maximum of 2^52 gives shift 0 at
    # beta = 53, so these integers are their own truncations
    row = np.array([[2.0**52, 118.0, -118.0, 354.0, -354.0, 117.0, -117.0]])
    assert list(oracle.scale(row, 53, axis=1)) == [0]
    U6 = oracle.planes(row, np.zeros(1, dtype=np.int32), MODS16, axis=1)
    k236 = list(MODS16).index(236)
    assert [int(v) for v in U6[k236, 0, 1:]] == [-118, -118, -118, -118, 117, -117]
    # B side: column shifts and the transposed planes
    _, B = synth.phi_pair(1, 5, 8, 1.0, 6)
    t = oracle.scale(B, 53, axis=0)
    V = oracle.planes(B, t, MODS16, axis=0)
    assert V.shape == (16, 5, 8)
    for j in range(5):
        assert t[j] == brute.shift(B[:, j], 53)
        for h in range(8):
            assert int(V[3, j, h]) == brute.balanced(brute.trunc_scaled(B[h, j], t[j]), MODS16[3])


def test_lossless_conversion_returns_fl_of_exact_product():
    """Sec. 'Emulation Problem': the result is fl(AB) when the conversion is
    lossless. Integer operands below 2^20 convert losslessly at beta = 53."""
    rng = np.random.default_rng(7)
    for K in (1, 3, 16, 40):
        A = rng.integers(-2**20, 2**20, size=(4, K)).astype(np.float64)
        B = rng.integers(-2**20, 2**20, size=(K, 3)).astype(np.float64)
        # scale rows by powers of two: still lossless
        A *= np.ldexp(1.0, rng.integers(-30, 30, size=4))[:, None]
        C = oracle.dgemm(A, B, MODS16, 53)
        exact = brute.exact_product(A, B)
        ref = np.array([[brute.to_float(exact[i][j]) for j in range(3)] for i in range(4)])
        assert np.array_equal(_bits(C), _bits(ref))


def test_lossless_53bit_operands_exercise_rounding():
    """53-bit integer operands: A'B' needs up to 112 bits, so the final rounding
    (ties to even included) decides the result."""
    rng = np.random.default_rng(11)
    A = rng.integers(2**52, 2**53, size=(3, 24)).astype(np.float64) * rng.choice([-1.0, 1.0], size=(3, 24))
    B = rng.integers(2**52, 2**53, size=(24, 3)).astype(np.float64) * rng.choice([-1.0, 1.0], size=(24, 3))
    C = oracle.dgemm(A, B, MODS16, 53)
    exact = brute.exact_product(A, B)
    ref = np.array([[brute.to_float(exact[i][j]) for j in range(3)] for i in range(3)])
    assert np.array_equal(_bits(C), _bits(ref))


def test_k1_is_the_plain_product():
    """K = 1: the one entry of each row and column is its maximum, so conversion
    is exact and C_ij = fl(a_i b_j), the binary64 product."""
    rng = np.random.default_rng(3)
    a = (rng.standard_normal((17, 1)) * np.ldexp(1.0, rng.integers(-300, 300, size=(17, 1))))
    b = (rng.standard_normal((1, 13)) * np.ldexp(1.0, rng.integers(-300, 300, size=(1, 13))))
    C = oracle.dgemm(a, b, MODS16, 53)
    assert np.array_equal(_bits(C), _bits(a * b))


def test_invariants_scaling_sign_transpose():
    A, B = synth.phi_pair(9, 7, 33, 1.0, 4)
    C = oracle.dgemm(A, B, MODS16, 53)
    # a power-of-two row scaling scales the row of C exactly
    D = np.ldexp(1.0, np.arange(-4, 5))[:, None]
    C2 = oracle.dgemm(A * D, B, MODS16, 53)
    assert np.array_equal(_bits(C2), _bits(C * D))
    # sign
    assert np.array_equal(_bits(oracle.dgemm(-A, B, MODS16, 53)), _bits(-C))
    # transpose: C(B^T, A^T) = C(A, B)^T
    Ct = oracle.dgemm(np.ascontiguousarray(B.T), np.ascontiguousarray(A.T), MODS16, 53)
    assert np.array_equal(_bits(Ct), _bits(np.ascontiguousarray(C.T)))


def test_crt_invariants_and_window():
    rng = np.random.default_rng(5)
    P = oracle.modulus_product(MODS16)
    w = np.stack([rng.integers(0, m, size=200) for m in MODS16], axis=1)
    xs = oracle.crt(w, MODS16)
    for x, row in zip(xs, w):
        assert -P // 2 <= x < (P + 1) // 2 and 2 * x < P and 2 * x >= -P
        assert all(x % m == int(r) for m, r in zip(MODS16, row))
    # an integer inside the window comes back unchanged
    for x in [0, 1, -1, 2**120, -(2**120) + 12345, P // 2 - 1, -(P // 2)]:
        back = oracle.crt(np.array([[x % m for m in MODS16]]), MODS16)[0]
        assert back == x


def test_garner_agrees_with_the_digit_sum():
    """The oracle's CRT (Garner's mixed radix) and the form the GPU
    reconstruct evaluates, X = sum_k y_k M_k mod P with M_k = P / m_k and the
    digit y_k = (w_k (M_k^-1 mod m_k)) mod m_k, taken to [-P/2, P/2), agree on
    random residues for every Q, in Python integers."""
    rng = np.random.default_rng(17)
    for q in (9, 12, 14, 16, 18, 20):
        mods = oracle.max_product_moduli(q, 239)
        P = oracle.modulus_product(mods)
        w = np.stack([rng.integers(0, m, size=64) for m in mods], axis=1)
        xs = oracle.crt(w, mods)
        for x, row in zip(xs, w):
            acc = 0
            for m, r in zip(mods, row):
                M = P // m
                acc += (int(r) * pow(M, -1, m) % m) * M
            acc %= P
            if 2 * acc >= P:
                acc -= P
            assert acc == x


def test_x_is_bounded_and_exact():
    """|X| <= K (2^beta - 1)^2 (eq. range), and X equals A'B' (eq. convert)."""
    A, B = synth.phi_pair(4, 4, 50, 2.0, 9)
    for beta in (50, 53, 55):
        _, X, _, _ = brute.emulated(A, B, beta)
        rows, cols = np.divmod(np.arange(16), 4)
        _, Xe = oracle.dgemm_entries(A, B, MODS16, beta, rows, cols, want_x=True)
        assert Xe == [X[i][j] for i, j in zip(rows, cols)]
        assert max(abs(x) for x in Xe) <= 50 * (2**beta - 1) ** 2


def test_rounding_against_exact_rationals():
    rng = np.random.default_rng(21)
    xs, es = [], []
    for _ in range(400):
        L = int(rng.integers(1, 200))
        x = int(rng.integers(0, 2**62)) << max(0, L - 62) if L > 62 else int(rng.integers(0, 2**L))
        x = -x if rng.random() < 0.5 else x
        e = int(rng.integers(-1300, 1100)) - L // 2
        xs.append(x)
        es.append(e)
    # exact ties at 53 bits, subnormal ties, overflow and underflow edges
    for sgn in (1, -1):
        xs += [sgn * ((2**53 + 1) << 3), sgn * ((2**53 + 3) << 7), sgn * 3, sgn * 5, sgn * (2**54 - 1), sgn * 1]
        es += [-3, -7, -1075, -1075, 970, -1075]
        xs += [sgn * (2**53 - 1), sgn * (2**60)]
        es += [971, -1200]
        # subnormal results of 55-58-bit integers where rounding to 53 bits
        # first and then to the subnormal grid gives another answer: the
        # rounding must be a single one
        xs += [sgn * 62551616293623058, sgn * 41442468988376657, sgn * 71048548309309803,
               sgn * 263350308324904376]
        es += [-1079, -1079, -1078, -1081]
    out = oracle.round_scaled(xs, es)
    ref = [brute.to_float(Fraction(x) * Fraction(2) ** e) for x, e in zip(xs, es)]
    assert np.array_equal(_bits(out), _bits(np.array(ref)))


def test_subnormal_and_huge_operands_match_definition():
    A = np.array([[1e-310, -3e-320, 2.5e-308], [1e300, -7e299, 3.3e298]])
    B = np.array([[4e-10, 1e10], [-2e-9, 3e9], [1e-12, -5e11]])
    C = oracle.dgemm(A, B, MODS16, 53)
    C_ref, _, _, _ = brute.emulated(A, B, 53)
    assert np.array_equal(_bits(C), _bits(C_ref))
    # overflow to inf
    A2 = np.array([[1e300, 1e300]])
    B2 = np.array([[1e300], [1e300]])
    C2 = oracle.dgemm(A2, B2, MODS16, 53)
    assert math.isinf(C2[0, 0]) and C2[0, 0] > 0


def test_zero_rows_and_columns():
    A, B = synth.phi_pair(5, 6, 11, 1.0, 2)
    A[2, :] = 0.0
    B[:, 4] = 0.0
    C, _, s_o, t_o = oracle.dgemm(A, B, MODS16, 53, want_residues=True)
    assert np.all(_bits(C[2, :]) == 0) and np.all(_bits(C[:, 4]) == 0)
    C_ref, _, s, t = brute.emulated(A, B, 53)
    assert s[2] == 0 and t[4] == 0                  # eq. convert: mu = 1 for a zero row
    assert list(s_o) == list(s) and list(t_o) == list(t)
    assert np.array_equal(_bits(C), _bits(C_ref))


def test_nonfinite_input_is_refused():
    A = np.ones((2, 2))
    A[1, 0] = np.nan
    with pytest.raises(ValueError):
        oracle.dgemm(A, np.ones((2, 2)), MODS16, 53)
    A[1, 0] = np.inf
    with pytest.raises(ValueError):
        oracle.dgemm(A, np.ones((2, 2)), MODS16, 53)


def test_exact_error_matches_fractions():
    A, B = synth.phi_pair(4, 3, 12, 2.0, 8)
    C = A @ B
    rows, cols = np.divmod(np.arange(12), 3)
    err, ab = oracle.exact_error(A, B, C, rows, cols)
    exact = brute.exact_product(A, B)
    for e, i, j in zip(err, rows, cols):
        assert e == brute.to_float(abs(Fraction(float(C[i, j])) - exact[i][j]))
    mag, _ = oracle.exact_error(A, B, None, rows, cols)
    for e, i, j in zip(mag, rows, cols):
        assert e == brute.to_float(abs(exact[i][j]))


@pytest.mark.parametrize("beta", [50, 53, 55])
def test_truncation_error_bound(beta):
    """Sec. 'May Be Less Accurate Than Native on Skewed Rows': truncation changes
    each entry by less than 2u times the largest in its row or column, so
    |C - AB| <= 2^(1-beta) (a_i^max sum|b_hj| + b_j^max sum|a_ih|) + second order
    + the final rounding u|C_ij|."""
    M, N, K = 16, 16, 64
    A, B = synth.phi_pair(M, N, K, 2.0, beta)
    mods = MODS16
    C = oracle.dgemm(A, B, mods, beta)
    rows, cols = np.divmod(np.arange(M * N), N)
    err, _ = oracle.exact_error(A, B, C, rows, cols)
    amax = np.abs(A).max(axis=1)
    bmax = np.abs(B).max(axis=0)
    sa = np.abs(A).sum(axis=1)
    sb = np.abs(B).sum(axis=0)
    for e, i, j in zip(err, rows, cols):
        bound = 2.0**(1 - beta) * (amax[i] * sb[j] + bmax[j] * sa[i]) + K * 2.0**(2 - 2 * beta) * amax[i] * bmax[j]
        bound += 2.0**-53 * abs(C[i, j])
        assert e <= bound * (1 + 1e-12)


def _spanned(rng, vecs, length, d, axis):
    """Entries with full 53-bit significands whose magnitudes, along each vector
    (row for axis=1, column for axis=0), lie within a factor 2^(d+1) of the
    vector's largest (exponent offsets 0..-d, offset 0 present in every vector)."""
    shape = (vecs, length) if axis == 1 else (length, vecs)
    sig = rng.integers(2**52, 2**53, size=shape).astype(np.float64) * rng.choice([-1.0, 1.0], size=shape)
    off = rng.integers(-d, 1, size=shape)
    if axis == 1:
        off[:, 0] = 0
        base = rng.integers(-40, 40, size=(vecs, 1))
    else:
        off[0, :] = 0
        base = rng.integers(-40, 40, size=(1, vecs))
    return np.ldexp(sig, (off + base - 52).astype(np.int64))


@pytest.mark.parametrize("d", [8, 16])
def test_widened_conversion_is_exact_emulation(d):
    """Sec. 'Not True Emulation of DGEMM' and Example widened: when the entries
    of every row of A and column of B lie within 2^d of its largest, keeping
    53 + d bits converts them without loss, so the product is fl(AB), the
    correctly rounded exact product; at 53 bits it is not."""
    rng = np.random.default_rng(100 + d)
    M, N, K = 4, 3, 24
    A = _spanned(rng, M, K, d, axis=1)
    B = _spanned(rng, N, K, d, axis=0)
    mods = oracle.max_product_moduli(20, 239)
    assert oracle.modulus_product(mods) > 2 * K * (2**(53 + d) - 1) ** 2
    exact = brute.exact_product(A, B)
    ref = np.array([[brute.to_float(exact[i][j]) for j in range(N)] for i in range(M)])
    C = oracle.dgemm(A, B, mods, 53 + d)
    assert np.array_equal(_bits(C), _bits(ref))
    C53 = oracle.dgemm(A, B, mods, 53)
    assert not np.array_equal(_bits(C53), _bits(ref))
    # and the oracle's arithmetic at that budget is the exact definition
    C_def, _, _, _ = brute.emulated(A, B, 53 + d)
    assert np.array_equal(_bits(C), _bits(C_def))


def test_sampled_rows_and_columns_give_the_same_entries():
    """Entry (i, j) depends only on row i of A and column j of B, their
    shifts included (eq. convert), so the product of sampled rows and columns
    equals those entries of the whole product. The error report on large
    sizes samples this way."""
    A, B = synth.row_scaled_pair(96, seed=3, m=80, k=130)
    rows = np.array([0, 7, 41, 79])
    cols = np.array([2, 3, 50, 95])
    C_sub = oracle.dgemm(np.ascontiguousarray(A[rows]), np.ascontiguousarray(B[:, cols]), MODS16, 53)
    r, c = np.meshgrid(rows, cols, indexing="ij")
    C_ent = oracle.dgemm_entries(A, B, MODS16, 53, r.ravel(), c.ravel())
    assert np.array_equal(_bits(C_sub.ravel()), _bits(C_ent))
    C_full = oracle.dgemm(A, B, MODS16, 53)
    assert np.array_equal(_bits(C_sub), _bits(C_full[np.ix_(rows, cols)]))


def test_error_report_helper_on_a_small_case():
    """The sampled-grid error of oracle/precision.py against entries computed
    one by one: the same values, and within 2u at the widest beta."""
    from oracle import precision as precision_oracle
    A, B = synth.phi_pair(200, 150, 300, 0.5, seed=4)
    rows, cols = np.array([0, 5, 199]), np.array([1, 149])
    beta = oracle.beta_max(MODS16, 300)
    rel = precision_oracle.errors(A, B, MODS16, beta, rows, cols)
    r, c = np.meshgrid(rows, cols, indexing="ij")
    C = np.zeros((200, 150))
    C[r.ravel(), c.ravel()] = oracle.dgemm_entries(A, B, MODS16, beta, r.ravel(), c.ravel())
    err, ab = oracle.exact_error(A, B, C, r.ravel(), c.ravel())
    assert np.array_equal(rel, err / (2.0**-53 * ab))
    assert rel.max() <= 2.0


def test_moduli_beyond_the_256_bit_crt_are_refused():
    """The oracle's CRT works in 256 bits: 33 moduli, or moduli whose product
    could reach 2^254, are refused rather than wrapped."""
    assert math.gcd(*MODS26) == 1 and all(math.gcd(a, b) == 1 for i, a in enumerate(MODS26) for b in MODS26[:i])
    A, B = synth.phi_pair(2, 2, 3, 1.0, 0)
    with pytest.raises(Exception):
        oracle.dgemm(A, B, list(range(3, 69, 2)), 53)          # 33 moduli
    big = [4093, 4091, 4079, 4073, 4057, 4051, 4049, 4027, 4021, 4019, 4013, 4007, 4003, 4001, 3989, 3967, 3947,
           3943, 3931, 3929, 3919, 3917]                      # 22 primes near 2^12: 264 bits of moduli
    with pytest.raises(Exception):
        oracle.dgemm(A, B, big, 53)
