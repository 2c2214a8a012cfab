"""Parity of the CUDA path with the CPU oracle, phase by phase and end to end.

Integer work (shifts, residue planes, W mod m) must match bit for bit; the
FP64 output must match bit for bit too, because both sides round the same
exact integer once (Sec. "Emulation Problem"). All calls go through the C ABI.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts but never run there
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2609_37693_gb300 as oz  # noqa: E402

DEV = torch.device("cuda:0")
ENGINES = [oz.OZ_ENGINE_IMMA, oz.OZ_ENGINE_TC, oz.OZ_ENGINE_TC1]
BF16 = (oz.OZ_ENGINE_TC, oz.OZ_ENGINE_TC1)


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _stream():
    return oz._stream_handle()


def _split(plan, X, contiguous, nvec, length, ld):
    nvec_pad = oz.round_up(max(nvec, 1), 256)
    k_pad = oz.round_up(max(length, 1), 128)
    elem = torch.bfloat16 if plan.engine in BF16 else torch.int8
    planes = torch.full((plan.q, nvec_pad, k_pad), 7, dtype=elem, device=DEV)  # poison: padding must be zeroed
    shifts = torch.zeros(max(nvec, 1), dtype=torch.int32, device=DEV)
    flag = torch.zeros(4, dtype=torch.int32, device=DEV)
    colmax = torch.zeros(max(nvec, 1), dtype=torch.int64, device=DEV)
    st = oz.oz_split(plan.handle, contiguous, nvec, length, X.data_ptr(), ld, nvec_pad, k_pad, shifts.data_ptr(),
                     planes.data_ptr(), flag.data_ptr(), colmax.data_ptr(), _stream())
    assert st == oz.OZ_OK
    torch.cuda.synchronize()
    return shifts.cpu().numpy()[:nvec], planes.float().cpu().numpy().astype(np.int16), flag.cpu().numpy()


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("m,k,phi", [(256, 256, 0.5), (300, 1000, 2.0), (1, 1, 1.0), (777, 129, 4.0)])
def test_split_rows_and_cols_match_oracle(engine, m, k, phi):
    plan = oz.Plan(16, 0, max(k, 1), engine)
    A, _ = synth.phi_pair(m, 1, k, phi, seed=m + k)
    # rows of A (contiguous)
    s, P, flag = _split(plan, _dev(A), 1, m, k, k)
    s_ref = oracle.scale(A, plan.bits, axis=1)
    U_ref = oracle.planes(A, s_ref, plan.moduli, axis=1)
    assert np.array_equal(s, s_ref)
    assert np.array_equal(P[:, :m, :k], U_ref)
    assert not P[:, m:, :].any() and not P[:, :, k:].any()
    assert flag[0] == 0
    # columns of A^T stored k x m (strided)
    At = np.ascontiguousarray(A.T)
    s2, P2, _ = _split(plan, _dev(At), 0, m, k, m)
    assert np.array_equal(s2, s_ref)
    assert np.array_equal(P2[:, :m, :k], U_ref)
    assert not P2[:, m:, :].any() and not P2[:, :, k:].any()


def test_split_special_values():
    plan = oz.Plan(16, 53, 64, oz.OZ_ENGINE_IMMA)
    A = np.array([[0.0] * 8, [1e-310, -3e-320, 5e-324, 0, 0, 0, 0, -2.5e-308], [1e300, -1e-300, 3.0, 0.5, 2**-1000,
                                                                                 -7.0, 1.0, 0.0],
                  [2.0**52, 2.0**53 - 1, -(2.0**52) - 1, 1.0, 0.75, -0.25, 3.5, 1e16]])
    s, P, _ = _split(plan, _dev(A), 1, 4, 8, 8)
    s_ref = oracle.scale(A, 53, axis=1)
    assert np.array_equal(s, s_ref)
    assert np.array_equal(P[:, :4, :8], oracle.planes(A, s_ref, plan.moduli, axis=1))


def test_split_flags_nonfinite():
    plan = oz.Plan(16, 53, 64, oz.OZ_ENGINE_IMMA)
    A = np.ones((3, 5))
    A[1, 2] = np.nan
    _, _, flag = _split(plan, _dev(A), 1, 3, 5, 5)
    assert flag[0] & 1
    A[1, 2] = -np.inf
    _, _, flag = _split(plan, _dev(np.ascontiguousarray(A.T)), 0, 3, 5, 3)
    assert flag[0] & 1


def _plane_dtype(plan):
    return torch.bfloat16 if plan.engine in BF16 else torch.int8


def _residues(plan, A, B):
    """GPU W mod m (raw epilogue) through oz_split + oz_residue_gemm."""
    m, k = A.shape
    n = B.shape[1]
    m_pad, n_pad, k_pad = oz.round_up(m, 256), oz.round_up(n, 256), oz.round_up(k, 128)
    U = torch.zeros((plan.q, m_pad, k_pad), dtype=_plane_dtype(plan), device=DEV)
    V = torch.zeros((plan.q, n_pad, k_pad), dtype=_plane_dtype(plan), device=DEV)
    flag = torch.zeros(4, dtype=torch.int32, device=DEV)
    s = torch.zeros(m, dtype=torch.int32, device=DEV)
    t = torch.zeros(n, dtype=torch.int32, device=DEV)
    cm = torch.zeros(max(m, n), dtype=torch.int64, device=DEV)
    Ad, Bd = _dev(A), _dev(B)
    st = _stream()
    assert oz.oz_split(plan.handle, 1, m, k, Ad.data_ptr(), k, m_pad, k_pad, s.data_ptr(), U.data_ptr(), None,
                       None, st) == oz.OZ_OK
    assert oz.oz_split(plan.handle, 0, n, k, Bd.data_ptr(), n, n_pad, k_pad, t.data_ptr(), V.data_ptr(), None,
                       cm.data_ptr(), st) == oz.OZ_OK
    Y = torch.zeros((plan.q, m, n), dtype=torch.uint8, device=DEV)
    Yd = torch.zeros((plan.q, m, n), dtype=torch.uint8, device=DEV)
    assert oz.oz_residue_gemm(plan.handle, m, n, m_pad, n_pad, k_pad, U.data_ptr(), V.data_ptr(), Y.data_ptr(), 1,
                              flag.data_ptr(), st) == oz.OZ_OK
    assert oz.oz_residue_gemm(plan.handle, m, n, m_pad, n_pad, k_pad, U.data_ptr(), V.data_ptr(), Yd.data_ptr(), 0,
                              flag.data_ptr(), st) == oz.OZ_OK
    C = torch.zeros((m, n), dtype=torch.float64, device=DEV)
    assert oz.oz_reconstruct(plan.handle, m, n, Yd.data_ptr(), s.data_ptr(), t.data_ptr(), C.data_ptr(), n,
                             st) == oz.OZ_OK
    torch.cuda.synchronize()
    assert int(flag[0].item()) == 0
    return Y.cpu().numpy(), Yd.cpu().numpy(), C.cpu().numpy()


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("m,n,k,q,bits", [(256, 256, 256, 14, 50), (300, 200, 1000, 16, 0), (129, 513, 700, 16, 53),
                                          (64, 300, 2048, 20, 0), (200, 520, 3000, 16, 0)])
def test_residue_products_and_reconstruct_match_oracle(engine, m, n, k, q, bits):
    plan = oz.Plan(q, bits, k, engine)
    A, B = synth.phi_pair(m, n, k, 1.0, seed=q + k)
    Y, Yd, C = _residues(plan, A, B)
    C_ref, W_ref, _, _ = oracle.dgemm(A, B, plan.moduli, plan.bits, want_residues=True)
    assert np.array_equal(Y, W_ref)                    # W mod m, bit for bit
    # the CRT digits are (W mod m) (P/m)^-1 mod m
    P = oracle.modulus_product(plan.moduli)
    for qq, mq in enumerate(plan.moduli):
        inv = pow((P // mq) % mq, -1, mq)
        assert np.array_equal(Yd[qq].astype(np.int64), (W_ref[qq].astype(np.int64) * inv) % mq)
    assert np.array_equal(_bits(C), _bits(C_ref))


def _digits(x, moduli):
    P = oracle.modulus_product(moduli)
    return [((x % mq) * pow((P // mq) % mq, -1, mq)) % mq for mq in moduli]


def _from_digits(d, moduli):
    """The integer in [-P/2, P/2) whose CRT digits are d."""
    P = oracle.modulus_product(moduli)
    x = sum(int(dq) * (P // mq) for dq, mq in zip(d, moduli)) % P
    return x - P if x >= P - P // 2 else x


@pytest.mark.parametrize("q", [9, 10, 11, 12, 13, 14, 15, 16, 17, 20])
@pytest.mark.parametrize("pitch4", [True, False])
def test_reconstruct_edge_integers(q, pitch4):
    """Integers at the window's edges, ties of the final rounding, subnormal and
    overflowing results, and digit patterns at the extremes of the CRT sum
    (every digit m_q - 1: the largest sum; every digit 0 but one), fed as CRT
    digits straight to the reconstruct phase. pitch4: a row length that is a
    multiple of 4 (whole digit words, the grouped-moduli kernel for Q <= 16)
    or one that is not (the byte-wise kernel)."""
    plan = oz.Plan(q, 0, 4, oz.OZ_ENGINE_IMMA)
    P = oracle.modulus_product(plan.moduli)
    rng = np.random.default_rng(q)
    xs = [0, 1, -1, P // 2 - 1, -(P // 2), P // 2 - 2**60, -(P // 2) + 3, (2**53 + 1) << 10, -((2**54 + 2) << 40),
          3 << 70, (2**53 + 1), -(2**53 + 3)]
    xs += [int(v) for v in rng.integers(-2**62, 2**62, size=20)]
    xs += [int(rng.integers(1, 2**62)) << int(rng.integers(0, 60)) for _ in range(20)]
    xs += [_from_digits([mq - 1 for mq in plan.moduli], plan.moduli)]
    for r in range(q):
        xs.append(_from_digits([mq - 1 if i == r else 0 for i, mq in enumerate(plan.moduli)], plan.moduli))
    xs += [_from_digits([int(rng.integers(0, mq)) for mq in plan.moduli], plan.moduli) for _ in range(24)]
    xs = [x for x in xs if -(P // 2) <= x < P // 2]
    while (len(xs) % 4 == 0) != pitch4:
        xs.append(int(rng.integers(-2**40, 2**40)))
    exps = [0, -1, 5, -1074, -1100, -1200, 1000, 900, 1023, -1022, -30, 60, -120, -140]
    n = len(xs)
    m = len(exps)
    # C[i][j] = X_j * 2^-(s_i + t_j): take t = 0, s_i = -exps[i]
    Ydig = np.zeros((plan.q, m, n), dtype=np.uint8)
    for j, x in enumerate(xs):
        d = _digits(x, plan.moduli)
        for qq in range(plan.q):
            Ydig[qq, :, j] = d[qq]
    s = np.array([-e for e in exps], dtype=np.int32)
    t = np.zeros(n, dtype=np.int32)
    C = torch.zeros((m, n), dtype=torch.float64, device=DEV)
    Yt, st_, tt = _dev(Ydig), _dev(s), _dev(t)
    assert oz.oz_reconstruct(plan.handle, m, n, Yt.data_ptr(), st_.data_ptr(), tt.data_ptr(), C.data_ptr(), n,
                             _stream()) == oz.OZ_OK
    torch.cuda.synchronize()
    ref = np.array([oracle.round_scaled(xs, [e] * n) for e in exps])
    assert np.array_equal(_bits(C.cpu().numpy()), _bits(ref))


def _dgemm(plan, A, B, trans_a=False, trans_b=False):
    Ad, Bd = _dev(A), _dev(B)
    C = oz.dgemm(Ad, Bd, plan, trans_a=trans_a, trans_b=trans_b)
    torch.cuda.synchronize()
    return C.cpu().numpy()


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("m,n,k,q,bits,phi", [(256, 256, 256, 14, 50, 0.5), (1000, 777, 300, 16, 53, 1.0),
                                              (300, 1000, 4096, 16, 0, 2.0), (33, 17, 5000, 16, 0, 4.0),
                                              (1, 1, 1, 16, 53, 1.0), (513, 129, 1, 9, 0, 1.0)])
def test_dgemm_matches_oracle(engine, m, n, k, q, bits, phi):
    plan = oz.Plan(q, bits, k, engine)
    A, B = synth.phi_pair(m, n, k, phi, seed=m * 7 + k)
    C = _dgemm(plan, A, B)
    C_ref = oracle.dgemm(A, B, plan.moduli, plan.bits)
    assert np.array_equal(_bits(C), _bits(C_ref))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("ta,tb", [(0, 1), (1, 0), (1, 1)])
def test_dgemm_transposed_operands(engine, ta, tb):
    m, n, k = 200, 300, 500
    plan = oz.Plan(16, 0, k, engine)
    A, B = synth.phi_pair(m, n, k, 1.0, seed=3)
    C_ref = oracle.dgemm(A, B, plan.moduli, plan.bits)
    Ain = np.ascontiguousarray(A.T) if ta else A
    Bin = np.ascontiguousarray(B.T) if tb else B
    C = _dgemm(plan, Ain, Bin, bool(ta), bool(tb))
    assert np.array_equal(_bits(C), _bits(C_ref))


@pytest.mark.parametrize("engine", ENGINES)
def test_dgemm_special_operands(engine):
    plan = oz.Plan(16, 53, 64, engine)
    A, B = synth.phi_pair(40, 30, 64, 1.0, seed=11)
    A[3, :] = 0.0
    B[:, 7] = 0.0
    A[5, :] *= 1e-300
    B[:, 9] *= 1e-20
    A[6, :] *= 1e200
    B[:, 11] *= 1e150                       # row 6 x column 11 overflows to +-inf
    A[8, 3] = 2.0**-1074
    C = _dgemm(plan, A, B)
    C_ref = oracle.dgemm(A, B, plan.moduli, 53)
    assert np.isinf(C_ref[6, 11])
    assert np.array_equal(_bits(C), _bits(C_ref))


def test_dgemm_lossless_is_fl_of_exact():
    """Integer operands convert losslessly, so C = fl(AB) (Sec. 'Emulation Problem')."""
    rng = np.random.default_rng(2)
    A = rng.integers(-2**20, 2**20, size=(64, 200)).astype(np.float64)
    B = rng.integers(-2**20, 2**20, size=(200, 48)).astype(np.float64)
    plan = oz.Plan(16, 53, 200, oz.OZ_ENGINE_IMMA)
    C = _dgemm(plan, A, B)
    Ai = A.astype(object)
    Bi = B.astype(object)
    exact = Ai.dot(Bi)
    ref = np.array([[float(v) for v in row] for row in exact])   # int -> float rounds to nearest even
    assert np.array_equal(_bits(C), _bits(ref))


def test_dgemm_k_zero_and_empty():
    plan = oz.Plan(16, 0, 16, oz.OZ_ENGINE_IMMA)
    A = torch.zeros((5, 0), dtype=torch.float64, device=DEV)
    B = torch.zeros((0, 3), dtype=torch.float64, device=DEV)
    C = torch.full((5, 3), 9.0, dtype=torch.float64, device=DEV)
    oz.dgemm(A, B, plan, out=C)
    torch.cuda.synchronize()
    assert torch.all(C == 0)
    E = oz.dgemm(torch.zeros((0, 4), dtype=torch.float64, device=DEV),
                 torch.zeros((4, 3), dtype=torch.float64, device=DEV), plan)
    assert E.shape == (0, 3)


def test_dgemm_reports_nonfinite():
    plan = oz.Plan(16, 0, 64, oz.OZ_ENGINE_IMMA)
    A, B = synth.phi_pair(20, 20, 64, 1.0, seed=1)
    A[4, 5] = np.nan
    Ad, Bd = _dev(A), _dev(B)
    ws = oz.workspace(plan, 20, 20, 64)
    oz.dgemm(Ad, Bd, plan, ws=ws)
    assert oz.query_status(ws) == oz.OZ_ERR_NONFINITE
    A[4, 5] = 1.0
    oz.dgemm(_dev(A), Bd, plan, ws=ws)
    assert oz.query_status(ws) == oz.OZ_OK


@pytest.mark.parametrize("m,n,k", [(2000, 17, 1100), (33, 1000, 5000), (300, 300, 1025), (257, 129, 2048)])
def test_dgemm_default_engine_long_rows(m, n, k):
    """Products on the default engine with k past one slab (A's rows split one
    block per row, B's columns split in place after their column maxima):
    many rows and few columns, the reverse, k just past 1024; zero, tiny and
    subnormal entries on both sides; bit for bit the oracle's product."""
    plan = oz.Plan(16, 0, k, oz.OZ_ENGINE_TC)
    A, B = synth.phi_pair(m, n, k, 1.5, seed=m + n + k)
    A[1, :] = 0.0
    B[:, min(3, n - 1)] = 0.0
    A[2, :] *= 1e-300
    B[:, n - 1] *= 1e-20
    A[m - 1, k - 1] = 2.0**-1074
    C = _dgemm(plan, A, B)
    C_ref = oracle.dgemm(A, B, plan.moduli, plan.bits)
    assert np.array_equal(_bits(C), _bits(C_ref))


@pytest.mark.parametrize("side", ["A", "B"])
def test_dgemm_reports_nonfinite_on_the_default_engine(side):
    """A non-finite entry of A (found by the row split's maximum) or of B (by
    the column maxima) sets the workspace status; the next clean call clears it."""
    m, n, k = 64, 96, 1500
    plan = oz.Plan(16, 0, k, oz.OZ_ENGINE_TC)
    A, B = synth.phi_pair(m, n, k, 1.0, seed=5)
    if side == "A":
        A[7, 1400] = np.inf
    else:
        B[1499, 90] = np.nan
    ws = oz.workspace(plan, m, n, k)
    oz.dgemm(_dev(A), _dev(B), plan, ws=ws)
    assert oz.query_status(ws) == oz.OZ_ERR_NONFINITE
    A, B = synth.phi_pair(m, n, k, 1.0, seed=5)
    oz.dgemm(_dev(A), _dev(B), plan, ws=ws)
    assert oz.query_status(ws) == oz.OZ_OK


@pytest.mark.parametrize("engine", ENGINES)
def test_full_size_8192_sampled_entries_and_error(engine):
    """m = n = k = 8192, Q = 16 (the headline size): sampled entries equal the
    oracle's bit for bit, and the error against the exact product is within
    2u (|A||B|)_ij at phi = 0.5."""
    n = 8192
    plan = oz.Plan(16, 0, n, engine)
    assert plan.bits == 55
    A, B = synth.phi_pair(n, n, n, 0.5, seed=0)
    C = _dgemm(plan, A, B)
    rows, cols = synth.sample_entries(n, n, 2048, seed=5)
    ref = oracle.dgemm_entries(A, B, plan.moduli, plan.bits, rows, cols)
    assert np.array_equal(_bits(C[rows, cols]), _bits(ref))
    err, ab = oracle.exact_error(A, B, C, rows, cols)
    assert np.max(err / (2.0**-53 * ab)) <= 2.0


@pytest.mark.parametrize("engine", BF16)
@pytest.mark.parametrize("pattern", ["all_max", "random_sign", "mixed"])
def test_tc_fp32_accumulation_is_exact(pattern, engine):
    """The FP32 accumulators of tcgen05.mma must add integer products without
    rounding while every partial sum stays within 2^24 (Sec. 'Exactness May
    Rely on Undocumented Accumulation'). Planes at the largest residue
    magnitude drive each 1024-term slab to 1024 * 119^2 = 14 500 864; the
    residues of the product must equal those of the exact integer product."""
    plan = oz.Plan(16, 0, 4096, engine)
    m, n, k = 256, 256, 4096
    rng = np.random.default_rng(17)
    if pattern == "all_max":
        Ui = np.full((m, k), 119, dtype=np.int64)
        Vi = np.where(np.arange(n)[:, None] % 2 == 0, 119, -119) * np.ones((n, k), dtype=np.int64)
    elif pattern == "random_sign":
        Ui = rng.choice([-119, 119], size=(m, k)).astype(np.int64)
        Vi = rng.choice([-119, 119], size=(n, k)).astype(np.int64)
    else:
        Ui = rng.integers(-119, 120, size=(m, k)).astype(np.int64)
        Ui[: m // 2] = 119
        Vi = rng.integers(-119, 120, size=(n, k)).astype(np.int64)
        Vi[: n // 2] = 119
    W = Ui @ Vi.T
    U = torch.zeros((plan.q, m, k), dtype=torch.bfloat16, device=DEV)
    V = torch.zeros((plan.q, n, k), dtype=torch.bfloat16, device=DEV)
    U[:] = torch.from_numpy(Ui.astype(np.float32)).to(DEV).to(torch.bfloat16)
    V[:] = torch.from_numpy(Vi.astype(np.float32)).to(DEV).to(torch.bfloat16)
    Y = torch.zeros((plan.q, m, n), dtype=torch.uint8, device=DEV)
    flag = torch.zeros(4, dtype=torch.int32, device=DEV)
    assert oz.oz_residue_gemm(plan.handle, m, n, m, n, k, U.data_ptr(), V.data_ptr(), Y.data_ptr(), 1,
                              flag.data_ptr(), _stream()) == oz.OZ_OK
    torch.cuda.synchronize()
    assert int(flag[0].item()) == 0
    Yh = Y.cpu().numpy()
    for q, mq in enumerate(plan.moduli):
        assert np.array_equal(Yh[q].astype(np.int64), W % mq), f"modulus {mq}"


@pytest.mark.parametrize("engine", [oz.OZ_ENGINE_IMMA, oz.OZ_ENGINE_TC])
def test_widened_split_matches_oracle(engine):
    """beta = 70 > 64 (Sec. 'Not True Emulation of DGEMM'): |a'| < 2^70 is cut
    into seven 12-bit pieces; shifts and planes equal the oracle's."""
    plan = oz.Plan(20, 70, 300, engine)
    assert plan.bits == 70
    A, _ = synth.phi_pair(300, 1, 1300, 2.0, seed=70)
    s, P, flag = _split(plan, _dev(A), 1, 300, 1300, 1300)
    s_ref = oracle.scale(A, 70, axis=1)
    U_ref = oracle.planes(A, s_ref, plan.moduli, axis=1)
    assert np.array_equal(s, s_ref)
    assert np.array_equal(P[:, :300, :1300], U_ref)
    At = np.ascontiguousarray(A.T)
    s2, P2, _ = _split(plan, _dev(At), 0, 300, 1300, 300)
    assert np.array_equal(s2, s_ref) and np.array_equal(P2[:, :300, :1300], U_ref)
    B, _ = synth.phi_pair(77, 1, 500, 1.0, seed=71)        # short rows: the warp-per-row split
    s3, P3, _ = _split(plan, _dev(B), 1, 77, 500, 500)
    assert np.array_equal(P3[:, :77, :500], oracle.planes(B, oracle.scale(B, 70, axis=1), plan.moduli, axis=1))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("m,n,k,bits,ta,tb", [(300, 200, 600, 70, 0, 0), (129, 257, 1500, 66, 1, 0),
                                              (33, 17, 129, 72, 0, 1)])
def test_widened_dgemm_matches_oracle(engine, m, n, k, bits, ta, tb):
    plan = oz.Plan(20, bits, k, engine)
    A, B = synth.phi_pair(m, n, k, 2.0, seed=m + bits)
    Ad = _dev(A.T if ta else A)
    Bd = _dev(B.T if tb else B)
    C = oz.dgemm(Ad, Bd, plan, trans_a=bool(ta), trans_b=bool(tb))
    torch.cuda.synchronize()
    assert np.array_equal(_bits(C.cpu().numpy()), _bits(oracle.dgemm(A, B, plan.moduli, bits)))


def test_widened_product_is_fl_of_exact():
    """Rows of A and columns of B spanning at most 2^16 (full 53-bit
    significands): at beta = 69 the product is fl(AB), bit for bit against
    exact rational arithmetic (Example widened)."""
    from tests import brute
    from tests.test_oracle_pins import _spanned
    rng = np.random.default_rng(69)
    M, N, K = 6, 5, 40
    A = _spanned(rng, M, K, 16, axis=1)
    B = _spanned(rng, N, K, 16, axis=0)
    plan = oz.Plan(20, 69, K, oz.OZ_ENGINE_TC)
    C = _dgemm(plan, A, B)
    exact = brute.exact_product(A, B)
    ref = np.array([[brute.to_float(exact[i][j]) for j in range(N)] for i in range(M)])
    assert np.array_equal(_bits(C), _bits(ref))


@pytest.mark.parametrize("rows,cols,ld", [(1, 1, 1), (33, 65, 65), (1000, 777, 800), (4096, 129, 129)])
def test_transpose_phase_is_exact(rows, cols, ld):
    """oz_transpose (the step oz_dgemm takes before splitting B's columns as
    rows) moves every double unchanged, ragged tiles and row pitch included."""
    X = np.random.default_rng(rows).standard_normal((rows, ld))
    Xd = _dev(X)
    Y = torch.full((cols, rows), np.nan, dtype=torch.float64, device=DEV)
    assert oz.oz_transpose(rows, cols, Xd.data_ptr(), ld, Y.data_ptr(), _stream()) == oz.OZ_OK
    torch.cuda.synchronize()
    assert np.array_equal(_bits(Y.cpu().numpy()), _bits(X[:, :cols].T))
