"""Parity of the float-format path with the CPU oracle: codes written by the
split, residues W mod m after each channel's GEMMs and fold (order R>C), and
the FP64 result, for E4M3, E5M2, E2M3, E3M2 and E2M1 configurations.

The result does not depend on the alphabet: every configuration reaches the
exact product A'B' of the truncated operands within the window (eq.
ov-crtgen), so C must equal the oracle's C at the plan's beta bit for bit
(Sec. "Emulation Problem"). All calls go through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from oracle import forms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts but never run there
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2609_37693_gb300 as oz  # noqa: E402

DEV = torch.device("cuda:0")
FORMATS = ["E4M3", "E5M2", "E2M3", "E3M2", "E2M1"]
KIND = {1: "one", 2: "school3", 3: "toom", 4: "school4"}
CODE_BITS = {"E4M3": 8, "E5M2": 8, "E2M3": 6, "E3M2": 6, "E2M1": 4}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _expected_values(plan, fmt, X, axis):
    """[plane][vec][len] scaled alphabet values the split must write, from the
    oracle's shifts and residues and its form tables."""
    sh = oracle.scale(X, plan.bits, axis)
    res = oracle.planes(X, sh, plan.moduli, axis).astype(np.int64)
    out = []
    for c, (m, f, b) in enumerate(zip(plan.moduli, plan.forms, plan.bases)):
        for tab in forms.tables(fmt, plan.k_cfg, m, KIND[f], b):
            out.append(np.asarray(tab, dtype=np.int64)[res[c] % m])
    return sh, np.stack(out)


def _decode(fmt, planes):
    """Plane bytes [..., row_bytes] -> scaled alphabet values [..., k_pad].
    8-bit codes one per byte; 6-bit codes packed little-endian 16 to a 16-byte
    chunk whose last 4 bytes are zero; 4-bit codes two per byte (even entry in
    the low half)."""
    nb = CODE_BITS[fmt]
    if nb == 8:
        codes = planes.astype(np.int64)
    elif nb == 6:
        chunks = planes.reshape(*planes.shape[:-1], -1, 16)
        assert not chunks[..., 12:].any(), "padding bytes of a chunk are not zero"
        bits = np.unpackbits(chunks, axis=-1, bitorder="little")[..., :96]
        bits = bits.reshape(*bits.shape[:-1], 16, 6).astype(np.int64)
        codes = (bits << np.arange(6)).sum(axis=-1).reshape(*planes.shape[:-1], -1)
    else:
        b = planes.astype(np.int64)
        codes = np.stack([b & 15, b >> 4], axis=-1).reshape(*planes.shape[:-1], -1)
    lut = np.zeros(256, dtype=np.int64)
    ok = np.zeros(256, dtype=bool)
    for code, v in forms.code_values(fmt).items():
        lut[code], ok[code] = v, True
    assert ok[codes].all(), "a code that is not a finite value of the format"
    return lut[codes]


def _split(plan, X, contiguous, nvec, length, ld):
    nvec_pad = oz.round_up(max(nvec, 1), 256)
    k_pad, row_bytes = plan.plane_geometry(length)
    planes = torch.full((plan.planes, nvec_pad, row_bytes), 0x55, dtype=torch.uint8, device=DEV)   # poison
    shifts = torch.zeros(max(nvec, 1), dtype=torch.int32, device=DEV)
    flag = torch.zeros(4, dtype=torch.int32, device=DEV)
    colmax = torch.zeros(max(nvec, 1), dtype=torch.int64, device=DEV)
    st = oz.oz_split(plan.handle, contiguous, nvec, length, X.data_ptr(), ld, nvec_pad, k_pad, shifts.data_ptr(),
                     planes.data_ptr(), flag.data_ptr(), colmax.data_ptr(), oz._stream_handle())
    assert st == oz.OZ_OK
    torch.cuda.synchronize()
    return shifts.cpu().numpy()[:nvec], planes, flag.cpu().numpy()


@pytest.mark.parametrize("fmt", FORMATS)
def test_split_codes_match_oracle_tables(fmt):
    plan = oz.PlanFP(fmt, 1000)
    m, n, k = 300, 520, 1000
    A, B = synth.phi_pair(m, n, k, 2.0, seed=11)
    # rows of A
    s, P, flag = _split(plan, _dev(A), 1, m, k, k)
    s_ref, V_ref = _expected_values(plan, fmt, A, 1)
    assert np.array_equal(s, s_ref) and flag[0] == 0
    got = _decode(fmt, P.cpu().numpy())
    assert np.array_equal(got[:, :m, :k], V_ref)
    assert not got[:, m:, :].any() and not got[:, :, k:].any()
    # columns of B
    t, P, flag = _split(plan, _dev(B), 0, n, k, n)
    t_ref, V_ref = _expected_values(plan, fmt, B, 0)
    assert np.array_equal(t, t_ref) and flag[0] == 0
    got = _decode(fmt, P.cpu().numpy())
    assert np.array_equal(got[:, :n, :k], V_ref)
    assert not got[:, n:, :].any() and not got[:, :, k:].any()


@pytest.mark.parametrize("fmt", FORMATS)
def test_residues_match_oracle(fmt):
    """W mod m per channel after the form's GEMMs and the R>C fold (raw)."""
    plan = oz.PlanFP(fmt, 1000)
    m, n, k = 300, 520, 1000
    A, B = synth.phi_pair(m, n, k, 1.0, seed=12)
    _, U, _ = _split(plan, _dev(A), 1, m, k, k)
    _, V, _ = _split(plan, _dev(B), 0, n, k, n)
    Y = torch.zeros((plan.channels, m, n), dtype=torch.int16, device=DEV)
    flag = torch.zeros(4, dtype=torch.int32, device=DEV)
    st = oz.oz_residue_gemm(plan.handle, m, n, U.shape[1], V.shape[1], plan.plane_geometry(k)[0], U.data_ptr(),
                            V.data_ptr(), Y.data_ptr(), 1, flag.data_ptr(), oz._stream_handle())
    assert st == oz.OZ_OK
    torch.cuda.synchronize()
    assert flag.cpu().numpy()[0] & 2 == 0
    _, W, _, _ = oracle.dgemm(A, B, plan.moduli, plan.bits, want_residues=True)
    assert np.array_equal(Y.cpu().numpy().view(np.uint16), W)


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("m,n,k,phi,ta,tb", [
    (300, 520, 1000, 0.5, False, False),
    (129, 257, 640, 4.0, True, False),
    (200, 100, 333, 1.0, False, True),
    (1, 1, 1, 1.0, False, False),
    (17, 300, 0, 1.0, False, False),
])
def test_dgemm_bit_exact(fmt, m, n, k, phi, ta, tb):
    plan = oz.PlanFP(fmt, 1000)
    A, B = synth.phi_pair(m, n, k, phi, seed=m * 7 + n + k)
    At = _dev(A.T.copy()) if ta else _dev(A)
    Bt = _dev(B.T.copy()) if tb else _dev(B)
    C = oz.dgemm(At, Bt, plan, trans_a=ta, trans_b=tb).cpu().numpy()
    ref = oracle.dgemm(A, B, plan.moduli, plan.bits) if k else np.zeros((m, n))
    assert np.array_equal(C.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("fmt", FORMATS)
def test_dgemm_at_configured_k_sampled(fmt):
    """K = 8192, the inner dimension the configurations are built for: sampled
    entries against the oracle's one-by-one entries, plus the interior of the
    ragged tile."""
    plan = oz.PlanFP(fmt, 8192)
    m, n, k = 260, 300, 8192
    A, B = synth.phi_pair(m, n, k, 1.0, seed=5)
    C = oz.dgemm(_dev(A), _dev(B), plan).cpu().numpy()
    rng = np.random.default_rng(1)
    rows = np.concatenate([rng.integers(0, m, 200), [0, m - 1, 255, 256, m - 1]])
    cols = np.concatenate([rng.integers(0, n, 200), [0, n - 1, 255, 256, 0]])
    ref = oracle.dgemm_entries(A, B, plan.moduli, plan.bits, rows, cols)
    assert np.array_equal(C[rows, cols].view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("fmt", ["E4M3", "E3M2", "E2M1"])
def test_dgemm_at_k_cfg_65536_sampled(fmt):
    """An inner dimension past 2^14 takes the configuration searched for
    K = 2^16 (plane radius 16, more or larger moduli): sampled entries of the
    product against the oracle's one-by-one entries, bit for bit."""
    plan = oz.PlanFP(fmt, 40000)
    assert plan.k_cfg == 65536 and plan.bits >= 53
    m, n, k = 136, 200, 40000
    A, B = synth.phi_pair(m, n, k, 1.0, seed=11)
    C = oz.dgemm(_dev(A), _dev(B), plan).cpu().numpy()
    rng = np.random.default_rng(2)
    rows = np.concatenate([rng.integers(0, m, 150), [0, m - 1, 128]])
    cols = np.concatenate([rng.integers(0, n, 150), [n - 1, 0, 199]])
    ref = oracle.dgemm_entries(A, B, plan.moduli, plan.bits, rows, cols)
    assert np.array_equal(C[rows, cols].view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("fmt", ["E2M1", "E4M3", "E3M2"])
def test_widened_dgemm_bit_exact(fmt):
    """A plan asked for 69 bits takes the widened configuration (Example
    ex:widened; E2M1: 78 GEMMs over 26 channels, P about 2^154.5, a five-limb
    CRT; the split cuts |a'| < 2^69 into five 16-bit pieces). The product is
    bit-exact against the oracle, and on skewed rows (phi = 4) the widened
    budget's error is below the base configuration's."""
    plan = oz.PlanFP(fmt, 2000, 69)
    base = oz.PlanFP(fmt, 2000)
    assert plan.bits == 69 and plan.k_cfg == 16384 and plan.q > base.q
    m, n, k = 150, 136, 2000
    A, B = synth.phi_pair(m, n, k, 4.0, seed=23)
    C = oz.dgemm(_dev(A), _dev(B), plan).cpu().numpy()
    ref = oracle.dgemm(A, B, plan.moduli, plan.bits)
    assert np.array_equal(C.view(np.uint64), ref.view(np.uint64))
    C0 = oz.dgemm(_dev(A), _dev(B), base).cpu().numpy()
    rows, cols = np.arange(0, m, 7), np.arange(0, n, 5)
    r, c = np.meshgrid(rows, cols, indexing="ij")
    r, c = r.ravel(), c.ravel()
    e69, _ = oracle.exact_error(A, B, C, r, c)
    e53, _ = oracle.exact_error(A, B, C0, r, c)
    assert e69.max() < e53.max()


def test_inner_dimension_above_k_max_is_refused():
    plan = oz.PlanFP("E4M3", 8192)
    A = torch.zeros((4, plan.k_max + 200), dtype=torch.float64, device=DEV)
    B = torch.zeros((plan.k_max + 200, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(oz.OzError):
        oz.dgemm(A, B, plan)


def _encode(fmt, codes):
    """Inverse of _decode: [..., k_pad] codes -> plane bytes [..., row_bytes]."""
    nb = CODE_BITS[fmt]
    if nb == 8:
        return codes.astype(np.uint8)
    if nb == 4:
        c = codes.reshape(*codes.shape[:-1], -1, 2).astype(np.int64)
        return (c[..., 0] | (c[..., 1] << 4)).astype(np.uint8)
    ch = codes.reshape(*codes.shape[:-1], -1, 16).astype(np.int64)
    bits = ((ch[..., None] >> np.arange(6)) & 1).reshape(*ch.shape[:-1], 96)
    pad = np.zeros((*bits.shape[:-1], 32), dtype=np.int64)
    return np.packbits(np.concatenate([bits, pad], -1).astype(np.uint8), axis=-1,
                       bitorder="little").reshape(codes.shape)


@pytest.mark.parametrize("fmt", FORMATS)
def test_fp32_accumulation_is_exact_at_capacity(fmt):
    """Every product at the largest plane value rho and K = K_max, so the FP32
    accumulators reach K rho^2 (at most 2^24, eq. ov-accgen): each channel's
    folded residue must equal sum_g lambda_g W_g mod m exactly. Rows of B
    alternate in sign so that both signs reach capacity."""
    plan = oz.PlanFP(fmt, 8192)
    vals = plan.plane_values()
    rho = max(abs(v) for tab in vals for v in tab)
    code_of = {v: c for c, v in forms.code_values(fmt).items() if not (v == 0 and c != 0)}
    k = plan.k_max
    assert k * rho * rho <= 2**24
    m, n = 128, 256
    k_pad, row_bytes = plan.plane_geometry(k)

    def row(code):
        r = np.zeros(k_pad, dtype=np.int64)
        r[:k] = code
        return _encode(fmt, r)

    Uh = np.zeros((plan.planes, 256, row_bytes), dtype=np.uint8)
    Vh = np.zeros((plan.planes, 256, row_bytes), dtype=np.uint8)
    Uh[:, :m] = row(code_of[rho])
    Vh[:, 0:n:2] = row(code_of[rho])
    Vh[:, 1:n:2] = row(code_of[-rho])
    U, V = _dev(Uh), _dev(Vh)
    Y = torch.zeros((plan.channels, m, n), dtype=torch.int16, device=DEV)
    flag = torch.zeros(4, dtype=torch.int32, device=DEV)
    st = oz.oz_residue_gemm(plan.handle, m, n, 256, 256, k_pad, U.data_ptr(), V.data_ptr(), Y.data_ptr(), 1,
                            flag.data_ptr(), oz._stream_handle())
    assert st == oz.OZ_OK
    torch.cuda.synchronize()
    y = Y.cpu().numpy().view(np.uint16)
    for c, (mod, f, b) in enumerate(zip(plan.moduli, plan.forms, plan.bases)):
        lam = sum(w[2] for w in forms.weights(KIND[f], b))
        for sign, cols in ((1, slice(0, n, 2)), (-1, slice(1, n, 2))):
            want = (lam * sign * k * rho * rho) % mod
            assert (y[c, :, cols] == want).all(), (c, mod, sign)
