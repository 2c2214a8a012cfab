"""The blocked call (Sec. "Slabs"): the inner dimension in slabs, each slab's
CRT digits added into a running residue, one Reconstruct at the end. Its
result is the unblocked product's, bit for bit: the shifts are taken over the
whole K, and the digits are linear in W = sum over slabs of the slab products.
Checked against the oracle, against oz_dgemm, and past the INT32 accumulation
cap of the IMMA engine, where only the blocked call applies. All calls go
through the C ABI."""
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


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _operands(A, B, ta, tb):
    """Device operands stored so that op(A) = A and op(B) = B."""
    return _dev(A.T if ta else A), _dev(B.T if tb else B)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("m,n,k,k_slab,ta,tb", [(300, 520, 1000, 256, 0, 0), (300, 520, 1000, 333, 1, 0),
                                                (129, 257, 2000, 700, 0, 1), (200, 100, 1500, 1500, 1, 1),
                                                (64, 64, 777, 5000, 0, 0), (17, 300, 129, 128, 0, 0),
                                                (1, 1, 3, 1, 0, 0)])
def test_blocked_equals_oracle_and_unblocked(engine, m, n, k, k_slab, ta, tb):
    plan = oz.Plan(16, 53, k, engine)
    A, B = synth.phi_pair(m, n, k, 1.0, seed=m + 3 * k)
    Ad, Bd = _operands(A, B, ta, tb)
    Cb = oz.dgemm_blocked(Ad, Bd, plan, k_slab, trans_a=bool(ta), trans_b=bool(tb))
    Cu = oz.dgemm(Ad, Bd, plan, trans_a=bool(ta), trans_b=bool(tb))
    torch.cuda.synchronize()
    ref = oracle.dgemm(A, B, plan.moduli, plan.bits)
    assert np.array_equal(_bits(Cb.cpu().numpy()), _bits(ref))
    assert torch.equal(Cb.view(torch.int64), Cu.view(torch.int64))


def test_blocked_past_the_int32_accumulation_cap():
    """K = 152 000 at Q = 16, beta = 53: above the IMMA engine's INT32 cap
    (151 647), below the window (159 819). oz_dgemm refuses it on that engine;
    the blocked call in slabs of 100 000 gives the oracle's bits, which are also
    the TC engine's (no accumulation cap) unblocked result."""
    m, n, k = 12, 20, 152000
    imma = oz.Plan(16, 53, 100000, oz.OZ_ENGINE_IMMA)
    assert imma.k_max < k <= imma.k_rec
    A, B = synth.phi_pair(m, n, k, 0.5, seed=7)
    Ad, Bd = _dev(A), _dev(B)
    with pytest.raises(oz.OzError):
        oz.dgemm(Ad, Bd, imma)
    Cb = oz.dgemm_blocked(Ad, Bd, imma, 100000)
    tc = oz.Plan(16, 53, k, oz.OZ_ENGINE_TC)
    Ct = oz.dgemm(Ad, Bd, tc)
    torch.cuda.synchronize()
    ref = oracle.dgemm(A, B, imma.moduli, 53)
    assert np.array_equal(_bits(Cb.cpu().numpy()), _bits(ref))
    assert torch.equal(Cb.view(torch.int64), Ct.view(torch.int64))


@pytest.mark.parametrize("fmt", ["E4M3", "E3M2", "E2M1"])
def test_blocked_float_formats(fmt):
    """Float-format plans: slabs within the FP32 accumulation cap, the 16-bit
    digits added modulo each channel's modulus; bit for bit the unblocked
    product and the oracle's."""
    plan = oz.PlanFP(fmt, 3000, 53)
    m, n, k = 200, 300, 3000
    A, B = synth.phi_pair(m, n, k, 1.0, seed=11)
    Ad, Bd = _dev(A), _dev(B)
    Cb = oz.dgemm_blocked(Ad, Bd, plan, 1024)
    Cu = oz.dgemm(Ad, Bd, plan)
    torch.cuda.synchronize()
    ref = oracle.dgemm(A, B, plan.moduli, plan.bits)
    assert np.array_equal(_bits(Cb.cpu().numpy()), _bits(ref))
    assert torch.equal(Cb.view(torch.int64), Cu.view(torch.int64))


def test_blocked_float_format_past_its_accumulation_cap():
    """An E4M3 plan built for K = 8192 has an FP32 accumulation cap k_acc and a
    window k_rec at its beta. Where the window is the larger, K between the two
    runs only blocked; the result is the exact product's rounding, the oracle's
    and the INT8 TC engine's at the same beta."""
    plan = oz.PlanFP("E4M3", 8192, 53)
    if plan.k_rec <= plan.k_acc:
        pytest.skip("the window is the binding cap of this configuration")
    k = min(plan.k_rec, plan.k_acc + 4096)
    m, n = 40, 24
    A, B = synth.phi_pair(m, n, k, 0.5, seed=5)
    Ad, Bd = _dev(A), _dev(B)
    Cb = oz.dgemm_blocked(Ad, Bd, plan, plan.k_acc)
    tc = oz.Plan(16, 53, k, oz.OZ_ENGINE_TC)
    Ct = oz.dgemm(Ad, Bd, tc)
    torch.cuda.synchronize()
    ref = oracle.dgemm(A, B, plan.moduli, 53)
    assert np.array_equal(_bits(Cb.cpu().numpy()), _bits(ref))
    assert torch.equal(Cb.view(torch.int64), Ct.view(torch.int64))


def test_blocked_edges_and_nonfinite():
    plan = oz.Plan(16, 53, 1000, oz.OZ_ENGINE_TC)
    C = torch.full((5, 3), 9.0, dtype=torch.float64, device=DEV)
    oz.dgemm_blocked(torch.zeros((5, 0), dtype=torch.float64, device=DEV),
                     torch.zeros((0, 3), dtype=torch.float64, device=DEV), plan, 64, out=C)
    torch.cuda.synchronize()
    assert torch.all(C == 0)
    A, B = synth.phi_pair(20, 30, 700, 1.0, seed=2)
    A[4, 650] = np.inf                         # in the last slab only
    ws = torch.empty(oz.oz_blocked_workspace_bytes(plan.handle, 20, 30, 256), dtype=torch.uint8, device=DEV)
    oz.dgemm_blocked(_dev(A), _dev(B), plan, 256, ws=ws)
    assert oz.query_status(ws) == oz.OZ_ERR_NONFINITE
    A[4, 650] = 1.0
    oz.dgemm_blocked(_dev(A), _dev(B), plan, 256, ws=ws)
    assert oz.query_status(ws) == oz.OZ_OK


def test_autotuned_configurations_agree():
    """The configuration trade-off (plane format and its GEMM count, slab
    length): every candidate keeps beta = 53 bits, so every one returns the
    oracle's bits, and the autotuner returns one of them with its timing."""
    m, n, k = 160, 96, 3000
    A, B = synth.phi_pair(m, n, k, 1.0, seed=21)
    Ad, Bd = _dev(A), _dev(B)
    cands = oz.blocked_candidates(k, 53, slabs=(1024,))
    labels = [c[0] for c in cands]
    assert any(l.startswith("int8") for l in labels) and any(l.startswith("E4M3") for l in labels)
    ref = _bits(oracle.dgemm(A, B, cands[0][1].moduli, 53))
    for label, plan, k_slab in cands:
        C = oz.dgemm_blocked(Ad, Bd, plan, k_slab)
        torch.cuda.synchronize()
        assert np.array_equal(_bits(C.cpu().numpy()), ref), label
    (label, plan, k_slab), times = oz.autotune_blocked(Ad, Bd, cands, reps=1)
    assert label in times and set(times) == set(labels)


@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1)])
def test_blocked_float_format_transposed(ta, tb):
    plan = oz.PlanFP("E4M3", 3000, 53)
    m, n, k = 150, 130, 2500
    A, B = synth.phi_pair(m, n, k, 1.0, seed=12 + ta)
    Ad, Bd = _operands(A, B, ta, tb)
    Cb = oz.dgemm_blocked(Ad, Bd, plan, 1000, trans_a=bool(ta), trans_b=bool(tb))
    torch.cuda.synchronize()
    assert np.array_equal(_bits(Cb.cpu().numpy()), _bits(oracle.dgemm(A, B, plan.moduli, plan.bits)))


@pytest.mark.parametrize("engine", ENGINES)
def test_blocked_widened_budget(engine):
    """beta = 70 (seven 12-bit pieces per entry) through the blocked call: the
    shifts over the whole K and the given-shift splits of each slab."""
    plan = oz.Plan(20, 70, 3000, engine)
    m, n, k = 140, 90, 3000
    A, B = synth.phi_pair(m, n, k, 2.0, seed=70)
    Ad, Bd = _dev(A), _dev(B)
    Cb = oz.dgemm_blocked(Ad, Bd, plan, 1100)
    torch.cuda.synchronize()
    assert np.array_equal(_bits(Cb.cpu().numpy()), _bits(oracle.dgemm(A, B, plan.moduli, 70)))
