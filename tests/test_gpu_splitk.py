"""Split-K of the TC GEMM: a product with too few output tiles for the GPU
cuts its inner dimension into ranges of whole 1024-term slabs, each range's
GEMMs write CRT digits of their own, and the digit sets are added modulo each
modulus before the Reconstruct (Sec. "Slabs": the digits are linear in W, and W
is the sum of the ranges' products). The result must equal the oracle's
product bit for bit, on both TC kernels, with ragged K, ragged output shapes
and the transposed operand modes the autograd products use."""
import numpy as np
import pytest

import synth
from tests.oracle_check import assert_oracle_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2609_37693_gb300 as oz  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("engine", [oz.OZ_ENGINE_TC, oz.OZ_ENGINE_TC1])
@pytest.mark.parametrize("m,n,k", [(256, 256, 65536), (300, 200, 40000), (64, 700, 5000), (1, 1, 3000),
                                   (256, 256, 2049), (512, 256, 1024 * 9 + 5)])
def test_split_k_matches_oracle(engine, m, n, k):
    plan = oz.Plan(16, 53, k, engine)
    # the layout reserves more than one residue set exactly when the GEMM splits
    splits = oz.oz_workspace_bytes(plan.handle, m, n, k) > oz.oz_blocked_workspace_bytes(plan.handle, m, n, k)
    if (m, n, k) == (256, 256, 65536):
        assert splits
    A, B = synth.phi_pair(m, n, k, 1.0, seed=m + n + k)
    C = oz.dgemm(_dev(A), _dev(B), plan)
    torch.cuda.synchronize()
    assert_oracle_bits(C, A, B, plan.moduli, plan.bits, what=f"split-K {m}x{n}x{k}", count=768)


@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1)])
def test_split_k_transposed_operands(ta, tb):
    """dB = A^T dC of a tall-skinny product: the inner dimension is the long
    one (65536), the output 256 x 256."""
    m, n, k = 256, 256, 65536
    plan = oz.Plan(16, 53, k, oz.OZ_ENGINE_TC)
    A, B = synth.phi_pair(m, n, k, 1.0, seed=7)
    Ain = A.T if ta else A
    Bin = B.T if tb else B
    C = oz.dgemm(_dev(Ain), _dev(Bin), plan, trans_a=bool(ta), trans_b=bool(tb))
    torch.cuda.synchronize()
    assert_oracle_bits(C, A, B, plan.moduli, plan.bits, what=f"split-K ta={ta} tb={tb}", count=768)


def test_split_k_reports_nonfinite_and_then_recovers():
    m, n, k = 256, 256, 30000
    plan = oz.Plan(16, 53, k, oz.OZ_ENGINE_TC)
    A, B = synth.phi_pair(m, n, k, 1.0, seed=9)
    A[3, 29999] = np.nan
    ws = oz.workspace(plan, m, n, k, DEV)
    oz.dgemm(_dev(A), _dev(B), plan, ws=ws)
    assert oz.query_status(ws) == oz.OZ_ERR_NONFINITE
    A[3, 29999] = 0.5
    C = oz.dgemm(_dev(A), _dev(B), plan, ws=ws)
    assert oz.query_status(ws) == oz.OZ_OK
    assert_oracle_bits(C, A, B, plan.moduli, plan.bits, what="split-K after a non-finite run")
