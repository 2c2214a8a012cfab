"""The differentiable emulated product (EmuMatmul): gradients dA = dC B^T and
dB = A^T dC through the same kernels, checked bit for bit against the oracle's
products (each is an emulated product of its own, rounded once from the exact
product of its truncated operands), against central finite differences,
torch.autograd.gradcheck, and FP64 autograd within the error bound of the two
computations."""
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
U = 2.0**-53


def _t(a, grad=False):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).requires_grad_(grad)


def test_gradcheck_small():
    rng = np.random.default_rng(0)
    A = _t(rng.standard_normal((7, 5)), True)
    B = _t(rng.standard_normal((5, 3)), True)
    assert torch.autograd.gradcheck(lambda a, b: oz.emu_matmul(a, b), (A, B), eps=1e-6, atol=1e-9, rtol=1e-7)


def _bound(X, Y, beta, K):
    """Entrywise bound on |emulated(X Y) - fp64 (X Y)|: truncation (2^(1-beta)
    times the row/column maxima against the absolute sums, Sec. 'May Be Less
    Accurate Than Native on Skewed Rows'), our final rounding, and the
    recursive-summation bound of the FP64 reference, (K + 2) u |X||Y|."""
    aX, aY = X.abs(), Y.abs()
    xmax = aX.max(dim=1).values[:, None]
    ymax = aY.max(dim=0).values[None, :]
    trunc = 2.0**(1 - beta) * (xmax * aY.sum(dim=0)[None, :] + ymax * aX.sum(dim=1)[:, None])
    return trunc + (K + 2) * U * (aX @ aY)


@pytest.mark.parametrize("m,k,n", [(4096, 4096, 4096), (65536, 256, 256), (300, 70, 129)])
def test_gradients_match_fp64_autograd_and_finite_differences(m, k, n):
    A_h, B_h = synth.phi_pair(m, n, k, 1.0, seed=5)
    rng = np.random.default_rng(6)
    dC_h = rng.standard_normal((m, n))
    A, B, dC = _t(A_h, True), _t(B_h, True), _t(dC_h)
    C = oz.emu_matmul(A, B)
    C.backward(dC)
    # the forward product and both gradients against the oracle, bit for bit:
    # every entry at 300 x 70 x 129, 2048 sampled entries (with the last row
    # and column) at the large shapes
    pc, pa, pb = oz.plan_for(k), oz.plan_for(n), oz.plan_for(m)
    assert_oracle_bits(C, A_h, B_h, pc.moduli, pc.bits, what="C = A B", count=2048, seed=1)
    assert_oracle_bits(A.grad, dC_h, B_h.T, pa.moduli, pa.bits, what="dA = dC B^T", count=2048, seed=2)
    assert_oracle_bits(B.grad, A_h.T, dC_h, pb.moduli, pb.bits, what="dB = A^T dC", count=2048, seed=3)
    # FP64 autograd
    A2, B2 = _t(A_h, True), _t(B_h, True)
    (A2 @ B2).backward(dC)
    with torch.no_grad():
        beta_c = oz.plan_for(k).bits
        assert torch.all((C - A2 @ B2).abs() <= _bound(A, B, beta_c, k))
        beta_a = oz.plan_for(n).bits              # dA = dC B^T: inner dimension n
        assert torch.all((A.grad - A2.grad).abs() <= _bound(dC, B.t(), beta_a, n))
        beta_b = oz.plan_for(m).bits              # dB = A^T dC: inner dimension m
        assert torch.all((B.grad - B2.grad).abs() <= _bound(A.t(), dC, beta_b, m))
        # central differences along random directions; the loss <dC, A B> is
        # bilinear, so the difference quotient at h = 1 is the exact directional
        # derivative up to the rounding of the two loss values
        EA = _t(rng.standard_normal((m, k)))
        EB = _t(rng.standard_normal((k, n)))
        loss = lambda a, b: float((dC * oz.emu_matmul(a, b)).sum())  # noqa: E731
        fd_a = (loss(A + EA, B) - loss(A - EA, B)) / 2.0
        fd_b = (loss(A, B + EB) - loss(A, B - EB)) / 2.0
        ga = float((A.grad * EA).sum())
        gb = float((B.grad * EB).sum())
        scale_a = float((dC.abs() * ((A.abs() + EA.abs()) @ B.abs())).sum())
        scale_b = float((dC.abs() * (A.abs() @ (B.abs() + EB.abs()))).sum())
        assert abs(fd_a - ga) <= 1e-12 * scale_a
        assert abs(fd_b - gb) <= 1e-12 * scale_b


def test_no_grad_inputs():
    A = _t(np.eye(3), False)
    B = _t(np.arange(9.0).reshape(3, 3), True)
    C = oz.emu_matmul(A, B)
    C.sum().backward()
    assert B.grad is not None and torch.equal(B.grad, torch.ones_like(B))
