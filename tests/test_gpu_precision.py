"""Accuracy per modulus count (the precision trade-off): errors against the
exact product fall as Q (and with it the bit budget) grows, and at Q = 16 and
phi = 0.5 they stay within 2 u (|A||B|)_ij. Every sampled entry of each GPU
product is first checked bit for bit against the oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2609_37693_gb300 as oz  # noqa: E402

U = 2.0**-53


def _sweep(n, phis, qs, samples):
    """Rows (phi, q, bits, max error in u |A||B|) of GPU products at the widest
    beta each Q's window allows at K = n, and also at 53 where it holds."""
    rows = []
    for phi in phis:
        A, B = synth.phi_pair(n, n, n, phi, seed=0)
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        r, c = synth.sample_entries(n, n, samples, seed=7)
        for q in qs:
            bmax = oz.Plan(q, 0, n).bits
            for bits in [bmax] + ([53] if 53 < bmax else []):
                plan = oz.Plan(q, bits, n)
                C = oz.dgemm(Ad, Bd, plan).cpu().numpy()
                ref = oracle.dgemm_entries(A, B, plan.moduli, plan.bits, r, c)
                assert np.array_equal(C[r, c].view(np.uint64), ref.view(np.uint64)), (phi, q, bits)
                err, ab = oracle.exact_error(A, B, C, r, c)
                rel = np.where(ab > 0, err / (U * np.where(ab > 0, ab, 1.0)), np.where(err > 0, np.inf, 0.0))
                rows.append({"phi": phi, "q": q, "bits": plan.bits, "max_err_u": float(rel.max())})
    return rows


def test_error_falls_with_q_and_meets_2u_at_q16():
    rows = _sweep(1024, [0.5, 2.0], [10, 12, 14, 16, 18, 20], samples=4096)
    for phi in (0.5, 2.0):
        top = [r for r in rows if r["phi"] == phi and r["bits"] == max(x["bits"] for x in rows
                                                                       if x["phi"] == phi and x["q"] == r["q"])]
        errs = [r["max_err_u"] for r in sorted(top, key=lambda r: r["q"])]
        # more moduli never hurt: each error at most that of two fewer moduli, up to
        # the noise of the final rounding once the truncation error is below 1 u
        assert all(b <= max(1.05 * a, 1.0) for a, b in zip(errs, errs[1:])), errs
        assert errs[0] > 10 * errs[-1]
    q16 = [r for r in rows if r["phi"] == 0.5 and r["q"] == 16]
    assert q16 and min(r["max_err_u"] for r in q16) <= 2.0
    q16b = [r for r in q16 if r["bits"] > 53]
    assert q16b and q16b[0]["max_err_u"] <= 2.0
