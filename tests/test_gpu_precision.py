"""Accuracy per modulus count (the precision trade-off): errors against the
exact product fall as Q (and with it the bit budget) grows, and at Q = 16 and
phi = 0.5 they stay within 2 u (|A||B|)_ij."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from tests.precision_sweep import sweep  # noqa: E402


def test_error_falls_with_q_and_meets_2u_at_q16():
    rows = sweep([1024], [0.5, 2.0], [10, 12, 14, 16, 18, 20], samples=4096, reps=1, dgemm=False, log=lambda s: None)
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
