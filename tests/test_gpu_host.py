"""oz_dgemm_host (host-resident operands, C in blocks, copies overlapped with
the phases of neighbouring blocks) gives the oracle's product bit for bit
(Sec. "Emulation Problem"), whatever the block shape (ragged last blocks,
edges not multiples of 16, one block, k = 0)."""
import numpy as np
import pytest

import synth
from tests.oracle_check import assert_oracle_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2609_37693_gb300 as oz  # noqa: E402


@pytest.mark.parametrize("engine", [oz.OZ_ENGINE_TC, oz.OZ_ENGINE_TC1, oz.OZ_ENGINE_IMMA])
@pytest.mark.parametrize("m,n,k,rows,cols", [(1000, 700, 900, 256, 0), (513, 300, 2000, 0, 0), (64, 64, 64, 0, 0),
                                             (2048, 1024, 1500, 512, 256), (700, 129, 0, 300, 50),
                                             (777, 1000, 700, 300, 333), (300, 520, 1024, 4096, 4096)])
def test_host_path_equals_device_path(engine, m, n, k, rows, cols):
    plan = oz.Plan(16, 0, max(k, 1), engine)
    A, B = synth.phi_pair(m, n, k, 1.0, seed=m + n)
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    Ch = torch.full((m, n), np.nan, dtype=torch.float64).pin_memory()
    hg = oz.HostGemm(plan, m, n, k, rows, cols_per_chunk=cols)
    hg(Ah, Bh, Ch)
    torch.cuda.synchronize()
    assert oz.query_status(hg.ws) == oz.OZ_OK
    assert_oracle_bits(Ch.numpy(), A, B, plan.moduli, plan.bits, what=f"host path {m}x{n}x{k}")


@pytest.mark.parametrize("fmt", ["E4M3", "E3M2", "E2M1"])
@pytest.mark.parametrize("m,n,k,rows,cols", [(1000, 700, 900, 256, 0), (300, 257, 1000, 0, 100)])
def test_host_path_float_formats(fmt, m, n, k, rows, cols):
    plan = oz.PlanFP(fmt, max(k, 1))
    A, B = synth.phi_pair(m, n, k, 1.0, seed=m + k)
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    Ch = torch.full((m, n), np.nan, dtype=torch.float64).pin_memory()
    hg = oz.HostGemm(plan, m, n, k, rows, cols_per_chunk=cols)
    hg(Ah, Bh, Ch)
    torch.cuda.synchronize()
    assert oz.query_status(hg.ws) == oz.OZ_OK
    assert_oracle_bits(Ch.numpy(), A, B, plan.moduli, plan.bits, what=f"host path {m}x{n}x{k}")


def test_host_path_widened_budget():
    """beta = 70 on the host-operand path (the splits of each chunk take seven
    12-bit pieces per entry)."""
    plan = oz.Plan(20, 70, 900, oz.OZ_ENGINE_TC)
    m, n, k = 600, 500, 900
    A, B = synth.phi_pair(m, n, k, 2.0, seed=7)
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    Ch = torch.full((m, n), np.nan, dtype=torch.float64).pin_memory()
    hg = oz.HostGemm(plan, m, n, k, 256, cols_per_chunk=256)
    hg(Ah, Bh, Ch)
    torch.cuda.synchronize()
    assert_oracle_bits(Ch.numpy(), A, B, plan.moduli, 70, what="host path, beta = 70")
