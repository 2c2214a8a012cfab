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


def test_host_path_back_to_back_calls_and_two_threads():
    """The pipeline's events come from a per-thread pool reused by every call:
    calls queued back to back on one thread (each recording the events the
    previous call's work still waits on), and two threads with their own
    streams and workspaces running at once, all give the oracle's product."""
    import threading
    plan = oz.Plan(16, 0, 1500, oz.OZ_ENGINE_TC)
    m, n, k = 900, 700, 1500
    ops = [synth.phi_pair(m, n, k, 1.0, seed=40 + i) for i in range(3)]
    pinned = [(torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()) for A, B in ops]
    outs = [torch.full((m, n), np.nan, dtype=torch.float64).pin_memory() for _ in ops]
    hg = oz.HostGemm(plan, m, n, k, 256, cols_per_chunk=256)
    for (Ah, Bh), Ch in zip(pinned, outs):           # queued without a synchronisation between them
        hg(Ah, Bh, Ch)
    torch.cuda.synchronize()
    assert oz.query_status(hg.ws) == oz.OZ_OK
    for (A, B), Ch in zip(ops, outs):
        assert_oracle_bits(Ch.numpy(), A, B, plan.moduli, plan.bits, what="back-to-back host calls", count=512)

    results, errors = {}, []

    def worker(t):
        try:
            torch.cuda.set_device(0)
            stream = torch.cuda.Stream()
            g = oz.HostGemm(plan, m, n, k, 256, cols_per_chunk=256)
            Ah, Bh = pinned[t]
            Cs = [torch.full((m, n), np.nan, dtype=torch.float64).pin_memory() for _ in range(2)]
            for Ch in Cs:
                g(Ah, Bh, Ch, stream)
            stream.synchronize()
            results[t] = (Cs, oz.query_status(g.ws, stream))
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert not errors, errors
    for t in range(2):
        Cs, status = results[t]
        assert status == oz.OZ_OK
        A, B = ops[t]
        for Ch in Cs:
            assert_oracle_bits(Ch.numpy(), A, B, plan.moduli, plan.bits, what=f"host thread {t}", count=512)
