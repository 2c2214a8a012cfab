"""Failure detection on the GPU without a fault (the waits of every GEMM kernel
are bounded): a wait on a barrier that nothing signals runs out after about
2 s, reports through the status word that oz_query_status reads, and the
kernel returns, leaving the context usable for the next product."""
import time

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


def test_bounded_wait_completes_when_signalled():
    status = torch.zeros(4, dtype=torch.int32, device=DEV)
    assert oz.oz_selftest_bounded_wait(1, status.data_ptr(), oz._stream_handle()) == oz.OZ_OK
    torch.cuda.synchronize()
    assert int(status[0]) == 4


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    plan = oz.Plan(16, 53, 300, oz.OZ_ENGINE_TC)
    ws = oz.workspace(plan, 40, 30, 300)
    ws.zero_()
    t0 = time.time()
    assert oz.oz_selftest_bounded_wait(0, ws.data_ptr(), oz._stream_handle()) == oz.OZ_OK
    assert oz.query_status(ws) == oz.OZ_ERR_CUDA          # bit 1: a bounded wait ran out
    waited = time.time() - t0
    assert 1.5 < waited < 30.0
    assert int(ws[:4].view(torch.int32)[0]) == 2
    # the next product on the same context and workspace is right, and clears the word
    A, B = synth.phi_pair(40, 30, 300, 1.0, seed=3)
    C = oz.dgemm(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), plan, ws=ws)
    assert oz.query_status(ws) == oz.OZ_OK
    ref = oracle.dgemm(A, B, plan.moduli, 53)
    assert np.array_equal(C.cpu().numpy().view(np.uint64), ref.view(np.uint64))
