"""oz_dgemm_static, the entry point for callers that cannot allocate device
memory: a BLAS-style dgemm interface, which has no workspace argument, or a
host program that owns every device allocation through its own pool and
forbids libraries to call cudaMalloc. Its workspace is a scratch array built
into the library.

What these tests show: call after call, on the same shared array, the entry
point returns the product oz_dgemm returns with a caller-provided workspace,
and both equal the oracle's bit for bit (Sec. "Emulation Problem"); leftovers
of an earlier call (an INT8 product before a float-format one, whose digits
and planes have another layout) never reach a later result; its status query
reports a clean run and non-finite input; and sizes beyond the array are
refused before any launch. They do not observe the absence of allocation
itself (the library does not allocate through torch, so no allocator counter
would see a call); that rests on the code, which calls no allocating routine.

This file is named so that pytest collects it last."""
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


def _run_both(plan, A, B, ta=0, tb=0):
    """C from oz_dgemm (own workspace) and from oz_dgemm_static, and the
    static path's status."""
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    Bd = torch.from_numpy(np.ascontiguousarray(B)).to(DEV)
    C_ref = torch.full((m, n), np.nan, dtype=torch.float64, device=DEV)
    C_st = torch.full((m, n), np.nan, dtype=torch.float64, device=DEV)
    ws = oz.workspace(plan, m, n, k, DEV)
    stream = oz._stream_handle()
    assert oz.oz_dgemm(plan.handle, ta, tb, m, n, k, Ad.data_ptr(), Ad.shape[1], Bd.data_ptr(), Bd.shape[1],
                       C_ref.data_ptr(), n, ws.data_ptr(), ws.numel(), stream) == oz.OZ_OK
    assert oz.oz_dgemm_static(plan.handle, ta, tb, m, n, k, Ad.data_ptr(), Ad.shape[1], Bd.data_ptr(), Bd.shape[1],
                              C_st.data_ptr(), n, stream) == oz.OZ_OK
    status = oz.oz_static_query_status(stream)
    torch.cuda.synchronize()
    return C_ref.cpu().numpy(), C_st.cpu().numpy(), status


def _check(plan, A, B, ta=0, tb=0, what=""):
    C_ref, C_st, status = _run_both(plan, A, B, ta, tb)
    assert status == oz.OZ_OK, what
    assert np.array_equal(C_ref.view(np.uint64), C_st.view(np.uint64)), what
    opA = A.T if ta else A
    opB = B.T if tb else B
    assert_oracle_bits(C_st, opA, opB, plan.moduli, plan.bits, what=what)


def test_static_scratch_matches_workspace_path_on_consecutive_calls():
    plan = oz.Plan(16, 0, 512, oz.OZ_ENGINE_AUTO)
    # two calls in a row with different shapes and data: the second must not
    # see anything the first left in the shared array
    for (m, n, k, seed) in ((300, 257, 512, 1), (129, 400, 333, 2)):
        A, B = synth.phi_pair(m, n, k, 1.0, seed=seed)
        _check(plan, A, B, what=f"INT8 {m}x{n}x{k}")
    # transposed operands through the same scratch
    A, B = synth.phi_pair(200, 100, 300, 2.0, seed=3)
    _check(plan, np.ascontiguousarray(A.T), B, ta=1, what="INT8, A transposed")


def test_static_scratch_float_format_after_int8():
    """A float-format product (uint16 digits, code planes, no B^T region)
    right after an INT8 product on the same array, then INT8 again."""
    int8 = oz.Plan(16, 0, 512, oz.OZ_ENGINE_AUTO)
    fp = oz.PlanFP("E4M3", 512)
    A, B = synth.phi_pair(256, 300, 512, 1.0, seed=11)
    _check(int8, A, B, what="INT8 before E4M3")
    A, B = synth.phi_pair(200, 190, 480, 1.5, seed=12)
    assert fp.workspace_bytes(200, 190, 480) <= oz.OZ_STATIC_SCRATCH_BYTES
    _check(fp, A, B, what="E4M3 after INT8")
    A, B = synth.phi_pair(140, 333, 500, 0.5, seed=13)
    _check(int8, A, B, what="INT8 after E4M3")


def test_static_status_reports_nonfinite_then_clears():
    plan = oz.Plan(16, 0, 256, oz.OZ_ENGINE_AUTO)
    A, B = synth.phi_pair(64, 64, 256, 1.0, seed=21)
    A[5, 7] = np.inf
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.empty((64, 64), dtype=torch.float64, device=DEV)
    stream = oz._stream_handle()
    assert oz.oz_dgemm_static(plan.handle, 0, 0, 64, 64, 256, Ad.data_ptr(), 256, Bd.data_ptr(), 64, C.data_ptr(),
                              64, stream) == oz.OZ_OK
    assert oz.oz_static_query_status(stream) == oz.OZ_ERR_NONFINITE
    A[5, 7] = 1.0
    _check(plan, A, B, what="finite input after a non-finite one")


def test_static_scratch_refuses_sizes_beyond_its_array():
    plan = oz.Plan(16, 0, 8192, oz.OZ_ENGINE_AUTO)
    n = 2048
    assert plan.workspace_bytes(n, n, n) > oz.OZ_STATIC_SCRATCH_BYTES
    dummy = torch.zeros(1, dtype=torch.float64, device=DEV)
    st = oz.oz_dgemm_static(plan.handle, 0, 0, n, n, n, dummy.data_ptr(), n, dummy.data_ptr(), n, dummy.data_ptr(),
                            n, oz._stream_handle())
    assert st == oz.OZ_ERR_WORKSPACE
