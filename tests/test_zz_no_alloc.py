"""oz_dgemm_static, the entry point for callers that cannot allocate device
memory (for example a BLAS-style dgemm interface, which has no workspace
argument, or a host program that owns every device allocation). It must give
the same product as oz_dgemm with a caller-provided workspace, call after call,
and refuse sizes that do not fit its built-in scratch array.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2609_37693_gb300 as oz  # noqa: E402

DEV = torch.device("cuda:0")


def _run_both(plan, A, B, ta=0, tb=0):
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
    torch.cuda.synchronize()
    return C_ref.cpu().numpy(), C_st.cpu().numpy()


def test_static_scratch_matches_workspace_path_on_consecutive_calls():
    plan = oz.Plan(16, 0, 512, oz.OZ_ENGINE_AUTO)
    # two calls in a row with different shapes and data: the second must not
    # see anything the first left in the shared array
    for (m, n, k, seed) in ((300, 257, 512, 1), (129, 400, 333, 2)):
        A, B = synth.phi_pair(m, n, k, 1.0, seed=seed)
        C_ref, C_st = _run_both(plan, A, B)
        assert np.array_equal(C_ref.view(np.uint64), C_st.view(np.uint64))
    # transposed operands through the same scratch
    A, B = synth.phi_pair(200, 100, 300, 2.0, seed=3)
    C_ref, C_st = _run_both(plan, np.ascontiguousarray(A.T), B, ta=1)
    assert np.array_equal(C_ref.view(np.uint64), C_st.view(np.uint64))


def test_static_scratch_refuses_sizes_beyond_its_array():
    plan = oz.Plan(16, 0, 8192, oz.OZ_ENGINE_AUTO)
    n = 2048
    assert plan.workspace_bytes(n, n, n) > oz.OZ_STATIC_SCRATCH_BYTES
    dummy = torch.zeros(1, dtype=torch.float64, device=DEV)
    st = oz.oz_dgemm_static(plan.handle, 0, 0, n, n, n, dummy.data_ptr(), n, dummy.data_ptr(), n, dummy.data_ptr(),
                            n, oz._stream_handle())
    assert st == oz.OZ_ERR_WORKSPACE
