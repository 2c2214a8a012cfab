// oz_static.cu -- oz_dgemm_static: oz_dgemm with its workspace in a scratch
// array built into the library, for callers that cannot allocate device
// memory (a BLAS-style dgemm interface has no workspace argument; some host
// programs own every device allocation themselves). The paper has no
// counterpart to this entry point. oz_static_query_status reads the status
// word the last such product left in the array.
#include <stdint.h>

#include "oz_internal.h"

namespace {

// One array per GPU that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_oz_scratch[OZ_STATIC_SCRATCH_BYTES];

// In host code g_oz_scratch names a host-side stand-in, not device memory.
// The device address comes from cudaGetSymbolAddress, looked up on every call
// with the caller's device and context current: a __device__ symbol has its
// own address in each context, so an address kept from another context (or
// from before a cudaDeviceReset) could be stale. The lookup is a host call.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_oz_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" oz_status oz_dgemm_static(oz_plan plan, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k,
                                     const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                                     int64_t ldc, void* stream) {
  if (!plan || m < 0 || n < 0 || k < 0) return OZ_ERR_INVALID_ARG;
  const size_t need = oz_workspace_bytes(plan, m, n, k);
  if (need == 0) return OZ_ERR_INVALID_ARG;
  if (need > (size_t)OZ_STATIC_SCRATCH_BYTES) return OZ_ERR_WORKSPACE;
  if (m == 0 || n == 0) return oz_dgemm(plan, trans_a, trans_b, m, n, k, A, lda, B, ldb, C, ldc, nullptr, 0, stream);
  void* ws = nullptr;
  if (scratch_address(&ws) != cudaSuccess || !ws) return OZ_ERR_CUDA;
  // oz_dgemm clears the status word and the column-maximum words it reuses;
  // every plane and residue it reads was written earlier in the same call.
  return oz_dgemm(plan, trans_a, trans_b, m, n, k, A, lda, B, ldb, C, ldc, ws, (size_t)OZ_STATIC_SCRATCH_BYTES,
                  stream);
}

extern "C" oz_status oz_static_query_status(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return OZ_ERR_CUDA;
  // the status word is the first word of the workspace layout (oz_workspace_layout)
  int32_t flag = 0;
  if (cudaMemcpyFromSymbol(&flag, g_oz_scratch, sizeof flag, 0, cudaMemcpyDeviceToHost) != cudaSuccess)
    return OZ_ERR_CUDA;
  if (flag & 2) return OZ_ERR_CUDA;   // a bounded device wait ran out
  return (flag & 1) ? OZ_ERR_NONFINITE : OZ_OK;
}
