// oz_selftest.cu -- a check of the failure path every GEMM kernel relies on:
// the bounded mbarrier wait of oz_sync.cuh. One thread waits on a barrier of
// its own block. With `arrive` it arrives first, so the wait completes; without,
// nothing ever arrives, the wait runs out after about 2 s of %globaltimer,
// records bit 1 in the status word, and the kernel returns, so the context
// stays usable. No memory but the block's shared memory and the status word
// is touched.
#include <stdint.h>

#include "oz_internal.h"
#include "oz_sync.cuh"

namespace oz {
namespace {

__global__ void bounded_wait_kernel(int32_t* status, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive(b);
    if (mbar_wait(b, 0, reinterpret_cast<volatile int*>(&abort_flag), status)) atomicOr(status, 4);
  }
}

}  // namespace
}  // namespace oz

extern "C" oz_status oz_selftest_bounded_wait(int arrive, int32_t* status, void* stream) {
  if (!status) return OZ_ERR_INVALID_ARG;
  oz::bounded_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(status, arrive ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? OZ_OK : OZ_ERR_CUDA;
}
