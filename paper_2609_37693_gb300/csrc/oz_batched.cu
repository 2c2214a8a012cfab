// oz_batched.cu -- many emulated products of uneven shapes in one call: the
// problems are spread over the caller's streams (largest first, each to the
// least-loaded stream) so that small products run side by side, with one
// workspace slice per stream, and the streams fork from and join back into
// streams[0] through events so that the batch captures into one CUDA graph.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "oz_internal.h"

namespace {

struct Assignment {
  std::vector<int> stream_of;   // problem -> stream
  std::vector<size_t> ws;       // stream -> largest workspace of its problems
};

bool assign(int count, const oz_plan* plans, const int64_t* mnk, int nstreams, Assignment* a) {
  if (count < 0 || nstreams < 1 || (count > 0 && (!plans || !mnk))) return false;
  a->stream_of.assign(count, 0);
  a->ws.assign(nstreams, 0);
  std::vector<int> order(count);
  std::vector<double> work(count);
  for (int i = 0; i < count; ++i) {
    const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
    if (!plans[i] || m < 0 || n < 0 || k < 0) return false;
    order[i] = i;
    // estimated cost: the Q low-precision products, plus the passes over the
    // operands and the output
    work[i] = (double)plans[i]->Q * ((double)m * n * (double)k + 64.0 * ((double)m * k + (double)k * n + (double)m * n));
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  std::vector<double> load(nstreams, 0.0);
  for (int idx : order) {
    int best = 0;
    for (int s = 1; s < nstreams; ++s)
      if (load[s] < load[best]) best = s;
    load[best] += work[idx];
    a->stream_of[idx] = best;
    const size_t w = oz_workspace_bytes(plans[idx], mnk[3 * idx], mnk[3 * idx + 1], mnk[3 * idx + 2]);
    a->ws[best] = std::max(a->ws[best], w);
  }
  return true;
}

size_t slice_bytes(const Assignment& a) {
  size_t mx = 0;
  for (size_t w : a.ws) mx = std::max(mx, w);
  return (mx + 255) & ~(size_t)255;
}

}  // namespace

extern "C" size_t oz_batched_workspace_bytes(int count, const oz_plan* plans, const int64_t* mnk, int nstreams) {
  Assignment a;
  if (!assign(count, plans, mnk, nstreams, &a)) return 0;
  return slice_bytes(a) * (size_t)nstreams;
}

extern "C" oz_status oz_dgemm_batched(int count, const oz_plan* plans, const int64_t* mnk, const int* trans,
                                      const double* const* A, const int64_t* lda, const double* const* B,
                                      const int64_t* ldb, double* const* C, const int64_t* ldc, void* workspace,
                                      size_t workspace_bytes, void* const* streams, int nstreams) {
  if (count == 0) return OZ_OK;
  if (count < 0 || nstreams < 1 || !streams || !A || !B || !C || !lda || !ldb || !ldc) return OZ_ERR_INVALID_ARG;
  Assignment a;
  if (!assign(count, plans, mnk, nstreams, &a)) return OZ_ERR_INVALID_ARG;
  const size_t slice = slice_bytes(a);
  if (!workspace || workspace_bytes < slice * (size_t)nstreams || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return OZ_ERR_WORKSPACE;
  // check every problem before anything launches
  for (int i = 0; i < count; ++i) {
    const int64_t m = mnk[3 * i], n = mnk[3 * i + 1], k = mnk[3 * i + 2];
    const int ta = trans ? trans[2 * i] : 0, tb = trans ? trans[2 * i + 1] : 0;
    if ((ta != 0 && ta != 1) || (tb != 0 && tb != 1)) return OZ_ERR_INVALID_ARG;
    const int64_t a_cols = ta ? m : k, b_cols = tb ? k : n;
    if (lda[i] < (a_cols > 1 ? a_cols : 1) || ldb[i] < (b_cols > 1 ? b_cols : 1) || ldc[i] < (n > 1 ? n : 1))
      return OZ_ERR_INVALID_ARG;
    if (k > plans[i]->k_max) return OZ_ERR_K_TOO_LARGE;
    if (m > 0 && n > 0 && (!C[i] || (k > 0 && (!A[i] || !B[i])))) return OZ_ERR_INVALID_ARG;
  }
  cudaStream_t s0 = static_cast<cudaStream_t>(streams[0]);
  std::vector<cudaEvent_t> ev(nstreams, nullptr);
  auto cleanup = [&]() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  };
  // fork: every stream waits for the work already queued on streams[0]
  for (int s = 0; s < nstreams; ++s)
    if (cudaEventCreateWithFlags(&ev[s], cudaEventDisableTiming) != cudaSuccess) { cleanup(); return OZ_ERR_CUDA; }
  if (nstreams > 1) {
    if (cudaEventRecord(ev[0], s0) != cudaSuccess) { cleanup(); return OZ_ERR_CUDA; }
    for (int s = 1; s < nstreams; ++s)
      if (cudaStreamWaitEvent(static_cast<cudaStream_t>(streams[s]), ev[0], 0) != cudaSuccess) {
        cleanup();
        return OZ_ERR_CUDA;
      }
  }
  oz_status st = OZ_OK;
  char* ws = static_cast<char*>(workspace);
  for (int i = 0; i < count && st == OZ_OK; ++i) {
    const int s = a.stream_of[i];
    const int ta = trans ? trans[2 * i] : 0, tb = trans ? trans[2 * i + 1] : 0;
    // several streams: the TC engine's GEMMs run with one CTA per tile, since
    // CTA-pair GEMMs of concurrent products were seen to stall one another
    st = oz::dgemm_run(plans[i], ta, tb, mnk[3 * i], mnk[3 * i + 1], mnk[3 * i + 2], A[i], lda[i], B[i], ldb[i],
                       C[i], ldc[i], ws + slice * (size_t)s, slice, streams[s], nstreams > 1);
  }
  // join: streams[0] waits for every other stream
  if (nstreams > 1) {
    for (int s = 1; s < nstreams; ++s) {
      cudaStream_t ss = static_cast<cudaStream_t>(streams[s]);
      if (cudaEventRecord(ev[s], ss) != cudaSuccess || cudaStreamWaitEvent(s0, ev[s], 0) != cudaSuccess) {
        if (st == OZ_OK) st = OZ_ERR_CUDA;
      }
    }
  }
  cleanup();
  return st;
}
