// oz_host.cu -- the emulated product on host-resident operands, with the
// host<->device copies overlapped with the phases of neighbouring row chunks:
//
//   stream_h2d:  A_0 | B | A_1 | A_2 | ...            (each into a free A slot)
//   stream:      split A_0 | split B | split A_1, GEMMs_1(?), ... per chunk:
//                split A_i -> GEMMs_i -> reconstruct_i
//   stream_d2h:                      C_0 | C_1 | ...  (each after its chunk)
//
// Two A slots and two C slots are reused in turn; events order every reuse.
#include <stdint.h>
#include <string.h>

#include <vector>

#include "oz_internal.h"

namespace {

using oz::round_up;

struct HostLayout {
  int64_t chunk, chunk_pad, n_pad, k_pad;
  int64_t ldy;       // row pitch of the residue planes: n rounded up to 16 bytes
  size_t flag, s, t, colmax, b, a[2], c[2], u, v, y, total;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

bool host_layout(const oz_plan p, int64_t m, int64_t n, int64_t k, int64_t rows, HostLayout* L) {
  if (!p || m < 0 || n < 0 || k < 0 || rows < 0) return false;
  if (rows == 0) rows = round_up((m + 3) / 4 > 0 ? (m + 3) / 4 : 1, 256);
  if (rows > m && m > 0) rows = m;
  if (rows < 1) rows = 1;
  const int64_t elem = oz::engine_bf16(p->engine) ? 2 : 1;
  const int64_t nplanes = p->is_fp ? p->fp.nplanes : p->Q;
  const int64_t ybytes = p->is_fp ? 2 : 1;
  L->chunk = rows;
  L->chunk_pad = round_up(rows, oz::kPadRows);
  L->n_pad = round_up(n > 0 ? n : 1, oz::kPadRows);
  L->k_pad = round_up(k > 0 ? k : 1, p->is_fp ? oz::fp_k_align(p->fp) : oz::kPadK);
  const int64_t row = p->is_fp ? oz::fp_row_bytes(p->fp, L->k_pad) : L->k_pad * elem;   // bytes per plane row
  size_t off = 0;
  L->flag = off; off = al(off + 16);
  L->s = off; off = al(off + 4 * (size_t)(m > 0 ? m : 1));
  L->t = off; off = al(off + 4 * (size_t)(n > 0 ? n : 1));
  L->colmax = off; off = al(off + 8 * (size_t)(n > 0 ? n : 1));
  L->b = off; off = al(off + 8 * (size_t)k * n);
  for (int i = 0; i < 2; ++i) { L->a[i] = off; off = al(off + 8 * (size_t)rows * k); }
  for (int i = 0; i < 2; ++i) { L->c[i] = off; off = al(off + 8 * (size_t)rows * n); }
  L->u = off; off = al(off + (size_t)nplanes * L->chunk_pad * row);
  L->v = off; off = al(off + (size_t)nplanes * L->n_pad * row);
  L->ldy = round_up(n > 0 ? n : 1, 16 / ybytes);
  L->y = off; off = al(off + (size_t)p->Q * rows * L->ldy * ybytes);
  L->total = off;
  return true;
}

}  // namespace

extern "C" size_t oz_host_workspace_bytes(oz_plan plan, int64_t m, int64_t n, int64_t k, int64_t rows) {
  HostLayout L;
  if (!host_layout(plan, m, n, k, rows, &L)) return 0;
  return L.total;
}

extern "C" oz_status oz_dgemm_host(oz_plan plan, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                   const double* B, int64_t ldb, double* C, int64_t ldc, int64_t rows,
                                   void* workspace, size_t workspace_bytes, void* stream, void* stream_h2d,
                                   void* stream_d2h) {
  if (!plan || m < 0 || n < 0 || k < 0 || rows < 0) return OZ_ERR_INVALID_ARG;
  if (plan->is_fp && !plan->d_words) return OZ_ERR_CUDA;
  if (lda < (k > 1 ? k : 1) || ldb < (n > 1 ? n : 1) || ldc < (n > 1 ? n : 1)) return OZ_ERR_INVALID_ARG;
  if (k > plan->k_max) return OZ_ERR_K_TOO_LARGE;
  if (stream == stream_h2d || stream == stream_d2h || stream_h2d == stream_d2h) return OZ_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return OZ_OK;
  if (!C || (k > 0 && (!A || !B))) return OZ_ERR_INVALID_ARG;
  HostLayout L;
  host_layout(plan, m, n, k, rows, &L);
  if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return OZ_ERR_WORKSPACE;
  cudaStream_t sc = static_cast<cudaStream_t>(stream);
  cudaStream_t sh = static_cast<cudaStream_t>(stream_h2d);
  cudaStream_t sd = static_cast<cudaStream_t>(stream_d2h);
  char* ws = static_cast<char*>(workspace);
  int32_t* flag = reinterpret_cast<int32_t*>(ws + L.flag);
  int32_t* s = reinterpret_cast<int32_t*>(ws + L.s);
  int32_t* t = reinterpret_cast<int32_t*>(ws + L.t);
  uint64_t* colmax = reinterpret_cast<uint64_t*>(ws + L.colmax);
  double* Bd = reinterpret_cast<double*>(ws + L.b);
  double* Ad[2] = {reinterpret_cast<double*>(ws + L.a[0]), reinterpret_cast<double*>(ws + L.a[1])};
  double* Cd[2] = {reinterpret_cast<double*>(ws + L.c[0]), reinterpret_cast<double*>(ws + L.c[1])};
  void* U = ws + L.u;
  void* V = ws + L.v;
  uint8_t* Y = reinterpret_cast<uint8_t*>(ws + L.y);
  const OzTables& T = plan->tab;
  const OzFpTables& F = plan->fp;
  const bool fp = plan->is_fp != 0;
  const int bf16 = oz::engine_bf16(plan->engine);
  uint8_t* U8 = static_cast<uint8_t*>(U);
  uint8_t* V8 = static_cast<uint8_t*>(V);
  uint16_t* Y16 = reinterpret_cast<uint16_t*>(Y);
  const int64_t nchunks = (m + L.chunk - 1) / L.chunk;

  // events: start, B ready, A slot ready/free, C slot ready/free, end of both copy streams
  std::vector<cudaEvent_t> evs;
  auto mk = [&](cudaEvent_t* e) {
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return false;
    evs.push_back(*e);
    return true;
  };
  auto cleanup = [&]() {
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
  };
  cudaEvent_t ev_start, ev_b, ev_a_ready[2], ev_a_free[2], ev_c_ready[2], ev_c_free[2], ev_h_end, ev_d_end;
  bool ok = mk(&ev_start) && mk(&ev_b) && mk(&ev_h_end) && mk(&ev_d_end);
  for (int i = 0; i < 2 && ok; ++i) ok = mk(&ev_a_ready[i]) && mk(&ev_a_free[i]) && mk(&ev_c_ready[i]) && mk(&ev_c_free[i]);
  if (!ok) { cleanup(); return OZ_ERR_CUDA; }

  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess && r != cudaSuccess) e = r; };
  // the copy streams start after the work already queued on `stream`
  chk(cudaEventRecord(ev_start, sc));
  chk(cudaStreamWaitEvent(sh, ev_start, 0));
  chk(cudaStreamWaitEvent(sd, ev_start, 0));
  chk(cudaMemsetAsync(flag, 0, 16, sc));

  auto copy_a = [&](int64_t ci) {
    const int slot = (int)(ci & 1);
    const int64_t r0 = ci * L.chunk, nr = (m - r0) < L.chunk ? (m - r0) : L.chunk;
    if (ci >= 2) chk(cudaStreamWaitEvent(sh, ev_a_free[slot], 0));     // split of chunk ci-2 done
    if (k > 0)
      chk(cudaMemcpy2DAsync(Ad[slot], (size_t)k * 8, A + r0 * lda, (size_t)lda * 8, (size_t)k * 8, (size_t)nr,
                            cudaMemcpyHostToDevice, sh));
    chk(cudaEventRecord(ev_a_ready[slot], sh));
  };

  // A_0 first so that its split overlaps the copy of B
  copy_a(0);
  if (k > 0)
    chk(cudaMemcpy2DAsync(Bd, (size_t)n * 8, B, (size_t)ldb * 8, (size_t)n * 8, (size_t)k, cudaMemcpyHostToDevice, sh));
  chk(cudaEventRecord(ev_b, sh));
  if (nchunks > 1) copy_a(1);

  for (int64_t ci = 0; ci < nchunks && e == cudaSuccess; ++ci) {
    const int slot = (int)(ci & 1);
    const int64_t r0 = ci * L.chunk, nr = (m - r0) < L.chunk ? (m - r0) : L.chunk;
    chk(cudaStreamWaitEvent(sc, ev_a_ready[slot], 0));
    if (k > 0) {
      chk(fp ? oz::launch_split_fp(T, F, 1, nr, k, Ad[slot], k, L.chunk_pad, L.k_pad, s + r0, U8, flag, nullptr, sc)
             : oz::launch_split_rows(T, nr, k, Ad[slot], k, L.chunk_pad, L.k_pad, s + r0, U, bf16, flag, sc));
      chk(cudaEventRecord(ev_a_free[slot], sc));
      if (ci + 2 < nchunks) copy_a(ci + 2);
      if (ci == 0) {
        chk(cudaStreamWaitEvent(sc, ev_b, 0));
        chk(fp ? oz::launch_split_fp(T, F, 0, n, k, Bd, n, L.n_pad, L.k_pad, t, V8, flag, colmax, sc)
               : oz::launch_split_cols(T, n, k, Bd, n, L.n_pad, L.k_pad, t, V, bf16, flag, colmax, sc));
      }
      chk(fp     ? oz::launch_gemm_fp(F, nr, n, L.chunk_pad, L.n_pad, L.k_pad, U8, V8, Y16, L.ldy, 0, flag, sc)
          : plan->engine == OZ_ENGINE_TC1
              ? oz::launch_gemm_tc_single(T, nr, n, L.chunk_pad, L.n_pad, L.k_pad, U, V, Y, L.ldy, 0, flag, sc)
          : bf16 ? oz::launch_gemm_tc(T, nr, n, L.chunk_pad, L.n_pad, L.k_pad, U, V, Y, L.ldy, 0, flag, sc)
                 : oz::launch_gemm_imma(T, nr, n, L.k_pad, static_cast<const int8_t*>(U), L.chunk_pad * L.k_pad,
                                        static_cast<const int8_t*>(V), L.n_pad * L.k_pad, Y, L.ldy, 0, sc));
    } else {
      chk(cudaEventRecord(ev_a_free[slot], sc));
      if (ci + 2 < nchunks) copy_a(ci + 2);
    }
    if (ci >= 2) chk(cudaStreamWaitEvent(sc, ev_c_free[slot], 0));      // copy-back of chunk ci-2 done
    if (k > 0)
      chk(fp ? oz::launch_reconstruct16(T, nr, n, Y16, L.ldy, s + r0, t, Cd[slot], n, sc)
             : oz::launch_reconstruct(T, nr, n, Y, L.ldy, s + r0, t, Cd[slot], n, sc));
    else chk(cudaMemsetAsync(Cd[slot], 0, (size_t)nr * n * 8, sc));
    chk(cudaEventRecord(ev_c_ready[slot], sc));
    chk(cudaStreamWaitEvent(sd, ev_c_ready[slot], 0));
    chk(cudaMemcpy2DAsync(C + r0 * ldc, (size_t)ldc * 8, Cd[slot], (size_t)n * 8, (size_t)n * 8, (size_t)nr,
                          cudaMemcpyDeviceToHost, sd));
    chk(cudaEventRecord(ev_c_free[slot], sd));
  }
  // `stream` finishes only after both copy streams
  chk(cudaEventRecord(ev_h_end, sh));
  chk(cudaEventRecord(ev_d_end, sd));
  chk(cudaStreamWaitEvent(sc, ev_h_end, 0));
  chk(cudaStreamWaitEvent(sc, ev_d_end, 0));
  cleanup();
  return e == cudaSuccess ? OZ_OK : OZ_ERR_CUDA;
}
