// oz_host.cu -- the emulated product on host-resident operands, with the
// host<->device copies overlapped with the phases. The output is cut into
// blocks of `rows` rows of A by `cols` columns of B (block (i, j)):
//
//   stream_h2d:  A_0 | B_0 | B_1 | ... | B_{J-1} | A_1 | A_2 | ...
//   stream:      split A_0 | split B_0, GEMMs (0,0), reconstruct (0,0) |
//                split B_1, GEMMs (0,1), reconstruct (0,1) | ... |
//                split A_1, GEMMs (1,0), reconstruct (1,0) | ...
//   stream_d2h:                          C(0,0) | C(0,1) | ...
//
// B_j (the columns of block column j, all k rows) is split once, when it
// arrives, into planes of its own; A_i is split when block row i starts.
// So the first GEMMs wait for one row chunk of A and one column chunk of B
// only, and the last copy back is one block. Two A slots and two C block
// slots are reused in turn; events order every reuse.
#include <stdint.h>
#include <string.h>

#include <vector>

#include "oz_internal.h"

namespace {

// The pipeline's events, created once per host thread and device and reused
// by every call from that thread: a call records each event and enqueues the
// waits on it before it returns, and a wait orders against the record made
// before it, so the next call may record the same events again while this
// call's work is still running. (Creating and destroying a dozen events per
// call put driver work on the host path of every product.)
struct EventPool {
  int device = -1;
  std::vector<cudaEvent_t> ev;
  void release() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
  }
  ~EventPool() { release(); }
};
thread_local EventPool t_events;

// At least `count` events of the current device, or nullptr.
std::vector<cudaEvent_t>* event_pool(size_t count) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (t_events.device != dev) {
    t_events.release();
    t_events.device = dev;
  }
  while (t_events.ev.size() < count) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    t_events.ev.push_back(e);
  }
  return &t_events.ev;
}

using oz::round_up;

struct HostLayout {
  int64_t rows, cols, chunk_pad, w_pad, k_pad, nbj;
  int64_t ldy;       // row pitch of the residue planes: n rounded up to 16 bytes
  size_t vplane;     // bytes of one column chunk's planes
  size_t flag, s, t, colmax, b, a[2], c[2], u, v, y, bt, total;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t default_edge(int64_t x) {
  const int64_t e = round_up((x + 3) / 4 > 0 ? (x + 3) / 4 : 1, 256);
  return e;
}

bool host_layout(const oz_plan p, int64_t m, int64_t n, int64_t k, int64_t rows, int64_t cols, HostLayout* L) {
  if (!p || m < 0 || n < 0 || k < 0 || rows < 0 || cols < 0) return false;
  if (rows == 0) rows = default_edge(m);
  if (cols == 0) cols = default_edge(n);
  if (rows > m && m > 0) rows = m;
  if (cols > n && n > 0) cols = n;
  if (rows < 1) rows = 1;
  if (cols < 1) cols = 1;
  const int64_t elem = oz::engine_bf16(p->engine) ? 2 : 1;
  const int64_t nplanes = p->is_fp ? p->fp.nplanes : p->Q;
  const int64_t ybytes = p->is_fp ? 2 : 1;
  L->rows = rows;
  L->cols = cols;
  L->chunk_pad = round_up(rows, oz::kPadRows);
  L->w_pad = round_up(cols, oz::kPadRows);
  L->k_pad = round_up(k > 0 ? k : 1, p->is_fp ? oz::fp_k_align(p->fp) : oz::kPadK);
  L->nbj = n > 0 ? (n + cols - 1) / cols : 1;
  const int64_t row = p->is_fp ? oz::fp_row_bytes(p->fp, L->k_pad) : L->k_pad * elem;   // bytes per plane row
  L->vplane = al((size_t)nplanes * L->w_pad * row);
  size_t off = 0;
  L->flag = off; off = al(off + 16);
  L->s = off; off = al(off + 4 * (size_t)(m > 0 ? m : 1));
  L->t = off; off = al(off + 4 * (size_t)(n > 0 ? n : 1));
  L->colmax = off; off = al(off + 8 * (size_t)(n > 0 ? n : 1));
  L->b = off; off = al(off + 8 * (size_t)k * n);
  for (int i = 0; i < 2; ++i) { L->a[i] = off; off = al(off + 8 * (size_t)rows * k); }
  for (int i = 0; i < 2; ++i) { L->c[i] = off; off = al(off + 8 * (size_t)rows * cols); }
  L->u = off; off = al(off + (size_t)nplanes * L->chunk_pad * row);
  L->v = off; off = al(off + L->vplane * (size_t)L->nbj);
  L->ldy = round_up(n > 0 ? n : 1, 16 / ybytes);
  L->y = off; off = al(off + (size_t)p->Q * rows * L->ldy * ybytes);
  // one column chunk of B transposed (cols x k doubles): its columns are
  // split as rows (int8 planes of the IMMA engine; bf16 planes are split from
  // the columns in place)
  L->bt = off; off = al(off + (p->is_fp || oz::engine_bf16(p->engine) ? 0 : 8 * (size_t)cols * k));
  L->total = off;
  return true;
}

}  // namespace

extern "C" size_t oz_host_workspace_bytes(oz_plan plan, int64_t m, int64_t n, int64_t k, int64_t rows,
                                          int64_t cols) {
  HostLayout L;
  if (!host_layout(plan, m, n, k, rows, cols, &L)) return 0;
  return L.total;
}

extern "C" oz_status oz_dgemm_host(oz_plan plan, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                   const double* B, int64_t ldb, double* C, int64_t ldc, int64_t rows, int64_t cols,
                                   void* workspace, size_t workspace_bytes, void* stream, void* stream_h2d,
                                   void* stream_d2h) {
  if (!plan || m < 0 || n < 0 || k < 0 || rows < 0 || cols < 0) return OZ_ERR_INVALID_ARG;
  if (plan->is_fp && !plan->d_words) return OZ_ERR_CUDA;
  if (lda < (k > 1 ? k : 1) || ldb < (n > 1 ? n : 1) || ldc < (n > 1 ? n : 1)) return OZ_ERR_INVALID_ARG;
  if (k > plan->k_max) return OZ_ERR_K_TOO_LARGE;
  if (stream == stream_h2d || stream == stream_d2h || stream_h2d == stream_d2h) return OZ_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return OZ_OK;
  if (!C || (k > 0 && (!A || !B))) return OZ_ERR_INVALID_ARG;
  HostLayout L;
  host_layout(plan, m, n, k, rows, cols, &L);
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
  uint8_t* Y = reinterpret_cast<uint8_t*>(ws + L.y);
  const OzTables& T = plan->tab;
  const OzFpTables& F = plan->fp;
  const bool fp = plan->is_fp != 0;
  const int bf16 = oz::engine_bf16(plan->engine);
  const int64_t ybytes = fp ? 2 : 1;
  const int64_t nbi = (m + L.rows - 1) / L.rows, nbj = L.nbj;
  auto vj = [&](int64_t j) { return static_cast<void*>(ws + L.v + L.vplane * (size_t)j); };

  // events: start, B_j ready, A slot ready/free, C slot ready/free, end of both copy streams
  std::vector<cudaEvent_t>* pool = event_pool((size_t)(11 + nbj));
  if (!pool) return OZ_ERR_CUDA;
  const cudaEvent_t* pe = pool->data();
  const cudaEvent_t ev_start = pe[0], ev_h_end = pe[1], ev_d_end = pe[2];
  const cudaEvent_t ev_a_ready[2] = {pe[3], pe[4]}, ev_a_free[2] = {pe[5], pe[6]};
  const cudaEvent_t ev_c_ready[2] = {pe[7], pe[8]}, ev_c_free[2] = {pe[9], pe[10]};
  const cudaEvent_t* ev_b = pe + 11;

  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess && r != cudaSuccess) e = r; };
  // the copy streams start after the work already queued on `stream`
  chk(cudaEventRecord(ev_start, sc));
  chk(cudaStreamWaitEvent(sh, ev_start, 0));
  chk(cudaStreamWaitEvent(sd, ev_start, 0));
  chk(cudaMemsetAsync(flag, 0, 16, sc));

  auto rows_of = [&](int64_t i) { return (m - i * L.rows) < L.rows ? (m - i * L.rows) : L.rows; };
  auto cols_of = [&](int64_t j) { return (n - j * L.cols) < L.cols ? (n - j * L.cols) : L.cols; };
  auto copy_a = [&](int64_t i) {
    const int slot = (int)(i & 1);
    if (i >= 2) chk(cudaStreamWaitEvent(sh, ev_a_free[slot], 0));     // split of chunk i-2 done
    if (k > 0)
      chk(cudaMemcpy2DAsync(Ad[slot], (size_t)k * 8, A + i * L.rows * lda, (size_t)lda * 8, (size_t)k * 8,
                            (size_t)rows_of(i), cudaMemcpyHostToDevice, sh));
    chk(cudaEventRecord(ev_a_ready[slot], sh));
  };

  // A_0, then B column chunk by column chunk, then A_1: the first GEMMs need
  // only A_0 and B_0
  copy_a(0);
  for (int64_t j = 0; j < nbj; ++j) {
    const int64_t c0 = j * L.cols;
    if (k > 0)
      chk(cudaMemcpy2DAsync(Bd + c0, (size_t)n * 8, B + c0, (size_t)ldb * 8, (size_t)cols_of(j) * 8, (size_t)k,
                            cudaMemcpyHostToDevice, sh));
    chk(cudaEventRecord(ev_b[j], sh));
  }
  if (nbi > 1) copy_a(1);

  // B_j (k x nc, row pitch n): bf16 planes split from its columns in place;
  // int8 planes from the rows of its transpose Bt
  double* Bt = reinterpret_cast<double*>(ws + L.bt);
  auto launch_split_b_chunk = [&](int64_t nc, int64_t c0, void* planes) {
    if (bf16) return oz::launch_split_cols(T, nc, k, Bd + c0, n, L.w_pad, L.k_pad, t + c0, planes, bf16, flag,
                                           colmax + c0, sc);
    cudaError_t r = oz::launch_transpose(k, nc, Bd + c0, n, Bt, sc);
    if (r != cudaSuccess) return r;
    return oz::launch_split_rows(T, nc, k, Bt, k, L.w_pad, L.k_pad, t + c0, planes, bf16, flag, sc);
  };

  int64_t blk = 0;   // block counter: C slot blk & 1
  for (int64_t i = 0; i < nbi && e == cudaSuccess; ++i) {
    const int slot = (int)(i & 1);
    const int64_t r0 = i * L.rows, nr = rows_of(i);
    chk(cudaStreamWaitEvent(sc, ev_a_ready[slot], 0));
    if (k > 0)
      chk(fp ? oz::launch_split_fp(T, F, 1, nr, k, Ad[slot], k, L.chunk_pad, L.k_pad, s + r0,
                                   static_cast<uint8_t*>(U), flag, nullptr, sc)
             : oz::launch_split_rows(T, nr, k, Ad[slot], k, L.chunk_pad, L.k_pad, s + r0, U, bf16, flag, sc));
    chk(cudaEventRecord(ev_a_free[slot], sc));
    if (i + 2 < nbi) copy_a(i + 2);
    for (int64_t j = 0; j < nbj && e == cudaSuccess; ++j, ++blk) {
      const int64_t c0 = j * L.cols, nc = cols_of(j);
      const int cs = (int)(blk & 1);
      uint8_t* Yj = Y + c0 * ybytes;
      if (k > 0) {
        if (i == 0) {
          chk(cudaStreamWaitEvent(sc, ev_b[j], 0));
          chk(fp ? oz::launch_split_fp(T, F, 0, nc, k, Bd + c0, n, L.w_pad, L.k_pad, t + c0,
                                       static_cast<uint8_t*>(vj(j)), flag, colmax + c0, sc)
                 : launch_split_b_chunk(nc, c0, vj(j)));
        }
        chk(fp ? oz::launch_gemm_fp(F, nr, nc, L.chunk_pad, L.w_pad, L.k_pad, static_cast<const uint8_t*>(U),
                                    static_cast<const uint8_t*>(vj(j)), reinterpret_cast<uint16_t*>(Yj), L.ldy, 0,
                                    flag, sc)
            : plan->engine == OZ_ENGINE_TC1
                ? oz::launch_gemm_tc_single(T, nr, nc, L.chunk_pad, L.w_pad, L.k_pad, U, vj(j), Yj, L.ldy, 0, flag,
                                            sc)
            : bf16 ? oz::launch_gemm_tc(T, nr, nc, L.chunk_pad, L.w_pad, L.k_pad, U, vj(j), Yj, L.ldy, 0, flag, sc)
                   : oz::launch_gemm_imma(T, nr, nc, L.k_pad, static_cast<const int8_t*>(U), L.chunk_pad * L.k_pad,
                                          static_cast<const int8_t*>(vj(j)), L.w_pad * L.k_pad, Yj, L.ldy, 0, sc));
      } else if (i == 0) {
        chk(cudaStreamWaitEvent(sc, ev_b[j], 0));
      }
      if (blk >= 2) chk(cudaStreamWaitEvent(sc, ev_c_free[cs], 0));      // copy-back of block blk-2 done
      if (k > 0)
        chk(fp ? oz::launch_reconstruct16(T, nr, nc, reinterpret_cast<const uint16_t*>(Yj), L.ldy, s + r0, t + c0,
                                          Cd[cs], nc, sc)
               : oz::launch_reconstruct(T, nr, nc, Yj, L.ldy, s + r0, t + c0, Cd[cs], nc, sc));
      else
        chk(cudaMemsetAsync(Cd[cs], 0, (size_t)nr * nc * 8, sc));
      chk(cudaEventRecord(ev_c_ready[cs], sc));
      chk(cudaStreamWaitEvent(sd, ev_c_ready[cs], 0));
      chk(cudaMemcpy2DAsync(C + r0 * ldc + c0, (size_t)ldc * 8, Cd[cs], (size_t)nc * 8, (size_t)nc * 8, (size_t)nr,
                            cudaMemcpyDeviceToHost, sd));
      chk(cudaEventRecord(ev_c_free[cs], sd));
    }
  }
  // `stream` finishes only after both copy streams
  chk(cudaEventRecord(ev_h_end, sh));
  chk(cudaEventRecord(ev_d_end, sd));
  chk(cudaStreamWaitEvent(sc, ev_h_end, 0));
  chk(cudaStreamWaitEvent(sc, ev_d_end, 0));
  return e == cudaSuccess ? OZ_OK : OZ_ERR_CUDA;
}
