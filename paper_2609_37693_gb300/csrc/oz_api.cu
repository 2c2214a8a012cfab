// oz_api.cu -- the C ABI entry points that run the phases (declared in
// include/oz.h): argument checks, the workspace layout, and the launch order
// Scale+Reduce (A), Scale+Reduce (B), GEMMs+Epilogue, Reconstruct of
// Sec. "Structure". Every call is asynchronous on the caller's stream and
// allocates nothing.
#include <stdint.h>
#include <string.h>

#include "oz_internal.h"

namespace {

using oz::round_up;

struct Layout {
  int64_t m_pad, n_pad, k_pad;
  int64_t ldy;       // row pitch of the residue planes Y: n rounded up to 16 bytes
  size_t flag, s, t, colmax, u, v, y, bt, total;
  oz::KSplit split;  // split-K of the TC GEMM (nsplit sets of residues, ysplit bytes apart)
  size_t ysplit;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// allow_split: reserve the residue sets of a split-K GEMM (oz_dgemm on a TC
// engine with too few output tiles for the GPU); a blocked call does not split.
bool make_layout(const oz_plan p, int64_t m, int64_t n, int64_t k, Layout* L, bool allow_split = true) {
  if (!p || m < 0 || n < 0 || k < 0) return false;
  const int64_t elem = oz::engine_bf16(p->engine) ? 2 : 1;     // bf16 planes; int8 residues or float codes
  const int64_t nplanes = p->is_fp ? p->fp.nplanes : p->Q;
  const int64_t ybytes = p->is_fp ? 2 : 1;                    // 16-bit digits for moduli above 255
  L->m_pad = round_up(m > 0 ? m : 1, oz::kPadRows);
  L->n_pad = round_up(n > 0 ? n : 1, oz::kPadRows);
  L->k_pad = round_up(k > 0 ? k : 1, p->is_fp ? oz::fp_k_align(p->fp) : oz::kPadK);
  const int64_t row = p->is_fp ? oz::fp_row_bytes(p->fp, L->k_pad) : L->k_pad * elem;   // bytes per plane row
  size_t off = 0;
  L->flag = off; off = align256(off + 16);
  L->s = off; off = align256(off + 4 * (size_t)m);
  L->t = off; off = align256(off + 4 * (size_t)n);
  L->colmax = off; off = align256(off + 8 * (size_t)(m > n ? m : n));
  L->u = off; off = align256(off + (size_t)nplanes * L->m_pad * row);
  L->v = off; off = align256(off + (size_t)nplanes * L->n_pad * row);
  L->ldy = round_up(n > 0 ? n : 1, 16 / ybytes);
  L->split = {1, (int)(L->k_pad / 64)};
  if (allow_split && !p->is_fp && oz::engine_bf16(p->engine) && m > 0 && n > 0 && k > 0) {
    const bool pairs = p->engine == OZ_ENGINE_TC;
    const int64_t tm = pairs ? 256 : 128;
    const int64_t tiles = (int64_t)p->Q * ((m + tm - 1) / tm) * ((n + 255) / 256);
    L->split = oz::ksplit_for(L->k_pad / 64, tiles, pairs ? oz::kPairWorkers : oz::kCtaWorkers);
  }
  L->ysplit = align256((size_t)p->Q * m * L->ldy * ybytes);
  L->y = off; off = align256(off + L->ysplit * L->split.nsplit);
  // B^T (n x k doubles): the IMMA engine's split takes B's columns as rows of
  // its transpose (the bf16 planes are split from B's columns directly)
  L->bt = off; off = align256(off + (p->is_fp || elem == 2 ? 0 : 8 * (size_t)n * k));
  L->total = off;
  return true;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

oz_status cuda_status(cudaError_t e) { return e == cudaSuccess ? OZ_OK : OZ_ERR_CUDA; }

}  // namespace

extern "C" size_t oz_workspace_bytes(oz_plan plan, int64_t m, int64_t n, int64_t k) {
  Layout L;
  if (!make_layout(plan, m, n, k, &L)) return 0;
  return L.total;
}

extern "C" oz_status oz_workspace_layout(oz_plan plan, int64_t m, int64_t n, int64_t k, int64_t* out) {
  Layout L;
  if (!out || !make_layout(plan, m, n, k, &L)) return OZ_ERR_INVALID_ARG;
  const size_t v[7] = {L.flag, L.s, L.t, L.colmax, L.u, L.v, L.y};
  for (int i = 0; i < 7; ++i) out[i] = (int64_t)v[i];
  out[7] = L.m_pad;
  out[8] = L.n_pad;
  out[9] = L.k_pad;
  out[10] = (int64_t)L.bt;
  return OZ_OK;
}

extern "C" oz_status oz_transpose(int64_t rows, int64_t cols, const double* X, int64_t ld, double* Y, void* stream) {
  if (rows < 0 || cols < 0 || ld < (cols > 1 ? cols : 1)) return OZ_ERR_INVALID_ARG;
  if (rows == 0 || cols == 0) return OZ_OK;
  if (!X || !Y || !aligned(X, 8) || !aligned(Y, 8)) return OZ_ERR_INVALID_ARG;
  return cuda_status(oz::launch_transpose(rows, cols, X, ld, Y, static_cast<cudaStream_t>(stream)));
}

extern "C" oz_status oz_plane_geometry(oz_plan plan, int64_t k_pad, int64_t* k_align, int64_t* row_bytes) {
  if (!plan || k_pad < 0) return OZ_ERR_INVALID_ARG;
  if (k_align) *k_align = plan->is_fp ? oz::fp_k_align(plan->fp) : oz::kPadK;
  if (row_bytes)
    *row_bytes = plan->is_fp ? oz::fp_row_bytes(plan->fp, k_pad) : k_pad * (oz::engine_bf16(plan->engine) ? 2 : 1);
  return OZ_OK;
}

namespace oz {

// oz_dgemm with one option: single_cta runs the TC engine's GEMM with one CTA
// per tile (no CTA pairs), for callers that run several products at once on
// different streams (oz_dgemm_batched).
oz_status dgemm_run(oz_plan plan, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k, const double* A,
                    int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, void* workspace,
                    size_t workspace_bytes, void* stream, bool single_cta) {
  if (!plan || m < 0 || n < 0 || k < 0) return OZ_ERR_INVALID_ARG;
  if ((trans_a != 0 && trans_a != 1) || (trans_b != 0 && trans_b != 1)) return OZ_ERR_INVALID_ARG;
  const int64_t a_cols = trans_a ? m : k, b_cols = trans_b ? k : n;
  if (lda < (a_cols > 1 ? a_cols : 1) || ldb < (b_cols > 1 ? b_cols : 1) || ldc < (n > 1 ? n : 1))
    return OZ_ERR_INVALID_ARG;
  if (k > plan->k_max) return OZ_ERR_K_TOO_LARGE;
  if (m == 0 || n == 0) return OZ_OK;
  if (!C || !aligned(C, 8)) return OZ_ERR_INVALID_ARG;
  if (k > 0 && (!A || !B || !aligned(A, 8) || !aligned(B, 8))) return OZ_ERR_INVALID_ARG;
  Layout L;
  make_layout(plan, m, n, k, &L);
  if (!workspace || workspace_bytes < L.total || !aligned(workspace, 256)) return OZ_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  int32_t* flag = reinterpret_cast<int32_t*>(ws + L.flag);
  cudaError_t e = cudaMemsetAsync(flag, 0, 16, st);
  if (e != cudaSuccess) return OZ_ERR_CUDA;
  if (k == 0) return cuda_status(cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)n * 8, (size_t)m, st));

  const OzTables& T = plan->tab;
  const int bf16 = oz::engine_bf16(plan->engine);
  int32_t* s = reinterpret_cast<int32_t*>(ws + L.s);
  int32_t* t = reinterpret_cast<int32_t*>(ws + L.t);
  uint64_t* colmax = reinterpret_cast<uint64_t*>(ws + L.colmax);
  void* U = ws + L.u;
  void* V = ws + L.v;
  uint8_t* Y = reinterpret_cast<uint8_t*>(ws + L.y);

  if (plan->is_fp) {
    if (!plan->d_words) return OZ_ERR_CUDA;
    const OzFpTables& F = plan->fp;
    uint8_t* U8 = static_cast<uint8_t*>(U);
    uint8_t* V8 = static_cast<uint8_t*>(V);
    uint16_t* Y16 = reinterpret_cast<uint16_t*>(Y);
    e = oz::launch_split_fp(T, F, !trans_a, m, k, A, lda, L.m_pad, L.k_pad, s, U8, flag, colmax, st);
    if (e != cudaSuccess) return OZ_ERR_CUDA;
    e = oz::launch_split_fp(T, F, trans_b, n, k, B, ldb, L.n_pad, L.k_pad, t, V8, flag, colmax, st);
    if (e != cudaSuccess) return OZ_ERR_CUDA;
    e = oz::launch_gemm_fp(F, m, n, L.m_pad, L.n_pad, L.k_pad, U8, V8, Y16, L.ldy, 0, flag, st);
    if (e != cudaSuccess) return OZ_ERR_CUDA;
    return cuda_status(oz::launch_reconstruct16(T, m, n, Y16, L.ldy, s, t, C, ldc, st));
  }
  // Scale + Reduce, A side: vectors are the rows of op(A).
  e = trans_a ? oz::launch_split_cols(T, m, k, A, lda, L.m_pad, L.k_pad, s, U, bf16, flag, colmax, st)
              : oz::launch_split_rows(T, m, k, A, lda, L.m_pad, L.k_pad, s, U, bf16, flag, st);
  if (e != cudaSuccess) return OZ_ERR_CUDA;
  // B side: vectors are the columns of op(B). Bf16 planes are split from
  // B's columns in place (column maxima, then tiles staged through shared
  // memory); for int8 planes B (k x n) is transposed first, so that its
  // columns are split as contiguous rows.
  if (trans_b) {
    e = oz::launch_split_rows(T, n, k, B, ldb, L.n_pad, L.k_pad, t, V, bf16, flag, st);
  } else if (bf16) {
    e = oz::launch_split_cols(T, n, k, B, ldb, L.n_pad, L.k_pad, t, V, bf16, flag, colmax, st);
  } else {
    double* Bt = reinterpret_cast<double*>(ws + L.bt);
    e = oz::launch_transpose(k, n, B, ldb, Bt, st);
    if (e == cudaSuccess) e = oz::launch_split_rows(T, n, k, Bt, k, L.n_pad, L.k_pad, t, V, bf16, flag, st);
  }
  if (e != cudaSuccess) return OZ_ERR_CUDA;
  // GEMMs + epilogue; with too few output tiles, the inner dimension split into
  // ranges whose residue sets are then added modulo m (the layout's split: a
  // TC plan forced onto one CTA per tile runs unsplit)
  const bool forced_single = single_cta && plan->engine == OZ_ENGINE_TC;
  const oz::KSplit split = forced_single ? oz::KSplit{1, 0} : L.split;
  e = (plan->engine == OZ_ENGINE_TC1 || forced_single)
          ? oz::launch_gemm_tc_single(T, m, n, L.m_pad, L.n_pad, L.k_pad, U, V, Y, L.ldy, 0, flag, st, split,
                                      (int64_t)L.ysplit)
      : bf16 ? oz::launch_gemm_tc(T, m, n, L.m_pad, L.n_pad, L.k_pad, U, V, Y, L.ldy, 0, flag, st, split,
                                  (int64_t)L.ysplit)
             : oz::launch_gemm_imma(T, m, n, L.k_pad, static_cast<const int8_t*>(U), L.m_pad * L.k_pad,
                                    static_cast<const int8_t*>(V), L.n_pad * L.k_pad, Y, L.ldy, 0, st);
  if (e != cudaSuccess) return OZ_ERR_CUDA;
  if (split.nsplit > 1) {
    e = oz::launch_combine_digits(T, m, L.ldy, Y, split.nsplit, (int64_t)L.ysplit, st);
    if (e != cudaSuccess) return OZ_ERR_CUDA;
  }
  // Reconstruct
  e = oz::launch_reconstruct(T, m, n, Y, L.ldy, s, t, C, ldc, st);
  return cuda_status(e);
}

}  // namespace oz

extern "C" oz_status oz_dgemm(oz_plan plan, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k,
                              const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                              void* workspace, size_t workspace_bytes, void* stream) {
  return oz::dgemm_run(plan, trans_a, trans_b, m, n, k, A, lda, B, ldb, C, ldc, workspace, workspace_bytes, stream,
                       false);
}

// ---------------------------------------------------------------------------
// Blocked call (Sec. "Slabs"): the shifts over the whole inner dimension, then
// per slab of k_slab terms the planes of that slab and the GEMMs, whose
// epilogues add the slab's digits into Y modulo m; one Reconstruct at the end.
// ---------------------------------------------------------------------------

extern "C" size_t oz_blocked_workspace_bytes(oz_plan plan, int64_t m, int64_t n, int64_t k_slab) {
  if (k_slab < 1) return 0;
  Layout L;
  if (!make_layout(plan, m, n, k_slab, &L, false)) return 0;
  return L.total;
}

extern "C" oz_status oz_dgemm_blocked(oz_plan plan, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k,
                                      int64_t k_slab, const double* A, int64_t lda, const double* B, int64_t ldb,
                                      double* C, int64_t ldc, void* workspace, size_t workspace_bytes, void* stream) {
  if (!plan || m < 0 || n < 0 || k < 0 || k_slab < 1) return OZ_ERR_INVALID_ARG;
  if ((trans_a != 0 && trans_a != 1) || (trans_b != 0 && trans_b != 1)) return OZ_ERR_INVALID_ARG;
  const int64_t a_cols = trans_a ? m : k, b_cols = trans_b ? k : n;
  if (lda < (a_cols > 1 ? a_cols : 1) || ldb < (b_cols > 1 ? b_cols : 1) || ldc < (n > 1 ? n : 1))
    return OZ_ERR_INVALID_ARG;
  if (k > plan->k_rec || k_slab > plan->k_acc) return OZ_ERR_K_TOO_LARGE;
  if (m == 0 || n == 0) return OZ_OK;
  if (!C || !aligned(C, 8)) return OZ_ERR_INVALID_ARG;
  if (k > 0 && (!A || !B || !aligned(A, 8) || !aligned(B, 8))) return OZ_ERR_INVALID_ARG;
  const int64_t kt = k_slab < k ? k_slab : (k > 0 ? k : 1);
  Layout L;
  make_layout(plan, m, n, kt, &L, false);
  if (!workspace || workspace_bytes < L.total || !aligned(workspace, 256)) return OZ_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  int32_t* flag = reinterpret_cast<int32_t*>(ws + L.flag);
  cudaError_t e = cudaMemsetAsync(flag, 0, 16, st);
  if (e != cudaSuccess) return OZ_ERR_CUDA;
  if (k == 0) return cuda_status(cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)n * 8, (size_t)m, st));

  const OzTables& T = plan->tab;
  const int bf16 = oz::engine_bf16(plan->engine);
  int32_t* s = reinterpret_cast<int32_t*>(ws + L.s);
  int32_t* t = reinterpret_cast<int32_t*>(ws + L.t);
  uint64_t* colmax = reinterpret_cast<uint64_t*>(ws + L.colmax);
  void* U = ws + L.u;
  void* V = ws + L.v;
  uint8_t* Y = reinterpret_cast<uint8_t*>(ws + L.y);
  if (plan->is_fp && !plan->d_words) return OZ_ERR_CUDA;

  // Scale over the whole inner dimension: rows of op(A), columns of op(B).
  e = trans_a ? oz::launch_shifts_cols(T.bits, m, k, A, lda, s, flag, colmax, st)
              : oz::launch_shifts_rows(T.bits, m, k, A, lda, s, flag, st);
  if (e != cudaSuccess) return OZ_ERR_CUDA;
  e = trans_b ? oz::launch_shifts_rows(T.bits, n, k, B, ldb, t, flag, st)
              : oz::launch_shifts_cols(T.bits, n, k, B, ldb, t, flag, colmax, st);
  if (e != cudaSuccess) return OZ_ERR_CUDA;

  const int64_t k_align = plan->is_fp ? oz::fp_k_align(plan->fp) : oz::kPadK;
  for (int64_t h0 = 0; h0 < k; h0 += kt) {
    const int64_t len = k - h0 < kt ? k - h0 : kt;
    const int64_t k_pad = round_up(len, k_align);
    // the slab: columns h0 .. h0 + len of op(A), rows of op(B)
    const double* As = trans_a ? A + h0 * lda : A + h0;
    const double* Bs = trans_b ? B + h0 : B + h0 * ldb;
    const int mode = h0 > 0 ? oz::kEpiAccumulate : 0;
    if (plan->is_fp) {
      const OzFpTables& F = plan->fp;
      uint8_t* U8 = static_cast<uint8_t*>(U);
      uint8_t* V8 = static_cast<uint8_t*>(V);
      e = oz::launch_split_fp(T, F, !trans_a, m, len, As, lda, L.m_pad, k_pad, s, U8, flag, colmax, st, true);
      if (e == cudaSuccess)
        e = oz::launch_split_fp(T, F, trans_b, n, len, Bs, ldb, L.n_pad, k_pad, t, V8, flag, colmax, st, true);
      if (e == cudaSuccess)
        e = oz::launch_gemm_fp(F, m, n, L.m_pad, L.n_pad, k_pad, U8, V8, reinterpret_cast<uint16_t*>(Y), L.ldy, mode,
                               flag, st);
    } else {
      e = trans_a ? oz::launch_split_cols(T, m, len, As, lda, L.m_pad, k_pad, s, U, bf16, flag, colmax, st, true)
                  : oz::launch_split_rows(T, m, len, As, lda, L.m_pad, k_pad, s, U, bf16, flag, st, true);
      if (e == cudaSuccess)
        e = trans_b ? oz::launch_split_rows(T, n, len, Bs, ldb, L.n_pad, k_pad, t, V, bf16, flag, st, true)
                    : oz::launch_split_cols(T, n, len, Bs, ldb, L.n_pad, k_pad, t, V, bf16, flag, colmax, st, true);
      if (e == cudaSuccess)
        e = plan->engine == OZ_ENGINE_TC1
                ? oz::launch_gemm_tc_single(T, m, n, L.m_pad, L.n_pad, k_pad, U, V, Y, L.ldy, mode, flag, st)
            : bf16 ? oz::launch_gemm_tc(T, m, n, L.m_pad, L.n_pad, k_pad, U, V, Y, L.ldy, mode, flag, st)
                   : oz::launch_gemm_imma(T, m, n, k_pad, static_cast<const int8_t*>(U), L.m_pad * k_pad,
                                          static_cast<const int8_t*>(V), L.n_pad * k_pad, Y, L.ldy, mode, st);
    }
    if (e != cudaSuccess) return OZ_ERR_CUDA;
  }
  e = plan->is_fp ? oz::launch_reconstruct16(T, m, n, reinterpret_cast<const uint16_t*>(Y), L.ldy, s, t, C, ldc, st)
                  : oz::launch_reconstruct(T, m, n, Y, L.ldy, s, t, C, ldc, st);
  return cuda_status(e);
}

extern "C" oz_status oz_query_status(void* workspace, void* stream) {
  if (!workspace) return OZ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return OZ_ERR_CUDA;
  int32_t flag = 0;
  if (cudaMemcpy(&flag, workspace, sizeof flag, cudaMemcpyDeviceToHost) != cudaSuccess) return OZ_ERR_CUDA;
  if (flag & 2) return OZ_ERR_CUDA;   // a bounded device wait ran out
  return (flag & 1) ? OZ_ERR_NONFINITE : OZ_OK;
}

extern "C" oz_status oz_split(oz_plan plan, int contiguous, int64_t nvec, int64_t len, const double* X, int64_t ld,
                              int64_t nvec_pad, int64_t k_pad, int32_t* shifts, void* planes, int32_t* flag,
                              uint64_t* colmax, void* stream) {
  if (!plan || nvec < 0 || len < 0) return OZ_ERR_INVALID_ARG;
  const int64_t k_align = plan->is_fp ? oz::fp_k_align(plan->fp) : oz::kPadK;
  if (nvec_pad < nvec || k_pad < len || nvec_pad % oz::kPadRows || k_pad % k_align || k_pad == 0)
    return OZ_ERR_INVALID_ARG;
  if (len > plan->k_max) return OZ_ERR_K_TOO_LARGE;
  if (nvec > 0 && (!shifts || (len > 0 && (!X || !aligned(X, 8))))) return OZ_ERR_INVALID_ARG;
  if (!planes || !aligned(planes, 16)) return OZ_ERR_INVALID_ARG;
  if (contiguous ? ld < (len > 1 ? len : 1) : ld < (nvec > 1 ? nvec : 1)) return OZ_ERR_INVALID_ARG;
  if (!contiguous && nvec > 0 && !colmax) return OZ_ERR_INVALID_ARG;
  const int bf16 = oz::engine_bf16(plan->engine);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->is_fp && !plan->d_words) return OZ_ERR_CUDA;
  if (plan->is_fp)
    return cuda_status(oz::launch_split_fp(plan->tab, plan->fp, contiguous, nvec, len, X, ld, nvec_pad, k_pad, shifts,
                                           static_cast<uint8_t*>(planes), flag, colmax, st));
  cudaError_t e = contiguous
                      ? oz::launch_split_rows(plan->tab, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, bf16,
                                              flag, st)
                      : oz::launch_split_cols(plan->tab, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, bf16,
                                              flag, colmax, st);
  return cuda_status(e);
}

extern "C" oz_status oz_residue_gemm(oz_plan plan, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad,
                                     int64_t k_pad, const void* U, const void* V, uint8_t* Y, int raw,
                                     int32_t* flag, void* stream) {
  if (!plan || m < 0 || n < 0) return OZ_ERR_INVALID_ARG;
  const int64_t k_align = plan->is_fp ? oz::fp_k_align(plan->fp) : oz::kPadK;
  if (m_pad < m || n_pad < n || m_pad % oz::kPadRows || n_pad % oz::kPadRows || k_pad <= 0 || k_pad % k_align)
    return OZ_ERR_INVALID_ARG;
  if (k_pad > oz::round_up(plan->k_max, k_align)) return OZ_ERR_K_TOO_LARGE;
  if (m == 0 || n == 0) return OZ_OK;
  if (!U || !V || !Y || !aligned(U, 16) || !aligned(V, 16)) return OZ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->is_fp)
    return cuda_status(oz::launch_gemm_fp(plan->fp, m, n, m_pad, n_pad, k_pad, static_cast<const uint8_t*>(U),
                                          static_cast<const uint8_t*>(V), reinterpret_cast<uint16_t*>(Y), n,
                                          raw ? 1 : 0, flag, st));
  if (plan->engine == OZ_ENGINE_TC)
    return cuda_status(oz::launch_gemm_tc(plan->tab, m, n, m_pad, n_pad, k_pad, U, V, Y, n, raw ? 1 : 0, flag, st));
  if (plan->engine == OZ_ENGINE_TC1)
    return cuda_status(
        oz::launch_gemm_tc_single(plan->tab, m, n, m_pad, n_pad, k_pad, U, V, Y, n, raw ? 1 : 0, flag, st));
  return cuda_status(oz::launch_gemm_imma(plan->tab, m, n, k_pad, static_cast<const int8_t*>(U), m_pad * k_pad,
                                          static_cast<const int8_t*>(V), n_pad * k_pad, Y, n, raw ? 1 : 0, st));
}

extern "C" oz_status oz_reconstruct(oz_plan plan, int64_t m, int64_t n, const uint8_t* Y, const int32_t* s,
                                    const int32_t* t, double* C, int64_t ldc, void* stream) {
  if (!plan || m < 0 || n < 0 || ldc < (n > 1 ? n : 1)) return OZ_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return OZ_OK;
  if (!Y || !s || !t || !C || !aligned(C, 8)) return OZ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->is_fp)
    return cuda_status(
        oz::launch_reconstruct16(plan->tab, m, n, reinterpret_cast<const uint16_t*>(Y), n, s, t, C, ldc, st));
  return cuda_status(oz::launch_reconstruct(plan->tab, m, n, Y, n, s, t, C, ldc, st));
}
