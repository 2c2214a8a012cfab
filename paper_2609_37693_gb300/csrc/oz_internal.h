// oz_internal.h -- plan constants shared by the host planner and the kernels.
#pragma once

#include <stdint.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/oz.h"

#define OZ_MAX_LIMBS 6     // 32-bit limbs of the CRT sum: Q P < 2^192 for Q <= 20
#define OZ_TABLE_CAP 32    // moduli a constant table can hold (INT8 plans use at most 20)
static_assert(OZ_TABLE_CAP == OZ_MAX_CHANNELS, "a float configuration's channels fill a table");
#define OZ_RG_MAX 8        // groups of the byte-digit reconstruct (Q <= 16 gives at most 6)

// Everything a kernel needs about a configuration. Passed by value as a kernel
// parameter, so it lives in the constant bank and every access indexed by a
// compile-time or warp-uniform modulus index is a uniform load.
struct OzTables {
  int Q;                                  // number of moduli (one GEMM each)
  int bits;                               // beta: |A'| < 2^beta
  int limbs;                              // 32-bit limbs for X in the reconstruct phase
  int pad_;
  uint32_t m[OZ_TABLE_CAP];              // moduli, decreasing
  uint32_t magic[OZ_TABLE_CAP];          // floor(2^32 / m), Barrett constant
  uint32_t inv[OZ_TABLE_CAP];            // (P/m)^-1 mod m: CRT coefficient
  float invm[OZ_TABLE_CAP];              // 1/m rounded to fp32: quotient estimate
  float mf[OZ_TABLE_CAP];                // m as fp32
  float c13f[4][OZ_TABLE_CAP];           // 2^(22 + 13 i) mod m, i = 0..3, each as the
                                          // representative nearest zero (|c| <= 119): the
                                          // split's pieces above its first 22 bits
  float c12f[6][OZ_TABLE_CAP];           // 2^(22 + 12 i) mod m, i = 0..5, nearest zero: the
                                          // 12-bit pieces of widened operands (beta > 64)
  float halfm[OZ_TABLE_CAP];             // m / 2 for an even m (the split maps +m/2 to -m/2)
  uint32_t P[OZ_MAX_LIMBS];               // P = product of the moduli, 32-bit limbs
  // Moduli taken in pairs (a, b) = (2p, 2p+1) for the reconstruct phase; an odd
  // Q ends with a pair whose second modulus is 1 (digit 0).
  int npairs;
  uint32_t pa[(OZ_TABLE_CAP + 1) / 2];   // m_a
  uint32_t pb[(OZ_TABLE_CAP + 1) / 2];   // m_b (1 for a lone last modulus)
  float pinv[(OZ_TABLE_CAP + 1) / 2];    // 1 / (m_a m_b) rounded to fp32
  uint32_t Np[(OZ_TABLE_CAP + 1) / 2][OZ_MAX_LIMBS];  // P / (m_a m_b), 32-bit limbs
  // Moduli in groups for the reconstruct of byte digits (Q <= 16): rg_nt
  // triples, then rg_np2 pairs or rg_nq4 quads, over consecutive moduli. A
  // group g of moduli M_g = prod m_q contributes t_g = sum_q y_q (M_g / m_q)
  // (below (size) M_g; a quad reduces each of its pairs first, t_g < 2 M_g)
  // times N_g = P / M_g to the CRT sum. rg_nt = rg_np2 = rg_nq4 = 0: not
  // available (the pairs above serve).
  int rg_nt, rg_np2, rg_nq4;
  uint32_t rg_w0[OZ_RG_MAX], rg_w1[OZ_RG_MAX];   // dp2a weights: two 16-bit per word
  uint32_t rg_m2a[OZ_RG_MAX], rg_m2b[OZ_RG_MAX]; // quad: the products of its two pairs
  uint32_t rg_N[OZ_RG_MAX][4];                   // N_g = P / M_g, 32-bit limbs
  float rg_invM[OZ_RG_MAX];                      // 1 / M_g rounded to fp32 (S / P = sum_g t_g / M_g)
};

// A low-precision float configuration (Sec. "Forms and Channels"): channels
// (a modulus with a form), their planes and GEMMs. Plane p of an operand
// holds, for every entry, the code of the format value the form's table
// assigns to the entry's class modulo its channel's modulus.
#define OZ_MAX_FP_GEMMS 128
#define OZ_MAX_FP_PLANES 96
struct OzFpTables {
  int fmt;                                // oz_format
  int e2;                                 // 2 e_S: an accumulator holds W 2^-e2 exactly
  int code_bits;                          // 8, 6 or 4: width of a code. 6-bit codes are packed 16
                                          // to a 16-byte chunk (bytes 12..15 unused); 4-bit codes
                                          // two to a byte, densely (block-scaled FP4 operands)
  int nch, ngemm, nplanes;
  int ch_gemm0[OZ_TABLE_CAP], ch_ngemm[OZ_TABLE_CAP];
  int ch_plane0[OZ_TABLE_CAP], ch_nplanes[OZ_TABLE_CAP];
  uint32_t m[OZ_TABLE_CAP];               // channel moduli (also in OzTables::m)
  uint32_t magic[OZ_TABLE_CAP];           // floor(2^32 / m)
  uint32_t c16[OZ_TABLE_CAP], c32[OZ_TABLE_CAP], c48[OZ_TABLE_CAP];  // 2^16k mod m
  uint32_t c64[OZ_TABLE_CAP];             // 2^64 mod m (widened budgets, beta > 64)
  uint32_t inv[OZ_TABLE_CAP];             // (P/m)^-1 mod m
  float mf[OZ_TABLE_CAP], invm[OZ_TABLE_CAP];
  uint8_t g_pa[OZ_MAX_FP_GEMMS], g_pb[OZ_MAX_FP_GEMMS];  // planes of GEMM g
  uint8_t g_ch[OZ_MAX_FP_GEMMS];          // channel of GEMM g
  float g_lam[OZ_MAX_FP_GEMMS];           // its weight lambda reduced into [0, m)
  uint32_t plane_off[OZ_MAX_FP_PLANES];   // offset of the plane's value table (host copy)
  uint32_t plane_ch[OZ_MAX_FP_PLANES];    // channel of plane p
  uint32_t ch_woff[OZ_TABLE_CAP];         // offset of the channel's code words
  // device: per channel 2 m words; word i < m is class i, word m + i is class
  // (m - i) mod m (the class of -x when x has class i); byte q of a word is
  // the code of the channel's plane q
  const uint32_t* words;
};

struct oz_plan_s {
  int Q;             // INT8: moduli = GEMMs; float formats: channels
  int bits;
  int engine;        // resolved engine (never AUTO)
  int64_t k_max;     // min(k_acc, k_rec): the largest K of one accumulation (eq. caps)
  int64_t k_acc;     // accumulation cap: the largest slab a blocked call may take
  int64_t k_rec;     // window cap (eq. ov-crtgen): the largest K of a blocked call
  OzTables tab;      // moduli and CRT constants
  int is_fp;
  int gemms;         // low-precision GEMMs per product
  int fp_form[OZ_TABLE_CAP], fp_base[OZ_TABLE_CAP];
  int64_t fp_kcfg;   // inner dimension the configuration was built for
  OzFpTables fp;
  uint32_t* d_words; // device copy of the code words (owned)
  int16_t* h_values; // host copy of the plane values, one table per plane (owned)
  size_t values_len;
};

// One product of a grouped call (oz_group_create): its operands, its part of
// the workspace and, per phase, the first block (or unit) of the group's
// launch that belongs to it. Device memory, aligned as its tensor maps
// require (128 bytes; the table starts on a 256-byte boundary).
struct OzGroupProblem {
  CUtensorMap mapA, mapB;            // residue planes of A and B (TMA, GEMM phase)
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int64_t m, n, k, m_pad, n_pad, k_pad, ldy;
  void* U;
  void* V;
  uint8_t* Y;
  int32_t* s;
  int32_t* t;
  uint64_t* colmax;
  int32_t* flag;
  int64_t rows_begin;   // split of A: one block per row of m_pad
  int64_t cm_begin;     // column maxima of B: ceil(n/32) * ceil(k/256) blocks
  int64_t sh_begin;     // shifts of B: ceil(n/256) blocks
  int64_t sc_begin;     // split of B: (n_pad/32) * (k_pad/64) blocks
  int64_t unit_begin;   // GEMMs: Q * tiles_m * tiles_n units
  int64_t rec_begin;    // reconstruct: m * ceil(n/1024) blocks
  int tiles_m, tiles_n, kblocks;
  int rec_tpr;          // reconstruct: threads per row chunk (8..32), 256 / rec_tpr rows per block, each
                        // thread 8 entries (the groups' kernel) or 4 (the pairs')
};

// the problem whose range [begin, next begin) holds index x (probs sorted by begin)
template <typename F>
__device__ __forceinline__ int group_find(const OzGroupProblem* probs, int count, int64_t x, F begin) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin(probs[mid]) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

namespace oz {

// Barrett reduction of y < 2^32 by m (2 <= m < 2^16) with magic = floor(2^32/m).
// q = floor(y * magic / 2^32) is floor(y/m) or one less, so one correction suffices.
__device__ __forceinline__ uint32_t mod_barrett(uint32_t y, uint32_t m, uint32_t magic) {
  uint32_t q = __umulhi(y, magic);
  uint32_t r = y - q * m;
  return r >= m ? r - m : r;
}

// Layout sizes shared by host and kernels.
constexpr int kTileM = 128;       // M tile of the GEMM engines; m_pad is a multiple of kPadRows
constexpr int kPadRows = 256;     // row padding of the residue planes
constexpr int kPadK = 128;        // k padding of the residue planes (entries)

// Epilogue modes of the GEMM launchers (their `raw` argument, a bit set).
constexpr int kEpiRaw = 1;         // store W mod m in [0, m) instead of the CRT digit
constexpr int kEpiAccumulate = 2;  // add the slab's value into the one already in Y, modulo m

// oz_dgemm with the TC engine's GEMM optionally forced onto one CTA per tile
// (oz_api.cu): products that run concurrently on several streams use it.
oz_status dgemm_run(oz_plan plan, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k, const double* A,
                    int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, void* workspace,
                    size_t workspace_bytes, void* stream, bool single_cta);

// Engines that hold the INT8 residues in BF16 planes.
inline bool engine_bf16(int e) { return e == OZ_ENGINE_TC || e == OZ_ENGINE_TC1; }

// Split-K of a TC-engine product: the inner dimension's kblocks k-blocks (64
// entries each) cut into nsplit ranges of kbps k-blocks, whole 1024-term slabs
// (16 k-blocks), each range's digits in a set of their own, added modulo m
// afterwards (the digits are linear in W). The count minimises the estimated
// time, waves of units times (slabs per range + one slab of overhead), over
// `workers` units at once (CTA pairs or CTAs of a GB300: 76 or 152); ties go
// to fewer ranges. Without a shortage of tiles it is one range. Depends on
// the shape only, so that the workspace size can be computed on the host.
struct KSplit {
  int nsplit, kbps;
};
inline KSplit ksplit_for(int64_t kblocks, int64_t tiles, int64_t workers) {
  const int64_t slab = 16, nslabs = (kblocks + slab - 1) / slab;
  KSplit best = {1, (int)kblocks};
  if (tiles >= workers || nslabs < 2) return best;
  int64_t best_t = ((tiles + workers - 1) / workers) * (nslabs + 1);
  for (int64_t s = 2; s <= nslabs && s <= 32; ++s) {
    const int64_t per = (nslabs + s - 1) / s;          // slabs per range
    const int64_t ns = (nslabs + per - 1) / per;       // ranges actually used
    const int64_t t = ((tiles * ns + workers - 1) / workers) * (per + 1);
    if (t < best_t) best_t = t, best.nsplit = (int)ns, best.kbps = (int)(per * slab);
  }
  return best;
}
constexpr int64_t kPairWorkers = 76;     // CTA pairs of a GB300 (152 SMs)
constexpr int64_t kCtaWorkers = 152;

// Geometry of a float-format plan's planes: k padding (entries) and bytes per
// row of k_pad entries.
inline int64_t fp_k_align(const OzFpTables& f) { return f.code_bits == 4 ? 256 : kPadK; }
inline int64_t fp_row_bytes(const OzFpTables& f, int64_t k_pad) { return f.code_bits == 4 ? k_pad / 2 : k_pad; }

inline int64_t round_up(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

// Launchers (defined in the .cu files). Each returns cudaGetLastError().
// given: the shifts are already in `shifts` (taken over a longer vector, as
// in a blocked call); the split then neither scans for the maximum nor flags.
cudaError_t launch_split_rows(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld,
                              int64_t nvec_pad, int64_t k_pad, int32_t* shifts, void* planes, int bf16,
                              int32_t* flag, cudaStream_t st, bool given = false);
cudaError_t launch_split_cols(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld,
                              int64_t nvec_pad, int64_t k_pad, int32_t* shifts, void* planes, int bf16,
                              int32_t* flag, uint64_t* colmax, cudaStream_t st, bool given = false);
cudaError_t launch_gemm_imma(const OzTables& t, int64_t m, int64_t n, int64_t k_pad, const int8_t* U,
                             int64_t u_plane, const int8_t* V, int64_t v_plane, uint8_t* Y, int64_t ldy, int raw,
                             cudaStream_t st);
// Y: residue planes [Q][m][ldy] (ldy >= n; a multiple of 16 lets the epilogue store whole 16-byte runs)
// split: the ranges of ksplit_for (nsplit 1: none), digit set j at Y + j ysplit
cudaError_t launch_gemm_tc(const OzTables& t, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                           const void* U, const void* V, uint8_t* Y, int64_t ldy, int raw, int32_t* status,
                           cudaStream_t st, KSplit split = {1, 0}, int64_t ysplit = 0);
cudaError_t launch_gemm_tc_single(const OzTables& t, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                           const void* U, const void* V, uint8_t* Y, int64_t ldy, int raw, int32_t* status,
                           cudaStream_t st, KSplit split = {1, 0}, int64_t ysplit = 0);
// Y[0] = sum of the nsplit digit sets Y[j] (at Y + j ysplit) modulo each
// modulus, over Q planes of m rows of ldy bytes (ldy a multiple of 16)
cudaError_t launch_combine_digits(const OzTables& t, int64_t m, int64_t ldy, uint8_t* Y, int nsplit, int64_t ysplit,
                                  cudaStream_t st);
cudaError_t launch_reconstruct(const OzTables& t, int64_t m, int64_t n, const uint8_t* Y, int64_t ldy,
                               const int32_t* s, const int32_t* tt, double* C, int64_t ldc, cudaStream_t st);
cudaError_t launch_reconstruct16_wide(const OzTables& t, int64_t m, int64_t n, const uint16_t* Y, int64_t ldy,
                                      const int32_t* s, const int32_t* tt, double* C, int64_t ldc, cudaStream_t st);
// grouped products (oz_grouped.cu): one launch per phase over count problems
// of one plan; probs is device memory; totals are the launch sizes. Per
// phase, a device array maps each block of the launch to its problem (an
// index into probs), written once when the group is created.
struct GroupMaps {
  const int32_t* rows;   // split of A, long rows: one block per row
  const int32_t* wrows;  // split of A, short rows: eight rows per block
  const int32_t* cm;     // column maxima of B
  const int32_t* sh;     // shifts of B
  const int32_t* sc;     // split of B
  const int32_t* rec;    // reconstruct
};
cudaError_t launch_split_rows_grouped(const OzTables& t, const OzGroupProblem* probs, const GroupMaps& maps,
                                      int64_t total_rows, int64_t total_wrows, cudaStream_t st);
cudaError_t launch_split_cols_grouped(const OzTables& t, const OzGroupProblem* probs, const GroupMaps& maps,
                                      int64_t total_cm, int64_t total_sh, int64_t total_sc, cudaStream_t st);
// pairs: CTA pairs on 256 x 256 tiles (units Q ceil(m/256) tiles_n), else one
// CTA per 128 x 256 tile (units Q tiles_m tiles_n); one_slab: every problem's
// k_pad is at most 1024 (each unit one slab)
cudaError_t launch_gemm_tc_grouped(const OzTables& t, const OzGroupProblem* probs, int count, int64_t total_units,
                                   int32_t* status, cudaStream_t st, bool pairs, bool one_slab);
bool group_maps_tc(OzGroupProblem* pr, int Q, bool pairs);   // host: the TMA maps of a grouped problem's planes
cudaError_t launch_reconstruct_grouped(const OzTables& t, const OzGroupProblem* probs, const GroupMaps& maps,
                                       int64_t total_rec, cudaStream_t st);
// the grouped reconstruct's entries per thread for a plan's products: 8 (the
// groups' kernel) when this holds, else 4 (the pairs' kernel)
bool reconstruct_grouped_eight(const OzTables& t);
// float-format path: planes of codes, 16-bit digits
cudaError_t launch_split_fp(const OzTables& t, const OzFpTables& f, int contiguous, int64_t nvec, int64_t len,
                            const double* X, int64_t ld, int64_t nvec_pad, int64_t k_pad, int32_t* shifts,
                            uint8_t* planes, int32_t* flag, uint64_t* colmax, cudaStream_t st, bool given = false);
cudaError_t launch_gemm_fp(const OzFpTables& f, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                           const uint8_t* U, const uint8_t* V, uint16_t* Y, int64_t ldy, int raw, int32_t* status,
                           cudaStream_t st);
cudaError_t launch_reconstruct16(const OzTables& t, int64_t m, int64_t n, const uint16_t* Y, int64_t ldy,
                                 const int32_t* s, const int32_t* tt, double* C, int64_t ldc, cudaStream_t st);
// shared by the split kernels: shifts of strided vectors (colmax must be zeroed)
cudaError_t launch_shifts_cols(int bits, int64_t nvec, int64_t len, const double* X, int64_t ld, int32_t* shifts,
                               int32_t* flag, uint64_t* colmax, cudaStream_t st);
// Y (cols x rows, row pitch rows) = X^T for X rows x cols with row pitch ld
cudaError_t launch_transpose(int64_t rows, int64_t cols, const double* X, int64_t ld, double* Y, cudaStream_t st);
// shifts of contiguous vectors (rows), one warp per row; flags non-finite entries
cudaError_t launch_shifts_rows(int bits, int64_t nvec, int64_t len, const double* X, int64_t ld, int32_t* shifts,
                               int32_t* flag, cudaStream_t st);

}  // namespace oz
