// oz_split.cu -- phases 1 (Scale) and 2 (Reduce) of Sec. "Structure".
//
// Scale (eq. convert): per vector (row of A, column of B) the exponent e with
// max|x| in [2^(e-1), 2^e), from the largest |x| bit pattern (for finite
// doubles the order of |x| is the order of its bits), and the shift
// s = beta - e (0 for a zero vector).
//
// Reduce: a' = trunc(x 2^s) taken straight from the IEEE fields: with the
// 53-bit significand f and exponent E, x 2^s = f 2^(E - 1075 + s), so a'
// is f shifted left or right (the right shift truncates toward zero). The
// residue modulo m (m <= 239) is formed in exact fp32 arithmetic (twice the
// integer issue rate): |a'| is cut once per entry into signed pieces, a first
// piece P0 of 22 bits and then pieces of 13 bits (P1..P3 when beta <= 61,
// P1..P4 when beta <= 64) or, for widened operands (beta up to 84, Sec. "Not
// True Emulation of DGEMM", a' in 128 bits), six of 12 bits. Per modulus
//   y = P0 + P1 c_1 + P2 c_2 + ...,   c_i = 2^(bits below piece i) mod m, |c_i| <= 119,
// an integer congruent to a' with |y| < 2^22 + 4 * 8191 * 119 < 2^23, so every
// partial sum is exact. One quotient q = rint(y * fl(1/m)) (an fma against
// the 1.5 * 2^23 rounding constant) is the integer nearest to y/m: the
// estimate is off by at most |y/m| 2^-24 < 1/(2m), and for odd m, y/m is at
// least 1/(2m) away from every half-integer. So r = y - q m is exactly the
// representative nearest zero. For the even modulus (236, always at index
// 2 of an INT8 plan) y/m can be a half-integer; the estimate then picks
// either neighbour, r is +-m/2, and +m/2 is mapped to -m/2: the result lies
// in [-floor(m/2), ceil(m/2) - 1] for every modulus. (The paper reduces a
// one-byte modulus in two 32-bit Barrett steps, Sec. "Around the GEMMs";
// this is the same reduction in the fp32 pipe: six fp32 operations per
// modulus and entry.)
//
// Planes are written K-major, Q planes of nvec_pad x k_pad entries, int8
// (two's complement, IMMA engine) or bf16 (TC engine; integers below 2^8 are
// exact in bf16).
#include <stdint.h>

#include <type_traits>

#include "oz_internal.h"
#include "oz_device.cuh"

namespace oz {
namespace {

// Signed pieces of a' as exact floats, NP of them: a 22-bit first piece,
// then 13-bit pieces (NP = 4: |a'| < 2^61; NP = 5: |a'| < 2^74) or 12-bit
// pieces (NP = 7, widened operands, |a'| < 2^84).
template <int NP>
struct Pieces {
  static constexpr int kW0 = 22;
  static constexpr int kBits = NP > 5 ? 12 : 13;
  float p[NP];
};

template <int NP>
__device__ __forceinline__ Pieces<NP> pieces_of(uint64_t bits, int32_t s) {
  Pieces<NP> P;
  constexpr int W0 = Pieces<NP>::kW0, PB = Pieces<NP>::kBits;
  constexpr uint32_t mask = (1u << PB) - 1u;
  if constexpr (NP > 5) {
    const TruncWide t = truncate_wide(bits, s);
    const float sg = t.neg ? -1.0f : 1.0f;
    const float off = t.neg ? 8388608.0f : -8388608.0f;
    P.p[0] = fmaf(__int_as_float(0x4B000000u | ((uint32_t)t.mag & ((1u << W0) - 1u))), sg, off);   // +-v, exact
#pragma unroll
    for (int i = 1; i < NP; ++i) {
      const uint32_t v = (uint32_t)(t.mag >> (W0 + PB * (i - 1))) & mask;
      P.p[i] = fmaf(__int_as_float(0x4B000000u | v), sg, off);
    }
  } else {
    const Trunc t = truncate(bits, s);
    const float sg = t.neg ? -1.0f : 1.0f;
    const float off = t.neg ? 8388608.0f : -8388608.0f;
    P.p[0] = fmaf(__int_as_float(0x4B000000u | ((uint32_t)t.mag & ((1u << W0) - 1u))), sg, off);
#pragma unroll
    for (int i = 1; i < NP; ++i) {
      const uint32_t v = (uint32_t)(t.mag >> (W0 + PB * (i - 1))) & mask;
      P.p[i] = fmaf(__int_as_float(0x4B000000u | v), sg, off);
    }
  }
  return P;
}

// The constants of one modulus, held in registers while a tile is reduced:
// c[i - 1] = 2^(bits below piece i) mod m, nearest zero.
template <int NP>
struct ModConst {
  float c[NP - 1];
  float invm, m;
};

template <int NP>
__device__ __forceinline__ ModConst<NP> mod_const(const OzTables& T, int q) {
  ModConst<NP> c;
#pragma unroll
  for (int i = 0; i < NP - 1; ++i) c.c[i] = NP > 5 ? T.c12f[i][q] : T.c13f[i][q];
  c.invm = T.invm[q];
  c.m = T.mf[q];
  return c;
}

// The tie of the even modulus (index 2): +m/2 becomes -m/2.
__device__ __forceinline__ float fix_tie(const OzTables& T, float r) {
  const float h = T.halfm[2];
  return r == h ? -h : r;
}

// Representatives of a' nearest zero modulo one modulus for EPT entries, as
// exact floats in [-m/2, m/2] (see the header; below m/2 in magnitude for an
// odd m): y = P0 + P1 c_1 + ..., q = rint(y / m) by one fma against the
// rounding constant, r = y - q m. Two entries go through each packed fp32
// operation (the f32x2 fma and add of sm_100 and later round each half as the
// scalar operation would), so the issued instructions are half those of the
// scalar chain and the results are the same bits.
template <int NP, int EPT>
__device__ __forceinline__ void residues_any(const ModConst<NP>& c, const Pieces<NP> (&P)[EPT], float (&r)[EPT]) {
  static_assert(EPT % 2 == 0, "entries in pairs");
  const float2 kC = make_float2(12582912.0f, 12582912.0f), kCn = make_float2(-12582912.0f, -12582912.0f);
  const float2 inv = make_float2(c.invm, c.invm), nm = make_float2(-c.m, -c.m);
  float2 ci[NP - 1];
#pragma unroll
  for (int i = 0; i < NP - 1; ++i) ci[i] = make_float2(c.c[i], c.c[i]);
#pragma unroll
  for (int e = 0; e < EPT; e += 2) {
    float2 y = make_float2(P[e].p[0], P[e + 1].p[0]);
#pragma unroll
    for (int i = 1; i < NP; ++i) y = __ffma2_rn(make_float2(P[e].p[i], P[e + 1].p[i]), ci[i - 1], y);
    const float2 qf = __fadd2_rn(__ffma2_rn(y, inv, kC), kCn);   // rint(y / m), exact
    const float2 rr = __ffma2_rn(qf, nm, y);
    r[e] = rr.x;
    r[e + 1] = rr.y;
  }
}

// Representatives in [-floor(m/2), ceil(m/2) - 1] of modulus q for EPT
// entries, q a compile-time index after unrolling: only q = 2 takes the tie
// fix.
template <int NP, int EPT>
__device__ __forceinline__ void residues_q(const OzTables& T, int q, const ModConst<NP>& c, const Pieces<NP> (&P)[EPT],
                                           float (&r)[EPT]) {
  residues_any<NP, EPT>(c, P, r);
  if (q == 2) {
#pragma unroll
    for (int e = 0; e < EPT; ++e) r[e] = fix_tie(T, r[e]);
  }
}

// bf16 bit pattern of the integers r (|r| < 2^8 needs at most 8 significand
// bits, so the upper half of the float is exact)
__device__ __forceinline__ uint32_t bf16_pair(float r_lo, float r_hi) {
  return __byte_perm(__float_as_uint(r_lo), __float_as_uint(r_hi), 0x7632u);
}

// two's-complement byte of r: r + 1.5 * 2^23 has r in its low byte
__device__ __forceinline__ uint32_t int8_bits(float r) { return __float_as_uint(r + 12582912.0f); }

__device__ __forceinline__ uint32_t int8_quad(float a, float b, float c, float d) {
  return __byte_perm(__byte_perm(int8_bits(a), int8_bits(b), 0x0040u), __byte_perm(int8_bits(c), int8_bits(d), 0x0040u),
                     0x5410u);
}

// The residues of EPT consecutive entries (pieces P) modulo every modulus,
// stored at planes[q plane + off]: one 16- or 8-byte store of bf16 (EPT = 8
// or 4), or 8 or 4 bytes of int8, per modulus. QT > 0: the modulus count is QT
// at compile time (no per-modulus test); QT = 0: T.Q at run time.
template <bool kBF16, int NP, int EPT, int QT>
__device__ __forceinline__ void store_residues(const OzTables& T, const Pieces<NP> (&P)[EPT], void* __restrict__ planes,
                                               int64_t plane, int64_t off) {
  static_assert(EPT == 4 || EPT == 8, "four or eight entries");
  const int Q = QT > 0 ? QT : T.Q;
#pragma unroll
  for (int q = 0; q < (QT > 0 ? QT : OZ_MAX_MODULI); ++q) {
    if (QT > 0 || q < Q) {
      const ModConst<NP> mc = mod_const<NP>(T, q);
      float r[EPT];
      residues_q<NP, EPT>(T, q, mc, P, r);
      const int64_t o = (int64_t)q * plane + off;
      if (kBF16) {
        uint16_t* dst = static_cast<uint16_t*>(planes) + o;
        if constexpr (EPT == 8)
          *reinterpret_cast<uint4*>(dst) = make_uint4(bf16_pair(r[0], r[1]), bf16_pair(r[2], r[3]),
                                                      bf16_pair(r[4], r[5]), bf16_pair(r[6], r[7]));
        else
          *reinterpret_cast<uint2*>(dst) = make_uint2(bf16_pair(r[0], r[1]), bf16_pair(r[2], r[3]));
      } else {
        int8_t* dst = static_cast<int8_t*>(planes) + o;
        if constexpr (EPT == 8)
          *reinterpret_cast<uint2*>(dst) = make_uint2(int8_quad(r[0], r[1], r[2], r[3]), int8_quad(r[4], r[5], r[6], r[7]));
        else
          *reinterpret_cast<uint32_t*>(dst) = int8_quad(r[0], r[1], r[2], r[3]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Contiguous vectors (rows of A, or of B^T): one CTA of 256 threads per
// vector. Pass 1 finds the max bits; pass 2 re-reads the row (from L2) and
// writes 8 consecutive entries per thread per plane.
// ---------------------------------------------------------------------------
// The largest |x| bit pattern over row[h], h = t, t + step, ... (t < step),
// and whether any of those entries is not finite: 16-byte loads (two
// entries) when the row is 16-byte aligned, four of them in flight per
// iteration, so that a short row's maximum is not a chain of load latencies.
__device__ __forceinline__ void row_absmax(const uint64_t* __restrict__ row, int64_t len, int t, int step,
                                           uint64_t& mx, uint32_t& bad) {
  auto fold = [&](uint64_t b) {
    b &= kAbsMask;
    bad |= (uint32_t)((b >> 52) == 0x7ff);
    mx = b > mx ? b : mx;
  };
  if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {
    const ulonglong2* r2 = reinterpret_cast<const ulonglong2*>(row);
    const int64_t np = len >> 1;
    int64_t p = t;
    for (; p + 3 * (int64_t)step < np; p += 4 * (int64_t)step) {
      ulonglong2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(r2 + p + u * step);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        fold(v[u].x);
        fold(v[u].y);
      }
    }
    for (; p < np; p += step) {
      const ulonglong2 v = __ldg(r2 + p);
      fold(v.x);
      fold(v.y);
    }
    if ((len & 1) && t == 0) fold(__ldg(row + len - 1));
  } else {
    for (int64_t h = t; h < len; h += step) fold(__ldg(row + h));
  }
}

template <bool kBF16, int NP, int QT>
__device__ __forceinline__ void split_row(const OzTables& T, int64_t v, int64_t nvec, int64_t len,
                                          const double* __restrict__ X, int64_t ld, int64_t nvec_pad, int64_t k_pad,
                                          int32_t* __restrict__ shifts, void* __restrict__ planes,
                                          int32_t* __restrict__ flag, bool given) {
  __shared__ uint64_t red[8];
  __shared__ int32_t s_sh;
  const int tid = threadIdx.x;
  const bool live = v < nvec;
  const uint64_t* row = reinterpret_cast<const uint64_t*>(X) + (live ? v * ld : 0);

  int32_t s;
  if (given) {                      // block-uniform: the shift of the whole row is known
    s = live ? shifts[v] : 0;
  } else {
    uint64_t mx = 0;
    uint32_t bad = 0;
    if (live) row_absmax(row, len, tid, 256, mx, bad);
    mx = warp_max_u64(mx);
    bad = __any_sync(0xffffffffu, bad);
    if ((tid & 31) == 0) red[tid >> 5] = mx | (bad ? (1ull << 63) : 0);
    __syncthreads();
    if (tid == 0) {
      uint64_t m = 0, anybad = 0;
      for (int w = 0; w < 8; ++w) {
        anybad |= red[w] >> 63;
        uint64_t x = red[w] & kAbsMask;
        m = x > m ? x : m;
      }
      if (anybad && flag) atomicOr(flag, 1);
      int32_t s0 = live ? shift_from_maxbits(anybad ? 0 : m, T.bits) : 0;
      s_sh = s0;
      if (live) shifts[v] = s0;
    }
    __syncthreads();
    s = s_sh;
  }

  const int64_t plane = nvec_pad * k_pad;
  const bool vec = live && ((reinterpret_cast<uintptr_t>(row) & 15) == 0);
  // eight entries per thread per pass
  for (int64_t h0 = (int64_t)tid * 8; h0 < k_pad; h0 += 256 * 8) {
    uint64_t b[8];
    if (vec && h0 + 8 <= len) {
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2*>(row + h0 + e));
        b[e] = w.x;
        b[e + 1] = w.y;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) b[e] = (live && h0 + e < len) ? __ldg(row + h0 + e) : 0ull;
    }
    Pieces<NP> P[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (((b[e] >> 52) & 0x7ff) == 0x7ff) b[e] = 0;  // non-finite: flagged above
      P[e] = pieces_of<NP>(b[e], s);
    }
    store_residues<kBF16, NP, 8, QT>(T, P, planes, plane, v * k_pad + h0);
  }
}

// The same for a short row (k_pad <= 1024 in one product's split, <= 4096
// in the grouped one): one warp per row, eight rows per block; the row's
// maximum is a warp reduction.
template <bool kBF16, int NP, int QT>
__device__ __forceinline__ void split_row_warp(const OzTables& T, int64_t v, int64_t nvec, int64_t len,
                                               const double* __restrict__ X, int64_t ld, int64_t nvec_pad,
                                               int64_t k_pad, int32_t* __restrict__ shifts,
                                               void* __restrict__ planes, int32_t* __restrict__ flag, bool given) {
  const int lane = threadIdx.x & 31;
  const bool live = v < nvec;
  const uint64_t* row = reinterpret_cast<const uint64_t*>(X) + (live ? v * ld : 0);
  int32_t s;
  if (given) {
    s = live ? shifts[v] : 0;
  } else {
    uint64_t mx = 0;
    uint32_t bad = 0;
    if (live) row_absmax(row, len, lane, 32, mx, bad);
    mx = warp_max_u64(mx);
    bad = __any_sync(0xffffffffu, bad);
    s = live ? shift_from_maxbits(bad ? 0 : mx, T.bits) : 0;
    if (lane == 0) {
      if (bad && flag) atomicOr(flag, 1);
      if (live) shifts[v] = s;
    }
  }
  const int64_t plane = nvec_pad * k_pad;
  const bool vec = live && ((reinterpret_cast<uintptr_t>(row) & 15) == 0);
  for (int64_t h0 = (int64_t)lane * 8; h0 < k_pad; h0 += 32 * 8) {
    uint64_t b[8];
    if (vec && h0 + 8 <= len) {
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2*>(row + h0 + e));
        b[e] = w.x;
        b[e + 1] = w.y;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) b[e] = (live && h0 + e < len) ? __ldg(row + h0 + e) : 0ull;
    }
    Pieces<NP> P[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (((b[e] >> 52) & 0x7ff) == 0x7ff) b[e] = 0;
      P[e] = pieces_of<NP>(b[e], s);
    }
    store_residues<kBF16, NP, 8, QT>(T, P, planes, plane, v * k_pad + h0);
  }
}

template <bool kBF16, int NP, int QT>
__global__ void __launch_bounds__(256) split_rows_warp_kernel(const __grid_constant__ OzTables T, int64_t nvec,
                                                              int64_t len, const double* __restrict__ X, int64_t ld,
                                                              int64_t nvec_pad, int64_t k_pad,
                                                              int32_t* __restrict__ shifts,
                                                              void* __restrict__ planes, int32_t* __restrict__ flag,
                                                              bool given) {
  const int64_t v = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  split_row_warp<kBF16, NP, QT>(T, v, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, given);
}

// Grouped, short rows: block b holds rows 8 (b - rows_begin) .. + 7 of its
// problem; map[b] is the problem.
// (three blocks per SM where the registers allow it without spilling)
template <int NP, int QT>
__global__ void __launch_bounds__(256, (QT > 0 && NP == 4) ? 3 : 2) split_rows_warp_grouped_kernel(const __grid_constant__ OzTables T,
                                                                         const OzGroupProblem* __restrict__ probs,
                                                                         const int32_t* __restrict__ map) {
  const int64_t b = blockIdx.x;
  const OzGroupProblem& P = probs[__ldg(map + b)];
  const int64_t v = (b - P.rows_begin) * 8 + (threadIdx.x >> 5);
  split_row_warp<true, NP, QT>(T, v, P.m, P.k, P.A, P.lda, P.m_pad, P.k_pad, P.s, P.U, P.flag, false);
}

template <bool kBF16, int NP, int QT>
__global__ void __launch_bounds__(256, 3) split_rows_kernel(const __grid_constant__ OzTables T, int64_t nvec, int64_t len,
                                                         const double* __restrict__ X, int64_t ld,
                                                         int64_t nvec_pad, int64_t k_pad,
                                                         int32_t* __restrict__ shifts, void* __restrict__ planes,
                                                         int32_t* __restrict__ flag, bool given) {
  split_row<kBF16, NP, QT>(T, blockIdx.x, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, given);
}

// Grouped: block b is row b - rows_begin of its problem's A; map[b] is the problem.
template <int NP, int QT>
__global__ void __launch_bounds__(256, (QT > 0 && NP == 4) ? 3 : 2) split_rows_grouped_kernel(const __grid_constant__ OzTables T,
                                                                    const OzGroupProblem* __restrict__ probs,
                                                                    const int32_t* __restrict__ map) {
  const int64_t b = blockIdx.x;
  const OzGroupProblem& P = probs[__ldg(map + b)];
  split_row<true, NP, QT>(T, b - P.rows_begin, P.m, P.k, P.A, P.lda, P.m_pad, P.k_pad, P.s, P.U, P.flag, false);
}

// ---------------------------------------------------------------------------
// Strided vectors (columns of B, or of A^T).
// Pass 1: column maxima by atomicMax into colmax (zeroed by the launcher).
// Block (32 x 8): 32 consecutive columns, 8 warps over rows; each CTA covers
// 256 rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void colmax_block(int64_t bx, int64_t by, int64_t nvec, int64_t len,
                                             const double* __restrict__ X, int64_t ld,
                                             uint64_t* __restrict__ colmax, int32_t* __restrict__ flag) {
  __shared__ uint64_t red[8][32];
  const int64_t j = bx * 32 + threadIdx.x;
  const int64_t h0 = by * 256 + threadIdx.y;
  uint64_t mx = 0;
  uint32_t bad = 0;
  if (j < nvec) {
    const uint64_t* col = reinterpret_cast<const uint64_t*>(X) + j;
    // 32 rows per thread, loads issued together (predicated, no early exit)
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int64_t h = h0 + 8 * i;
      const uint64_t b = h < len ? __ldg(col + h * ld) & kAbsMask : 0ull;
      bad |= (uint32_t)((b >> 52) == 0x7ff);
      mx = b > mx ? b : mx;
    }
  }
  if (bad && flag) atomicOr(flag, 1);
  red[threadIdx.y][threadIdx.x] = bad ? 0 : mx;
  __syncthreads();
  if (threadIdx.y == 0 && j < nvec) {
    uint64_t m = 0;
    for (int w = 0; w < 8; ++w) m = red[w][threadIdx.x] > m ? red[w][threadIdx.x] : m;
    if (m) atomicMax(reinterpret_cast<unsigned long long*>(colmax + j), (unsigned long long)m);
  }
}

__global__ void __launch_bounds__(256) colmax_kernel(int64_t nvec, int64_t len, const double* __restrict__ X,
                                                     int64_t ld, uint64_t* __restrict__ colmax,
                                                     int32_t* __restrict__ flag) {
  colmax_block(blockIdx.x, blockIdx.y, nvec, len, X, ld, colmax, flag);
}

// Grouped: block b is block b - cm_begin of its problem's (ceil(n/32) x
// ceil(k/256)) grid, x fastest; map[b] is the problem.
__global__ void __launch_bounds__(256) colmax_grouped_kernel(const OzGroupProblem* __restrict__ probs,
                                                             const int32_t* __restrict__ map) {
  const int64_t b = blockIdx.x;
  const OzGroupProblem& P = probs[__ldg(map + b)];
  const int64_t l = b - P.cm_begin, nbx = (P.n + 31) / 32;
  colmax_block(l % nbx, l / nbx, P.n, P.k, P.B, P.ldb, P.colmax, P.flag);
}

__global__ void shifts_from_colmax_kernel(int64_t nvec, const uint64_t* __restrict__ colmax, int beta,
                                          int32_t* __restrict__ shifts) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nvec) shifts[j] = shift_from_maxbits(colmax[j], beta);
}

__global__ void shifts_grouped_kernel(const OzGroupProblem* __restrict__ probs, const int32_t* __restrict__ map,
                                      int beta) {
  const int64_t b = blockIdx.x;
  const OzGroupProblem& P = probs[__ldg(map + b)];
  const int64_t j = (b - P.sh_begin) * blockDim.x + threadIdx.x;
  if (j < P.n) P.t[j] = shift_from_maxbits(P.colmax[j], beta);
}

// Shifts of contiguous vectors without a split (a blocked call takes them over
// the whole row before splitting it slab by slab): one warp per row.
__global__ void __launch_bounds__(256) shifts_rows_kernel(int64_t nvec, int64_t len, const double* __restrict__ X,
                                                          int64_t ld, int beta, int32_t* __restrict__ shifts,
                                                          int32_t* __restrict__ flag) {
  const int64_t v = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= nvec) return;                 // the whole warp shares v
  const uint64_t* row = reinterpret_cast<const uint64_t*>(X) + v * ld;
  uint64_t mx = 0;
  uint32_t bad = 0;
  row_absmax(row, len, lane, 32, mx, bad);
  mx = warp_max_u64(mx);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    if (bad && flag) atomicOr(flag, 1);
    shifts[v] = shift_from_maxbits(bad ? 0 : mx, beta);
  }
}

// Pass 2: 64 (h) x 64 (vector) tiles; residues go through shared memory so
// that the planes, which are K-major per vector, are written along h.
// Thread t handles vector j = t % 64 and 16 consecutive h.
template <bool kBF16, int NP>
__device__ __forceinline__ void split_cols_block(const OzTables& T, int64_t bx, int64_t by, int64_t nvec,
                                                 int64_t len, const double* __restrict__ X, int64_t ld,
                                                 int64_t nvec_pad, int64_t k_pad,
                                                 const int32_t* __restrict__ shifts, void* __restrict__ planes) {
  constexpr int kPitchWords = kBF16 ? 33 : 17;   // 64 entries + 4 bytes of padding per row
  __shared__ uint32_t tile[2][64 * kPitchWords];
  const int tid = threadIdx.x;
  const int jl = tid & 63;
  const int hg = tid >> 6;                         // 0..3: h = hg*16 .. hg*16+15
  const int64_t j0 = bx * 64;
  const int64_t hbase = by * 64;
  const int64_t j = j0 + jl;
  const bool live = j < nvec;
  const int32_t s = live ? shifts[j] : 0;

  Pieces<NP> P[16];
  const uint64_t* Xb = reinterpret_cast<const uint64_t*>(X);
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    int64_t h = hbase + hg * 16 + e;
    uint64_t b = (live && h < len) ? __ldg(Xb + h * ld + j) : 0ull;
    if (((b >> 52) & 0x7ff) == 0x7ff) b = 0;
    P[e] = pieces_of<NP>(b, s);
  }
  const int Q = T.Q;
  const int64_t plane = nvec_pad * k_pad;
#pragma unroll 1
  for (int q = 0; q < Q; ++q) {
    uint32_t* tb = tile[q & 1];
    const ModConst<NP> mc = mod_const<NP>(T, q);
    float r[16];
    residues_any<NP, 16>(mc, P, r);
    if (q == 2) {                                    // block-uniform branch: the even modulus
#pragma unroll
      for (int e = 0; e < 16; ++e) r[e] = fix_tie(T, r[e]);
    }
    if (kBF16) {
#pragma unroll
      for (int w = 0; w < 8; ++w) tb[jl * kPitchWords + hg * 8 + w] = bf16_pair(r[2 * w], r[2 * w + 1]);
    } else {
#pragma unroll
      for (int w = 0; w < 4; ++w)
        tb[jl * kPitchWords + hg * 4 + w] = int8_quad(r[4 * w], r[4 * w + 1], r[4 * w + 2], r[4 * w + 3]);
    }
    __syncthreads();
    // write 64 rows of 64 entries: int8 -> 4 words of 16 B per row, bf16 -> 8
    constexpr int kChunks = kBF16 ? 8 : 4;          // 16-byte chunks per row
    for (int c = tid; c < 64 * kChunks; c += 256) {
      int row = c / kChunks, ch = c % kChunks;
      if (j0 + row >= nvec_pad) continue;
      uint4 o;
      o.x = tb[row * kPitchWords + ch * 4 + 0];
      o.y = tb[row * kPitchWords + ch * 4 + 1];
      o.z = tb[row * kPitchWords + ch * 4 + 2];
      o.w = tb[row * kPitchWords + ch * 4 + 3];
      const int64_t off = (int64_t)q * plane + (j0 + row) * k_pad + hbase;
      char* dst = static_cast<char*>(planes) + (off * (kBF16 ? 2 : 1)) + ch * 16;
      *reinterpret_cast<uint4*>(dst) = o;
    }
    // tile[q & 1] is rewritten two moduli later, after the next barrier
  }
}

template <bool kBF16, int NP>
__global__ void __launch_bounds__(256) split_cols_kernel(const __grid_constant__ OzTables T, int64_t nvec, int64_t len,
                                                         const double* __restrict__ X, int64_t ld,
                                                         int64_t nvec_pad, int64_t k_pad,
                                                         const int32_t* __restrict__ shifts,
                                                         void* __restrict__ planes) {
  split_cols_block<kBF16, NP>(T, blockIdx.x, blockIdx.y, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes);
}

// bf16 planes (TC engine): tiles of 32 vectors x 64 h. Lane l holds vector
// j0 + l, warp w the eight h = hbase + 8w .. + 7 (each load instruction reads
// 32 consecutive doubles of one row of X). The residues of every modulus are
// staged in shared memory, [q][32 vectors][64 h + 8 pad] bf16 (rows of 144
// bytes: the 16-byte stores and loads of a quarter-warp fall in distinct
// banks), and after one barrier each thread writes one 16-byte run per
// modulus, so the planes (K-major per vector) receive whole 128-byte rows.
constexpr int kColTileJ = 32, kColTileH = 64;
constexpr int kColPitchWords = 36;
constexpr int kColPlaneWords = kColTileJ * kColPitchWords;     // 1152 words = 4608 bytes per modulus

template <int NP, int QT>
__device__ __forceinline__ void split_cols_tile(const OzTables& T, int64_t j0, int64_t hbase, int64_t nvec,
                                                int64_t len, const double* __restrict__ X, int64_t ld,
                                                int64_t nvec_pad, int64_t k_pad, const int32_t* __restrict__ shifts,
                                                uint16_t* __restrict__ planes, uint32_t* tile) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t j = j0 + lane;
  const bool live = j < nvec;
  const int32_t s = live ? __ldg(shifts + j) : 0;
  const uint64_t* Xb = reinterpret_cast<const uint64_t*>(X);
  const int64_t h0 = hbase + 8 * w;
  uint64_t b[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) b[e] = (live && h0 + e < len) ? __ldg(Xb + (h0 + e) * ld + j) : 0ull;
  Pieces<NP> P[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    if (((b[e] >> 52) & 0x7ff) == 0x7ff) b[e] = 0;   // non-finite: flagged by the column maxima
    P[e] = pieces_of<NP>(b[e], s);
  }
  const int Q = QT > 0 ? QT : T.Q;
  uint4* const mine = reinterpret_cast<uint4*>(tile + lane * kColPitchWords + 4 * w);
#pragma unroll
  for (int q = 0; q < (QT > 0 ? QT : OZ_MAX_MODULI); ++q) {
    if (QT > 0 || q < Q) {
      const ModConst<NP> mc = mod_const<NP>(T, q);
      float r[8];
      residues_q<NP, 8>(T, q, mc, P, r);
      mine[q * (kColPlaneWords / 4)] =
          make_uint4(bf16_pair(r[0], r[1]), bf16_pair(r[2], r[3]), bf16_pair(r[4], r[5]), bf16_pair(r[6], r[7]));
    }
  }
  __syncthreads();
  // thread t: vector row t / 8 of the tile, 16-byte chunk t % 8 of its 64 h
  const int row = threadIdx.x >> 3, ch = threadIdx.x & 7;
  if (j0 + row < nvec_pad) {
    const int64_t plane = nvec_pad * k_pad;
    uint16_t* dst = planes + (j0 + row) * k_pad + hbase + 8 * ch;
    const uint4* src = reinterpret_cast<const uint4*>(tile + row * kColPitchWords + 4 * ch);
#pragma unroll 4
    for (int q = 0; q < Q; ++q)
      *reinterpret_cast<uint4*>(dst + q * plane) = src[q * (kColPlaneWords / 4)];
  }
}

template <int NP, int QT>
__global__ void __launch_bounds__(256, 3) split_cols_bf16_kernel(const __grid_constant__ OzTables T, int64_t nvec,
                                                                int64_t len, const double* __restrict__ X, int64_t ld,
                                                                int64_t nvec_pad, int64_t k_pad,
                                                                const int32_t* __restrict__ shifts,
                                                                uint16_t* __restrict__ planes) {
  extern __shared__ uint4 col_tile[];
  split_cols_tile<NP, QT>(T, (int64_t)blockIdx.x * kColTileJ, (int64_t)blockIdx.y * kColTileH, nvec, len, X, ld,
                          nvec_pad, k_pad, shifts, planes, reinterpret_cast<uint32_t*>(col_tile));
}

// Grouped: block b is tile l = b - sc_begin of its problem's
// (n_pad / 32) x (k_pad / 64) grid, vectors fastest; map[b] is its problem.
template <int NP, int QT>
__global__ void __launch_bounds__(256, 3) split_cols_grouped_kernel(const __grid_constant__ OzTables T,
                                                                   const OzGroupProblem* __restrict__ probs,
                                                                   const int32_t* __restrict__ map) {
  extern __shared__ uint4 col_tile[];
  const int64_t b = blockIdx.x;
  const OzGroupProblem& P = probs[__ldg(map + b)];
  const int64_t l = b - P.sc_begin, nbx = P.n_pad / kColTileJ;
  split_cols_tile<NP, QT>(T, (l % nbx) * kColTileJ, (l / nbx) * kColTileH, P.n, P.k, P.B, P.ldb, P.n_pad, P.k_pad,
                          P.t, static_cast<uint16_t*>(P.V), reinterpret_cast<uint32_t*>(col_tile));
}

// Transpose of a rows x cols block of doubles (row pitch ld) into cols x rows
// (row pitch rows), through 32 x 33 shared tiles: reads and writes both
// coalesced. Lets the column vectors of B be split as rows.
__global__ void __launch_bounds__(256) transpose_kernel(int64_t rows, int64_t cols, const double* __restrict__ X,
                                                        int64_t ld, double* __restrict__ Y) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;    // 32 x 8 threads
  const int64_t ctiles = (cols + 31) / 32;                   // block b: tile (b / ctiles, b % ctiles)
  const int64_t c0 = ((int64_t)blockIdx.x % ctiles) * 32, r0 = ((int64_t)blockIdx.x / ctiles) * 32;
#pragma unroll
  for (int i = 0; i < 32; i += 8) {
    const int64_t r = r0 + ty + i, c = c0 + tx;
    if (r < rows && c < cols) tile[ty + i][tx] = __ldg(X + r * ld + c);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 32; i += 8) {
    const int64_t c = c0 + ty + i, r = r0 + tx;
    if (r < rows && c < cols) Y[c * rows + r] = tile[tx][ty + i];
  }
}

// Rows v in [nvec, nvec_pad) of the strided layout are covered by the grid
// (grid.x spans nvec_pad), so no separate padding pass is needed.

}  // namespace

namespace {

// pieces per entry for a bit budget: 22 bits and three or four of 13 bits,
// or 22 bits and six of 12 (widened operands)
int pieces_for(int bits) { return bits <= 61 ? 4 : bits <= 64 ? 5 : 7; }

template <bool kBF16, int NP, int QT>
void split_rows_qt(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld, int64_t nvec_pad,
                   int64_t k_pad, int32_t* shifts, void* planes, int32_t* flag, cudaStream_t st, bool given) {
  if (k_pad <= 1024)                             // short rows: one warp per row
    split_rows_warp_kernel<kBF16, NP, QT><<<(unsigned)(nvec_pad / 8), 256, 0, st>>>(t, nvec, len, X, ld, nvec_pad,
                                                                                     k_pad, shifts, planes, flag,
                                                                                     given);
  else
    split_rows_kernel<kBF16, NP, QT><<<(unsigned)nvec_pad, 256, 0, st>>>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts,
                                                                          planes, flag, given);
}

// Q = 16 (the paper's INT8 configuration) with the modulus count fixed at
// compile time; other counts read it from the table
template <bool kBF16, int NP>
void split_rows_np(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld, int64_t nvec_pad,
                   int64_t k_pad, int32_t* shifts, void* planes, int32_t* flag, cudaStream_t st, bool given) {
  if (t.Q == 16)
    split_rows_qt<kBF16, NP, 16>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, st, given);
  else
    split_rows_qt<kBF16, NP, 0>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, st, given);
}

template <int NP, int QT>
cudaError_t split_cols_bf16_qt(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld,
                               int64_t nvec_pad, int64_t k_pad, const int32_t* shifts, void* planes, cudaStream_t st) {
  const int smem = (QT > 0 ? QT : t.Q) * kColPlaneWords * 4;
  cudaError_t e = cudaFuncSetAttribute(split_cols_bf16_kernel<NP, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (QT > 0 ? QT : OZ_MAX_MODULI) * kColPlaneWords * 4);
  if (e != cudaSuccess) return e;
  dim3 g((unsigned)(nvec_pad / kColTileJ), (unsigned)(k_pad / kColTileH));
  split_cols_bf16_kernel<NP, QT><<<g, 256, smem, st>>>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts,
                                                       static_cast<uint16_t*>(planes));
  return cudaGetLastError();
}

template <bool kBF16, int NP>
cudaError_t split_cols_np(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld, int64_t nvec_pad,
                          int64_t k_pad, const int32_t* shifts, void* planes, cudaStream_t st) {
  if constexpr (kBF16 && NP <= 5) {
    if (t.Q == 16) return split_cols_bf16_qt<NP, 16>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, st);
    return split_cols_bf16_qt<NP, 0>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, st);
  } else {
    dim3 g((unsigned)(nvec_pad / 64), (unsigned)(k_pad / 64));
    split_cols_kernel<kBF16, NP><<<g, 256, 0, st>>>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes);
    return cudaGetLastError();
  }
}

}  // namespace

cudaError_t launch_split_rows(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld,
                              int64_t nvec_pad, int64_t k_pad, int32_t* shifts, void* planes, int bf16,
                              int32_t* flag, cudaStream_t st, bool given) {
  if (nvec_pad == 0) return cudaSuccess;
  switch (pieces_for(t.bits) * 2 + (bf16 ? 1 : 0)) {
    case 9: split_rows_np<true, 4>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, st, given); break;
    case 8: split_rows_np<false, 4>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, st, given); break;
    case 11: split_rows_np<true, 5>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, st, given); break;
    case 10: split_rows_np<false, 5>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, st, given); break;
    case 15: split_rows_np<true, 7>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, st, given); break;
    default: split_rows_np<false, 7>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, st, given); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_transpose(int64_t rows, int64_t cols, const double* X, int64_t ld, double* Y, cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  const int64_t tiles = ((cols + 31) / 32) * ((rows + 31) / 32);
  if (tiles > INT32_MAX) return cudaErrorInvalidValue;
  transpose_kernel<<<(unsigned)tiles, 256, 0, st>>>(rows, cols, X, ld, Y);
  return cudaGetLastError();
}

cudaError_t launch_shifts_cols(int bits, int64_t nvec, int64_t len, const double* X, int64_t ld, int32_t* shifts,
                               int32_t* flag, uint64_t* colmax, cudaStream_t st) {
  if (nvec == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(colmax, 0, sizeof(uint64_t) * (size_t)nvec, st);
  if (e != cudaSuccess) return e;
  if (len > 0) {
    dim3 g1((unsigned)((nvec + 31) / 32), (unsigned)((len + 255) / 256));
    colmax_kernel<<<g1, dim3(32, 8), 0, st>>>(nvec, len, X, ld, colmax, flag);
  }
  shifts_from_colmax_kernel<<<(unsigned)((nvec + 255) / 256), 256, 0, st>>>(nvec, colmax, bits, shifts);
  return cudaGetLastError();
}

cudaError_t launch_shifts_rows(int bits, int64_t nvec, int64_t len, const double* X, int64_t ld, int32_t* shifts,
                               int32_t* flag, cudaStream_t st) {
  if (nvec == 0) return cudaSuccess;
  shifts_rows_kernel<<<(unsigned)((nvec + 7) / 8), 256, 0, st>>>(nvec, len, X, ld, bits, shifts, flag);
  return cudaGetLastError();
}

cudaError_t launch_split_cols(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld,
                              int64_t nvec_pad, int64_t k_pad, int32_t* shifts, void* planes, int bf16,
                              int32_t* flag, uint64_t* colmax, cudaStream_t st, bool given) {
  if (nvec_pad == 0) return cudaSuccess;
  if (!given) {
    cudaError_t e0 = launch_shifts_cols(t.bits, nvec, len, X, ld, shifts, flag, colmax, st);
    if (e0 != cudaSuccess) return e0;
  }
  switch (pieces_for(t.bits) * 2 + (bf16 ? 1 : 0)) {
    case 9: return split_cols_np<true, 4>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, st);
    case 8: return split_cols_np<false, 4>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, st);
    case 11: return split_cols_np<true, 5>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, st);
    case 10: return split_cols_np<false, 5>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, st);
    case 15: return split_cols_np<true, 7>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, st);
    default: return split_cols_np<false, 7>(t, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, st);
  }
}

// Long rows (one block per row, total_rows blocks, problems in map_rows) and
// short rows (eight per block, total_wrows blocks, map_wrows); each range has
// its own rows_begin numbering. The map entries index probs.
cudaError_t launch_split_rows_grouped(const OzTables& t, const OzGroupProblem* probs, const GroupMaps& maps,
                                      int64_t total_rows, int64_t total_wrows, cudaStream_t st) {
  if (total_rows > INT32_MAX || total_wrows > INT32_MAX || t.bits > 64) return cudaErrorInvalidValue;
  auto launch = [&](auto np, auto qt) {
    constexpr int NP = decltype(np)::value, QT = decltype(qt)::value;
    if (total_rows > 0)
      split_rows_grouped_kernel<NP, QT><<<(unsigned)total_rows, 256, 0, st>>>(t, probs, maps.rows);
    if (total_wrows > 0)
      split_rows_warp_grouped_kernel<NP, QT><<<(unsigned)total_wrows, 256, 0, st>>>(t, probs, maps.wrows);
  };
  using I4 = std::integral_constant<int, 4>;
  using I5 = std::integral_constant<int, 5>;
  if (t.bits <= 61) {   // 22 bits and three 13-bit pieces
    if (t.Q == 16) launch(I4{}, std::integral_constant<int, 16>{});
    else if (t.Q == 15) launch(I4{}, std::integral_constant<int, 15>{});
    else launch(I4{}, std::integral_constant<int, 0>{});
  } else {
    launch(I5{}, std::integral_constant<int, 0>{});
  }
  return cudaGetLastError();
}

// column maxima, shifts and split of the B operands (colmax zeroed by the caller)
cudaError_t launch_split_cols_grouped(const OzTables& t, const OzGroupProblem* probs, const GroupMaps& maps,
                                      int64_t total_cm, int64_t total_sh, int64_t total_sc, cudaStream_t st) {
  if (total_cm > INT32_MAX || total_sh > INT32_MAX || total_sc > INT32_MAX || t.bits > 64) return cudaErrorInvalidValue;
  if (total_cm > 0) colmax_grouped_kernel<<<(unsigned)total_cm, dim3(32, 8), 0, st>>>(probs, maps.cm);
  if (total_sh > 0) shifts_grouped_kernel<<<(unsigned)total_sh, 256, 0, st>>>(probs, maps.sh, t.bits);
  if (total_sc == 0) return cudaGetLastError();
  auto launch = [&](auto np, auto qt) {
    constexpr int NP = decltype(np)::value, QT = decltype(qt)::value;
    const int smem = (QT > 0 ? QT : t.Q) * kColPlaneWords * 4;
    cudaError_t e = cudaFuncSetAttribute(split_cols_grouped_kernel<NP, QT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (QT > 0 ? QT : OZ_MAX_MODULI) * kColPlaneWords * 4);
    if (e != cudaSuccess) return e;
    split_cols_grouped_kernel<NP, QT><<<(unsigned)total_sc, 256, smem, st>>>(t, probs, maps.sc);
    return cudaGetLastError();
  };
  using I4 = std::integral_constant<int, 4>;
  using I5 = std::integral_constant<int, 5>;
  if (t.bits <= 61) {
    if (t.Q == 16) return launch(I4{}, std::integral_constant<int, 16>{});
    if (t.Q == 15) return launch(I4{}, std::integral_constant<int, 15>{});
    return launch(I4{}, std::integral_constant<int, 0>{});
  }
  return launch(I5{}, std::integral_constant<int, 0>{});
}

}  // namespace oz
