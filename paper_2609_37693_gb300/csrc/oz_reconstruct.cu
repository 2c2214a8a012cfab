// oz_reconstruct.cu -- phase 5 of Sec. "Structure" (Reconstruct, Sec. "Around
// the GEMMs"): the CRT sum in digits whose sums stay exact, the balanced
// representative from one quotient estimate with an exact fallback, one
// rounding, and the unscaling.
//
// Input per entry: the CRT digits y_q = (W_q mod m_q) (P/m_q)^-1 mod m_q in
// [0, m_q), written by the GEMM epilogue. Then
//   S = sum_q y_q (P/m_q) == X (mod P),  0 <= S < Q P.
// The moduli are taken in pairs, z = y_a m_b + y_b m_a < 2^17, so that
// S = sum_pairs z P/(m_a m_b): half as many wide products, formed in 32-bit
// limbs with 64-bit accumulators (each z limb product is below 2^49; ten of
// them stay below 2^53). The quotient estimate is round(sum z / (m_a m_b)) in
// fp32 (error far below 1/2); X = S - qP is formed
// modulo 2^(32 L) in two's complement and corrected once by +-P into
// [-P/2, P/2). The window (eq. ov-crtgen) makes that X the exact integer
// product (A'B')_ij.
//
// The binary64 result fl(X 2^-(s_i + t_j)) is assembled from integer fields:
// the leading 53 bits (fewer below 2^-1022), round to nearest even from the
// round bit and the sticky bits, overflow to +-inf. No floating-point
// operation touches the value, so the rounding happens exactly once.
#include <stdint.h>

#include "oz_internal.h"

namespace oz {
namespace {

template <int L>
struct Limbs {
  uint32_t w[L];
};

template <int L>
__device__ __forceinline__ int bitlen(const Limbs<L>& x) {
  int r = 0;
#pragma unroll
  for (int i = 0; i < L; ++i)
    if (x.w[i]) r = 32 * i + 32 - __clz(x.w[i]);
  return r;
}

// bits [sh, sh + 64) of x (sh >= 0), with zeros above the top limb
template <int L>
__device__ __forceinline__ uint64_t bits64(const Limbs<L>& x, int sh) {
  const int wi = sh >> 5, b = sh & 31;
  uint32_t lo = 0, mid = 0, hi = 0;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    if (i == wi) lo = x.w[i];
    if (i == wi + 1) mid = x.w[i];
    if (i == wi + 2) hi = x.w[i];
  }
  uint64_t v = ((uint64_t)mid << 32) | lo;
  if (b) v = (v >> b) | ((uint64_t)hi << (64 - b));
  return v;
}

// any bit of x below position p set (p >= 0)
template <int L>
__device__ __forceinline__ bool any_below(const Limbs<L>& x, int p) {
  bool r = false;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    int lo = 32 * i;
    if (lo + 32 <= p) r |= x.w[i] != 0;
    else if (lo < p) r |= (x.w[i] & ((1u << (p - lo)) - 1u)) != 0;
  }
  return r;
}

template <int L>
__device__ __forceinline__ bool bit_at(const Limbs<L>& x, int p) {
  bool r = false;
#pragma unroll
  for (int i = 0; i < L; ++i)
    if (p >= 32 * i && p < 32 * i + 32) r = (x.w[i] >> (p - 32 * i)) & 1u;
  return r;
}

// x -= c * P (c >= 0 small), modulo 2^(32L)
template <int L>
__device__ __forceinline__ void sub_mul_P(Limbs<L>& x, uint32_t c, const uint32_t* P) {
  uint64_t borrow = 0;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    uint64_t sub = (uint64_t)c * P[i] + borrow;           // < 2^32 * 2^5 + 2^37
    uint64_t cur = x.w[i];
    uint64_t subl = sub & 0xffffffffull;
    x.w[i] = (uint32_t)(cur - subl);
    borrow = (sub >> 32) + (cur < subl ? 1 : 0);
  }
}

template <int L>
__device__ __forceinline__ void add_P(Limbs<L>& x, const uint32_t* P) {
  uint64_t carry = 0;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    uint64_t t = (uint64_t)x.w[i] + P[i] + carry;
    x.w[i] = (uint32_t)t;
    carry = t >> 32;
  }
}

// sign of 2x - P (x two's complement): true if 2x >= P
template <int L>
__device__ __forceinline__ bool twice_ge_P(const Limbs<L>& x, const uint32_t* P) {
  if (x.w[L - 1] >> 31) return false;     // x < 0
  // compare 2x with P limb by limb from the top
  Limbs<L> d;
  uint32_t carry = 0;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    d.w[i] = (x.w[i] << 1) | carry;
    carry = x.w[i] >> 31;
  }
  int res = 0;                             // 0 equal, 1 greater, -1 less
#pragma unroll
  for (int i = L - 1; i >= 0; --i)
    if (res == 0 && d.w[i] != P[i]) res = d.w[i] > P[i] ? 1 : -1;
  return res >= 0;
}

// true if 2x < -P, i.e. -2x > P (x two's complement)
template <int L>
__device__ __forceinline__ bool twice_lt_minus_P(const Limbs<L>& x, const uint32_t* P) {
  if (!(x.w[L - 1] >> 31)) return false;  // x >= 0
  Limbs<L> nx;                             // -x
  uint64_t carry = 1;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    uint64_t t = (uint64_t)(~x.w[i]) + carry;
    nx.w[i] = (uint32_t)t;
    carry = t >> 32;
  }
  Limbs<L> d;
  uint32_t c2 = 0;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    d.w[i] = (nx.w[i] << 1) | c2;
    c2 = nx.w[i] >> 31;
  }
  int res = 0;
#pragma unroll
  for (int i = L - 1; i >= 0; --i)
    if (res == 0 && d.w[i] != P[i]) res = d.w[i] > P[i] ? 1 : -1;
  return res > 0;
}

// binary64 bits of (-1)^neg mag 2^e, rounded to nearest even
template <int L>
__device__ __forceinline__ uint64_t round_to_binary64(const Limbs<L>& mag, uint32_t neg, int e) {
  const uint64_t sign = (uint64_t)neg << 63;
  const int nb = bitlen(mag);
  if (nb == 0) return 0ull;                               // X = 0 gives +0
  const int E = nb - 1 + e;                               // exponent of the leading bit
  if (E > 1023) return sign | 0x7ff0000000000000ull;
  const int lsb = E >= -1022 ? E - 52 : -1074;            // exponent of the last kept bit
  const int sh = lsb - e;                                 // low bits of mag dropped
  uint64_t q;
  if (sh <= 0) {
    q = bits64(mag, 0) << (-sh);                          // nb - sh <= 53 bits
  } else {
    q = sh < 32 * L ? bits64(mag, sh) : 0ull;
    const bool half = bit_at(mag, sh - 1);
    const bool sticky = any_below(mag, sh - 1);
    if (half && (sticky || (q & 1ull))) q += 1ull;
  }
  uint64_t b = E >= -1022 ? ((uint64_t)(E + 1022) << 52) + q : q;
  if (b >= 0x7ff0000000000000ull) b = 0x7ff0000000000000ull;
  return sign | b;
}

template <int L, int EPT>
__global__ void __launch_bounds__(256) reconstruct_kernel(const __grid_constant__ OzTables T, int64_t m, int64_t n,
                                                          const uint8_t* __restrict__ Y, int64_t ldy,
                                                          const int32_t* __restrict__ s,
                                                          const int32_t* __restrict__ t, double* __restrict__ C,
                                                          int64_t ldc) {
  constexpr int kMaxPairs = (OZ_MAX_MODULI + 1) / 2;
  const int64_t i = blockIdx.x;
  const int64_t j0 = ((int64_t)blockIdx.y * 256 + threadIdx.x) * EPT;
  if (i >= m || j0 >= n) return;
  const int Q = T.Q;
  const int npairs = T.npairs;
  const int64_t plane = m * ldy;
  const uint8_t* yp = Y + i * ldy + j0;
  const bool vec = (EPT == 4) && (j0 + 4 <= n) && ((reinterpret_cast<uintptr_t>(yp) & 3) == 0) &&
                   ((plane & 3) == 0);
  // S = sum over pairs (a, b) of z (P / (m_a m_b)), z = y_a m_b + y_b m_a < 2^17,
  // since y_a (P/m_a) + y_b (P/m_b) = (P / (m_a m_b)) (y_a m_b + y_b m_a).
  uint64_t acc[EPT][L];
  float f[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    f[e] = 0.f;
#pragma unroll
    for (int l = 0; l < L; ++l) acc[e][l] = 0;
  }
#pragma unroll
  for (int pi = 0; pi < kMaxPairs; ++pi) {
    if (pi < npairs) {
      const int qa = 2 * pi, qb = 2 * pi + 1;
      uint32_t da[EPT], db[EPT];
      if (vec) {
        const uint32_t wa = __ldg(reinterpret_cast<const uint32_t*>(yp + qa * plane));
        const uint32_t wb = qb < Q ? __ldg(reinterpret_cast<const uint32_t*>(yp + qb * plane)) : 0u;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          da[e] = (wa >> (8 * e)) & 0xffu;
          db[e] = (wb >> (8 * e)) & 0xffu;
        }
      } else {
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          da[e] = (j0 + e < n) ? __ldg(yp + qa * plane + e) : 0u;
          db[e] = (j0 + e < n && qb < Q) ? __ldg(yp + qb * plane + e) : 0u;
        }
      }
      const uint32_t ma = T.pa[pi], mb = T.pb[pi];
      const float pinv = T.pinv[pi];
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const uint32_t z = da[e] * mb + db[e] * ma;
        f[e] = fmaf(__int_as_float(0x4B000000 | z) - 8388608.0f, pinv, f[e]);
#pragma unroll
        for (int l = 0; l < L; ++l) acc[e][l] += (uint64_t)z * T.Np[pi][l];
      }
    }
  }
  const int32_t si = s[i];
  double out[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    Limbs<L> X;
    uint64_t carry = 0;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      uint64_t v = acc[e][l] + carry;
      X.w[l] = (uint32_t)v;
      carry = v >> 32;
    }
    const uint32_t qe = (uint32_t)__float2int_rn(f[e]);
    sub_mul_P(X, qe, T.P);
    if (twice_ge_P(X, T.P)) sub_mul_P(X, 1u, T.P);
    else if (twice_lt_minus_P(X, T.P)) add_P(X, T.P);
    const uint32_t neg = X.w[L - 1] >> 31;
    if (neg) {
      uint64_t c = 1;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        uint64_t v = (uint64_t)(~X.w[l]) + c;
        X.w[l] = (uint32_t)v;
        c = v >> 32;
      }
    }
    const int64_t j = j0 + e;
    const int ex = j < n ? -(si + t[j]) : 0;
    out[e] = __longlong_as_double((long long)round_to_binary64(X, neg, ex));
  }
  double* cp = C + i * ldc + j0;
  if (EPT == 4 && j0 + 4 <= n && (reinterpret_cast<uintptr_t>(cp) & 15) == 0) {
    reinterpret_cast<double2*>(cp)[0] = make_double2(out[0], out[1]);
    reinterpret_cast<double2*>(cp)[1] = make_double2(out[2], out[3]);
  } else {
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (j0 + e < n) cp[e] = out[e];
  }
}

typedef unsigned __int128 u128;

// binary64 bits of (-1)^neg mag 2^e for a 128-bit magnitude, nearest even
__device__ __forceinline__ uint64_t round128(u128 mag, uint32_t neg, int e) {
  const uint64_t sign = (uint64_t)neg << 63;
  const uint64_t hi = (uint64_t)(mag >> 64), lo = (uint64_t)mag;
  const int nb = hi ? 128 - __clzll((long long)hi) : (lo ? 64 - __clzll((long long)lo) : 0);
  if (nb == 0) return 0ull;
  const int E = nb - 1 + e;
  if (E > 1023) return sign | 0x7ff0000000000000ull;
  const int lsb = E >= -1022 ? E - 52 : -1074;
  const int sh = lsb - e;
  uint64_t q;
  if (sh <= 0) {
    q = lo << (-sh);                                   // at most 53 bits: exact
  } else if (sh > nb) {
    q = 0;                                             // below half of the last place
  } else if (sh == nb) {                               // the round bit is the leading bit
    const bool sticky = (mag & ~((u128)1 << (nb - 1))) != 0;
    q = sticky ? 1 : 0;                                // a tie goes to the even 0
  } else {                                             // 0 < sh < nb <= 128
    q = (uint64_t)(mag >> sh);
    const bool half = (mag >> (sh - 1)) & 1;
    const bool sticky = (mag & (((u128)1 << (sh - 1)) - 1)) != 0;
    if (half && (sticky || (q & 1ull))) q += 1ull;
  }
  uint64_t b = E >= -1022 ? ((uint64_t)(E + 1022) << 52) + q : q;
  if (b >= 0x7ff0000000000000ull) b = 0x7ff0000000000000ull;
  return sign | b;
}

// The same product for P < 2^125 (Q <= 16): X held in 128-bit integers, and
// the exact +-P correction only when the quotient estimate is within 1e-3 of
// a tie (X correct makes |f - q| = |X/P| + fp32 error < 1/2, so an estimate
// farther than 1e-3 from a tie cannot pick the wrong quotient). The pair
// count is a template parameter so that every digit load is issued before
// any arithmetic.
// One thread: entries (i, j0 .. j0 + 3).
template <int NP, int EPT>
__device__ __forceinline__ void reconstruct128_entries(const OzTables& T, int64_t i, int64_t j0, int64_t m, int64_t n,
                                                       const uint8_t* __restrict__ Y, int64_t ldy,
                                                       const int32_t* __restrict__ s, const int32_t* __restrict__ t,
                                                       double* __restrict__ C, int64_t ldc) {
  static_assert(EPT == 4, "one 32-bit digit word per plane");
  if (i >= m || j0 >= n) return;
  const int Q = T.Q;
  const int64_t plane = m * ldy;
  const uint8_t* yp = Y + i * ldy + j0;
  // whole 4-byte words whenever the row pitch has room (bytes past n are unused)
  const bool vec = (j0 + 4 <= ldy) && ((reinterpret_cast<uintptr_t>(yp) & 3) == 0) && ((plane & 3) == 0);
  uint32_t wa[NP], wb[NP];
  if (vec) {
#pragma unroll
    for (int pi = 0; pi < NP; ++pi) {
      wa[pi] = __ldg(reinterpret_cast<const uint32_t*>(yp + (2 * pi) * plane));
      wb[pi] = (2 * pi + 1 < Q) ? __ldg(reinterpret_cast<const uint32_t*>(yp + (2 * pi + 1) * plane)) : 0u;
    }
  } else {
#pragma unroll
    for (int pi = 0; pi < NP; ++pi) {
      uint32_t a = 0, b = 0;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        if (j0 + e < n) {
          a |= (uint32_t)__ldg(yp + (2 * pi) * plane + e) << (8 * e);
          if (2 * pi + 1 < Q) b |= (uint32_t)__ldg(yp + (2 * pi + 1) * plane + e) << (8 * e);
        }
      }
      wa[pi] = a;
      wb[pi] = b;
    }
  }
  uint64_t acc[EPT][4];
  float f[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    f[e] = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[e][l] = 0;
  }
#pragma unroll
  for (int pi = 0; pi < NP; ++pi) {
    const uint32_t ma = T.pa[pi], mb = T.pb[pi];
    const float pinv = T.pinv[pi];
    const uint32_t n0 = T.Np[pi][0], n1 = T.Np[pi][1], n2 = T.Np[pi][2], n3 = T.Np[pi][3];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const uint32_t z = __byte_perm(wa[pi], 0, 0x4440 + e) * mb + __byte_perm(wb[pi], 0, 0x4440 + e) * ma;
      f[e] = fmaf(__int_as_float(0x4B000000 | z) - 8388608.0f, pinv, f[e]);
      acc[e][0] += (uint64_t)z * n0;
      acc[e][1] += (uint64_t)z * n1;
      acc[e][2] += (uint64_t)z * n2;
      acc[e][3] += (uint64_t)z * n3;
    }
  }
  const u128 P = ((u128)(((uint64_t)T.P[3] << 32) | T.P[2]) << 64) | (((uint64_t)T.P[1] << 32) | T.P[0]);
  const int32_t si = s[i];
  double out[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    // S modulo 2^128 from the limb accumulators
    const uint64_t c0 = acc[e][0];
    const uint64_t c1 = acc[e][1] + (c0 >> 32);
    const uint64_t c2 = acc[e][2] + (c1 >> 32);
    const uint64_t c3 = acc[e][3] + (c2 >> 32);
    const uint64_t lo = (c0 & 0xffffffffull) | (c1 << 32);
    const uint64_t hi = (c2 & 0xffffffffull) | (c3 << 32);
    const float qf = rintf(f[e]);
    __int128 X = (__int128)((((u128)hi) << 64 | lo) - (u128)(uint32_t)qf * P);
    if (fabsf(f[e] - qf) > 0.499f) {               // near a tie: exact check of [-P/2, P/2)
      if (2 * X >= (__int128)P) X -= (__int128)P;
      else if (2 * X < -(__int128)P) X += (__int128)P;
    }
    const uint32_t neg = X < 0;
    const u128 mag = neg ? (u128)(-X) : (u128)X;
    const int64_t j = j0 + e;
    const int ex = j < n ? -(si + t[j]) : 0;
    // normalise the magnitude so that its leading bit is bit 63 of h
    const uint64_t mh = (uint64_t)(mag >> 64), ml = (uint64_t)mag;
    const int lz = mh ? __clzll((long long)mh) : 64 + (ml ? __clzll((long long)ml) : 64);
    const int nb = 128 - lz;
    const int E = nb - 1 + ex;
    uint64_t bits;
    if (nb == 0) {
      bits = 0;
    } else if (E >= -1022 && E <= 1023) {            // normal result: 53 bits, round, sticky
      const u128 nm = mag << lz;
      const uint64_t h = (uint64_t)(nm >> 64), l = (uint64_t)nm;
      const uint64_t m53 = h >> 11;
      const uint64_t half = (h >> 10) & 1ull;
      const uint64_t sticky = ((h & 0x3ffull) | l) != 0;
      const uint64_t q = m53 + (half & (sticky | (m53 & 1ull)));
      uint64_t b = ((uint64_t)(E + 1022) << 52) + q;
      if (b >= 0x7ff0000000000000ull) b = 0x7ff0000000000000ull;
      bits = ((uint64_t)neg << 63) | b;
    } else {
      bits = round128(mag, neg, ex);                 // subnormal or overflowing result
    }
    out[e] = __longlong_as_double((long long)bits);
  }
  double* cp = C + i * ldc + j0;
  if (j0 + 4 <= n && (reinterpret_cast<uintptr_t>(cp) & 15) == 0) {
    reinterpret_cast<double2*>(cp)[0] = make_double2(out[0], out[1]);
    reinterpret_cast<double2*>(cp)[1] = make_double2(out[2], out[3]);
  } else {
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (j0 + e < n) cp[e] = out[e];
  }
}

template <int NP, int EPT>
__global__ void __launch_bounds__(256) reconstruct128_kernel(const __grid_constant__ OzTables T, int64_t m,
                                                             int64_t n, const uint8_t* __restrict__ Y,
                                                             int64_t ldy, const int32_t* __restrict__ s,
                                                             const int32_t* __restrict__ t,
                                                             double* __restrict__ C, int64_t ldc) {
  reconstruct128_entries<NP, EPT>(T, blockIdx.x, ((int64_t)blockIdx.y * 256 + threadIdx.x) * EPT, m, n, Y, ldy, s, t,
                                  C, ldc);
}

// Grouped: a block covers 256 / tpr rows of one column chunk of 4 tpr entries
// (tpr = rec_tpr threads per row chunk, so short rows share a block); block b
// is row group l / nch, chunk l % nch of its problem, l = b - rec_begin.
template <int NP>
__global__ void __launch_bounds__(256) reconstruct128_grouped_kernel(const __grid_constant__ OzTables T,
                                                                     const OzGroupProblem* __restrict__ probs,
                                                                     int count) {
  const int64_t b = blockIdx.x;
  const int pi = group_find(probs, count, b, [](const OzGroupProblem& q) { return q.rec_begin; });
  const OzGroupProblem& P = probs[pi];
  const int tpr = P.rec_tpr, rows = 256 / tpr;
  const int64_t l = b - P.rec_begin, nch = (P.n + 4 * tpr - 1) / (4 * tpr);
  const int64_t i = (l / nch) * rows + threadIdx.x / tpr;
  const int64_t j0 = ((l % nch) * tpr + threadIdx.x % tpr) * 4;
  reconstruct128_entries<NP, 4>(T, i, j0, P.m, P.n, P.Y, P.ldy, P.s, P.t, P.C, P.ldc);
}

template <int NP>
cudaError_t launch128(const OzTables& T, int64_t m, int64_t n, const uint8_t* Y, int64_t ldy, const int32_t* s,
                      const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  constexpr int EPT = 4;
  dim3 grid((unsigned)m, (unsigned)((n + 256 * EPT - 1) / (256 * EPT)));
  reconstruct128_kernel<NP, EPT><<<grid, 256, 0, st>>>(T, m, n, Y, ldy, s, t, C, ldc);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_L(const OzTables& T, int64_t m, int64_t n, const uint8_t* Y, int64_t ldy, const int32_t* s,
                     const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  constexpr int EPT = 4;
  dim3 grid((unsigned)m, (unsigned)((n + 256 * EPT - 1) / (256 * EPT)));
  reconstruct_kernel<L, EPT><<<grid, 256, 0, st>>>(T, m, n, Y, ldy, s, t, C, ldc);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_reconstruct(const OzTables& T, int64_t m, int64_t n, const uint8_t* Y, int64_t ldy,
                               const int32_t* s, const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (ldy < n) return cudaErrorInvalidValue;
  if (T.limbs <= 4) {
    switch (T.npairs) {
      case 5: return launch128<5>(T, m, n, Y, ldy, s, t, C, ldc, st);
      case 6: return launch128<6>(T, m, n, Y, ldy, s, t, C, ldc, st);
      case 7: return launch128<7>(T, m, n, Y, ldy, s, t, C, ldc, st);
      case 8: return launch128<8>(T, m, n, Y, ldy, s, t, C, ldc, st);
      default: break;
    }
  }
  switch (T.limbs) {
    case 5: return launch_L<5>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 6: return launch_L<6>(T, m, n, Y, ldy, s, t, C, ldc, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_reconstruct_grouped(const OzTables& T, const OzGroupProblem* probs, int count, int64_t total_rec,
                                       cudaStream_t st) {
  if (count == 0 || total_rec == 0) return cudaSuccess;
  if (total_rec > INT32_MAX || T.limbs > 4) return cudaErrorInvalidValue;
  switch (T.npairs) {
    case 5: reconstruct128_grouped_kernel<5><<<(unsigned)total_rec, 256, 0, st>>>(T, probs, count); break;
    case 6: reconstruct128_grouped_kernel<6><<<(unsigned)total_rec, 256, 0, st>>>(T, probs, count); break;
    case 7: reconstruct128_grouped_kernel<7><<<(unsigned)total_rec, 256, 0, st>>>(T, probs, count); break;
    case 8: reconstruct128_grouped_kernel<8><<<(unsigned)total_rec, 256, 0, st>>>(T, probs, count); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace oz
