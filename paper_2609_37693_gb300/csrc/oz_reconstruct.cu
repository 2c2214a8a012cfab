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
// For byte digits with Q <= 16 the moduli are taken in groups instead
// (reconstruct_groups_kernel): triples (a, b, c) with
//   t = y_a (m_b m_c) + y_b (m_a m_c) + y_c (m_a m_b) < 3 m_a m_b m_c < 2^26,
// two packed 16-bit x 8-bit dot products (dp2a) of the three digit bytes,
// and for Q = 16 a last quad whose two pairs are reduced first (t < 2 M_4 <
// 2^32). S = sum_g t_g (P / M_g) then takes five groups of four 32-bit
// limbs instead of eight pairs: 20 wide multiply-adds per entry against 32,
// and no reduction inside the triples. S is formed modulo 2^128 (it can reach
// 15 P); its quotient by P comes from S / P = sum_g t_g / M_g in fp32 (all
// terms non-negative: within 2^-18), X = S - qP from a shared table of qP,
// and an estimate within 2^-10 of a tie is settled exactly. The kernel is persistent: each thread loads the digits of its next
// four entries before it reconstructs the current ones, so the loads of one
// chunk overlap the arithmetic of the last.
//
// The binary64 result fl(X 2^-(s_i + t_j)) is assembled from integer fields:
// the leading 53 bits (fewer below 2^-1022), round to nearest even from the
// round bit and the sticky bits, overflow to +-inf. No floating-point
// operation touches the value, so the rounding happens exactly once.
#include <stdint.h>

#include <type_traits>

#include "oz_internal.h"
#include "oz_device.cuh"

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

// D: the digit type, uint8_t (moduli below 256, Q <= 20) or uint16_t (the
// 16-bit digits of float-format configurations, moduli up to 4000 and up to
// OZ_TABLE_CAP channels).
template <int L, int EPT, typename D = uint8_t>
__global__ void __launch_bounds__(256) reconstruct_kernel(const __grid_constant__ OzTables T, int64_t m, int64_t n,
                                                          const D* __restrict__ Y, int64_t ldy,
                                                          const int32_t* __restrict__ s,
                                                          const int32_t* __restrict__ t, double* __restrict__ C,
                                                          int64_t ldc) {
  constexpr int kMaxPairs = ((sizeof(D) == 1 ? OZ_MAX_MODULI : OZ_TABLE_CAP) + 1) / 2;
  using W = typename std::conditional<sizeof(D) == 1, uint32_t, unsigned long long>::type;   // four digits
  const int64_t i = blockIdx.x;
  const int64_t j0 = ((int64_t)blockIdx.y * 256 + threadIdx.x) * EPT;
  if (i >= m || j0 >= n) return;
  const int Q = T.Q;
  const int npairs = T.npairs;
  const int64_t plane = m * ldy;
  const D* yp = Y + i * ldy + j0;
  const bool vec = (EPT == 4) && (j0 + 4 <= n) && ((reinterpret_cast<uintptr_t>(yp) & (sizeof(W) - 1)) == 0) &&
                   ((plane & 3) == 0);
  // S = sum over pairs (a, b) of z (P / (m_a m_b)), z = y_a m_b + y_b m_a
  // (< 2^17 for byte digits, < 2^25 for 16-bit ones), since
  // y_a (P/m_a) + y_b (P/m_b) = (P / (m_a m_b)) (y_a m_b + y_b m_a).
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
        constexpr int kb = 8 * (int)sizeof(D);
        constexpr uint32_t mask = sizeof(D) == 1 ? 0xffu : 0xffffu;
        const W wa = __ldg(reinterpret_cast<const W*>(yp + qa * plane));
        const W wb = qb < Q ? __ldg(reinterpret_cast<const W*>(yp + qb * plane)) : (W)0;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          da[e] = (uint32_t)(wa >> (kb * e)) & mask;
          db[e] = (uint32_t)(wb >> (kb * e)) & mask;
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
        f[e] = fmaf(sizeof(D) == 1 ? __int_as_float(0x4B000000 | z) - 8388608.0f : __uint2float_rn(z), pinv, f[e]);
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

// ---------------------------------------------------------------------------
// Byte digits in groups of moduli (Q <= 16; tables rg_* of OzTables).
// ---------------------------------------------------------------------------

// t_g of group g for entry e of the digit words w (byte e of each word is that
// entry's digit for one modulus)
template <int NT, int NP2, int NQ4>
__device__ __forceinline__ uint32_t group_t(int g, const uint32_t* w, int e, uint32_t w0, uint32_t w1, uint32_t m2a,
                                            uint32_t m2b) {
  const uint32_t s2 = (uint32_t)e | ((uint32_t)(4 + e) << 4);         // bytes [w_a.e, w_b.e, -, -]
  if (g < NT) {                                    // triple: moduli 3g, 3g+1, 3g+2
    const int q = 3 * g;
    const uint32_t s3 = 0x0010u | ((uint32_t)(4 + e) << 8);           // bytes [y.0, y.1, w_c.e, -]
    const uint32_t y = __byte_perm(__byte_perm(w[q], w[q + 1], s2), w[q + 2], s3);
    return __dp2a_lo(w0, y, __dp2a_hi(w1, y, 0u));
  }
  if (g < NT + NP2) {                              // pair
    const int q = 3 * NT + 2 * (g - NT);
    return __dp2a_lo(w0, __byte_perm(w[q], w[q + 1], s2), 0u);
  }
  const int q = 3 * NT + 2 * NP2;                  // quad: both pairs reduced, then combined
  const uint32_t zab = __dp2a_lo(w0, __byte_perm(w[q], w[q + 1], s2), 0u);
  const uint32_t zcd = __dp2a_lo(w1, __byte_perm(w[q + 2], w[q + 3], s2), 0u);
  const uint32_t wab = min(zab, zab - m2a);        // z < 2 M_2: z mod M_2
  const uint32_t wcd = min(zcd, zcd - m2b);
  return wab * m2b + wcd * m2a;                    // < 2 M_4 < 2^32
}

// The CRT sum of entry e of the digit words w[0..Q-1]: S modulo 2^128 as
// 32-bit limbs s[0..3], and f = sum_g fl(t_g) fl(1 / M_g), an estimate of
// S / P. Per limb l, a_l = sum_g t_g n_{g,l} in 64 bits (below 2^64: the sum
// of the largest t_g is below 2^32); only the low 32 bits of a_3 reach S.
template <int NT, int NP2, int NQ4>
__device__ __forceinline__ void crt_groups(const OzTables& T, const uint32_t* w, int e, uint32_t (&s)[4], float& f) {
  uint64_t a0 = 0, a1 = 0, a2 = 0;
  uint32_t a3 = 0;
  f = 0.0f;
#pragma unroll
  for (int g = 0; g < NT + NP2 + NQ4; ++g) {
    const bool quad = g >= NT + NP2;
    const uint32_t tg = group_t<NT, NP2, NQ4>(g, w, e, T.rg_w0[g], T.rg_w1[g], quad ? T.rg_m2a[g] : 0u,
                                              quad ? T.rg_m2b[g] : 0u);
    a0 += (uint64_t)tg * T.rg_N[g][0];
    a1 += (uint64_t)tg * T.rg_N[g][1];
    a2 += (uint64_t)tg * T.rg_N[g][2];
    a3 += tg * T.rg_N[g][3];
    f = fmaf(__uint2float_rn(tg), T.rg_invM[g], f);
  }
  // S = a0 + a1 2^32 + a2 2^64 + a3 2^96 modulo 2^128
  s[0] = (uint32_t)a0;
  asm("add.cc.u32 %0, %3, %4;\n\taddc.cc.u32 %1, %5, %6;\n\taddc.u32 %2, %7, %8;"
      : "=r"(s[1]), "=r"(s[2]), "=r"(s[3])
      : "r"((uint32_t)(a0 >> 32)), "r"((uint32_t)a1), "r"((uint32_t)(a1 >> 32)), "r"((uint32_t)a2),
        "r"((uint32_t)(a2 >> 32)), "r"(a3));
}

// x -= y over four 32-bit limbs (modulo 2^128)
__device__ __forceinline__ void sub128(uint32_t (&x)[4], const uint32_t (&y)[4]) {
  asm("sub.cc.u32 %0, %0, %4;\n\tsubc.cc.u32 %1, %1, %5;\n\tsubc.cc.u32 %2, %2, %6;\n\tsubc.u32 %3, %3, %7;"
      : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3])
      : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]));
}

__device__ __forceinline__ u128 to_u128(const uint32_t (&x)[4]) {
  return ((u128)(((uint64_t)x[3] << 32) | x[2]) << 64) | (((uint64_t)x[1] << 32) | x[0]);
}

// fl(X 2^ex) for X = S - qP, q the quotient estimate; kP[q] = q P (shared),
// in the usual case: the estimate clear of a tie, 2^96 <= |X| and a normal
// result. It runs in 32-bit limbs: the magnitude by a sign mask, the leading
// bit by clz of the top limb, 64 bits below it by funnel shifts, one
// round-to-nearest-even increment. Returns false (out unset) otherwise.
__device__ __forceinline__ bool round_groups_fast(const uint4* kP, const uint32_t (&s)[4], float f, int ex,
                                                  uint64_t& out) {
  const float kf = rintf(f);
  const int k = min((int)kf, 15);
  const uint4 kp = kP[k];
  uint32_t x[4] = {s[0], s[1], s[2], s[3]};
  const uint32_t kq[4] = {kp.x, kp.y, kp.z, kp.w};
  sub128(x, kq);
  // magnitude: (x ^ mask) - mask
  const uint32_t mask = (uint32_t)((int32_t)x[3] >> 31);
  uint32_t m[4] = {x[0] ^ mask, x[1] ^ mask, x[2] ^ mask, x[3] ^ mask};
  const uint32_t mk[4] = {mask, mask, mask, mask};
  sub128(m, mk);
  const int lz = __clz((int)m[3]);
  const int E = 127 - lz + ex;                             // exponent of the leading bit
  if (fabsf(f - kf) > 0.499f || m[3] == 0 || (unsigned)(E + 1022) > 2045u) return false;
  // 64 bits from the leading one down (h1:h0), and whether any bit below is set
  const uint32_t h1 = __funnelshift_l(m[2], m[3], lz);
  const uint32_t h0 = __funnelshift_l(m[1], m[2], lz);
  const uint32_t r = __funnelshift_l(m[0], m[1], lz) | (m[0] << lz);
  const uint64_t mant = (((uint64_t)h1 << 32) | h0) >> 11;  // 53 bits, leading one at bit 52
  const uint32_t half = (h0 >> 10) & 1u;
  const uint32_t sticky = ((h0 & 0x3ffu) | r) != 0u;
  const uint64_t q = mant + (half & (sticky | (uint32_t)mant));
  uint64_t b = ((uint64_t)(E + 1022) << 52) + q;            // a carry out of the significand bumps E
  if (b >= 0x7ff0000000000000ull) b = 0x7ff0000000000000ull;
  out = ((uint64_t)(mask & 1u) << 63) | b;
  return true;
}

// Every other case, recomputed from the digits (wsm[q * QS], this thread's
// shared-memory slots): the CRT sum S exactly in 128 bits (S < 15 P < 2^128),
// X = S - qP corrected exactly into [-P/2, P/2), and the general rounding.
template <int NT, int NP2, int NQ4, int QS>
__device__ __noinline__ uint64_t round_groups_slow(const OzTables& T, const uint4* kP, const uint32_t* wsm, int e,
                                                   int ex) {
  constexpr int Q = 3 * NT + 2 * NP2 + 4 * NQ4;
  uint32_t w[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) w[q] = wsm[q * QS];
  uint32_t s[4];
  float f;
  crt_groups<NT, NP2, NQ4>(T, w, e, s, f);
  const int k = min((int)rintf(f), 15);
  const uint4 kp = kP[k];
  const uint32_t kq[4] = {kp.x, kp.y, kp.z, kp.w};
  sub128(s, kq);
  __int128 X = (__int128)to_u128(s);
  const uint4 p = kP[1];
  const u128 P = ((u128)(((uint64_t)p.w << 32) | p.z) << 64) | (((uint64_t)p.y << 32) | p.x);
  if (2 * X >= (__int128)P) X -= (__int128)P;
  else if (2 * X < -(__int128)P) X += (__int128)P;
  const uint32_t neg = X < 0;
  const u128 mag = neg ? (u128)(-X) : (u128)X;
  return round128(mag, neg, ex);
}

// kP[q] = q P for q = 0..15, as four 32-bit limbs (threads 0..15 of the block)
__device__ __forceinline__ void fill_kP(const OzTables& T, uint4* kP) {
  if (threadIdx.x < 16) {
    const u128 P = ((u128)(((uint64_t)T.P[3] << 32) | T.P[2]) << 64) | (((uint64_t)T.P[1] << 32) | T.P[0]);
    const u128 v = P * (u128)threadIdx.x;
    kP[threadIdx.x] = make_uint4((uint32_t)v, (uint32_t)(v >> 32), (uint32_t)(v >> 64), (uint32_t)(v >> 96));
  }
}

// Four entries (i, j0 .. j0 + 3), j0 < n, from their digit words, which this
// thread holds in its shared-memory slots wsm[q * QS].
template <int NT, int NP2, int NQ4, int QS = 256>
__device__ __forceinline__ void rec4_groups(const OzTables& T, const uint4* kP, const uint32_t* wsm, int64_t i,
                                            int64_t j0, int64_t n, int32_t si, const int32_t* __restrict__ t,
                                            double* __restrict__ C, int64_t ldc) {
  constexpr int Q = 3 * NT + 2 * NP2 + 4 * NQ4;
  int32_t tj[4];
  if (j0 + 4 <= n && (reinterpret_cast<uintptr_t>(t + j0) & 15) == 0) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(t + j0));
    tj[0] = v.x, tj[1] = v.y, tj[2] = v.z, tj[3] = v.w;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) tj[e] = j0 + e < n ? __ldg(t + j0 + e) : 0;
  }
  uint32_t w[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) w[q] = wsm[q * QS];
  uint64_t out[4];
  uint32_t slow = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    uint32_t S[4];
    float f;
    crt_groups<NT, NP2, NQ4>(T, w, e, S, f);
    if (!round_groups_fast(kP, S, f, -(si + tj[e]), out[e])) slow |= 1u << e;
  }
  if (slow) {                                              // rare: one branch for the four entries
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if ((slow >> e) & 1u) out[e] = round_groups_slow<NT, NP2, NQ4, QS>(T, kP, wsm, e, -(si + tj[e]));
  }
  double* cp = C + i * ldc + j0;
  if (j0 + 4 <= n && (reinterpret_cast<uintptr_t>(cp) & 15) == 0) {
    __stcs(reinterpret_cast<double2*>(cp), make_double2(__longlong_as_double((long long)out[0]),
                                                        __longlong_as_double((long long)out[1])));
    __stcs(reinterpret_cast<double2*>(cp) + 1, make_double2(__longlong_as_double((long long)out[2]),
                                                            __longlong_as_double((long long)out[3])));
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (j0 + e < n) cp[e] = __longlong_as_double((long long)out[e]);
  }
}

// Asynchronous 4-byte copy global -> shared (cp.async, cached at all levels)
// and its group commit / wait.
__device__ __forceinline__ void cp_async4(uint32_t* smem_dst, const uint32_t* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t* smem_dst, const uint32_t* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// The digit words of the four entries (i, j0 .. j0 + 3) into this thread's
// slots buf[q * 256] of a shared buffer (nothing when j0 >= n). Whole words:
// the row pitch ldy is a multiple of 4 and j0 + 4 <= ldy.
template <int Q>
__device__ __forceinline__ void issue_digits(const uint8_t* __restrict__ Y, int64_t plane, int64_t ldy, int64_t i,
                                             int64_t j0, int64_t n, uint32_t* buf) {
  if (j0 < n) {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(Y + i * ldy + j0);
    const int64_t pw = plane >> 2;
#pragma unroll
    for (int q = 0; q < Q; ++q) cp_async4(buf + q * 256, p + q * pw);
  }
}

// The digit words of the eight entries (i, j0 .. j0 + 7) into this thread's
// slots buf[q * 512 + 0, 1] (two words per modulus: entries j0 .. j0 + 3 and
// j0 + 4 .. j0 + 7). Whole 8-byte runs: the row pitch ldy is a multiple of 8
// and j0 + 8 <= ldy.
template <int Q>
__device__ __forceinline__ void issue_digits8(const uint8_t* __restrict__ Y, int64_t plane, int64_t ldy, int64_t i,
                                              int64_t j0, int64_t n, uint32_t* buf) {
  if (j0 < n) {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(Y + i * ldy + j0);
    const int64_t pw = plane >> 2;
#pragma unroll
    for (int q = 0; q < Q; ++q) cp_async8(buf + q * 512, p + q * pw);
  }
}

// Persistent: block task b = (row group, column chunk), b advancing by the
// grid size. A task covers 256 / tpr rows of one chunk of 4 tpr entries (tpr
// threads per row: 256 for long rows, fewer for rows shorter than 1024, so
// that short rows do not leave threads idle). Every thread copies the next
// task's digit words into its own shared-memory slots (cp.async, two buffers)
// before it reconstructs the current task's four entries, so the loads of one
// task overlap the arithmetic of the last without holding registers; each
// thread reads only the slots it filled, so no barrier is needed.
template <int NT, int NP2, int NQ4>
__global__ void __launch_bounds__(256, 2) reconstruct_groups_kernel(const __grid_constant__ OzTables T, int64_t m,
                                                                    int64_t n, const uint8_t* __restrict__ Y,
                                                                    int64_t ldy, const int32_t* __restrict__ s,
                                                                    const int32_t* __restrict__ t,
                                                                    double* __restrict__ C, int64_t ldc,
                                                                    int64_t nch, int tpr_log2) {
  constexpr int Q = 3 * NT + 2 * NP2 + 4 * NQ4;
  __shared__ uint4 kP[16];
  __shared__ uint32_t buf[2][Q * 256];
  fill_kP(T, kP);
  __syncthreads();
  const int tpr = 1 << tpr_log2, rows = 256 >> tpr_log2;
  const int r_in = threadIdx.x >> tpr_log2, c_in = threadIdx.x & (tpr - 1);
  const int64_t plane = m * ldy;
  const int64_t ngroups = (m + rows - 1) / rows, total = ngroups * nch;
  const int64_t step_g = gridDim.x / nch, step_c = gridDim.x % nch;
  int64_t b = blockIdx.x, gi = b / nch, c = b % nch;
  uint32_t* const mine = buf[0] + threadIdx.x;       // slot s: mine + s * Q * 256
  int slot = 0;
  auto row_of = [&](int64_t g) { return g * rows + r_in; };
  auto col_of = [&](int64_t cc) { return (cc * tpr + c_in) * 4; };
  if (b < total && row_of(gi) < m) issue_digits<Q>(Y, plane, ldy, row_of(gi), col_of(c), n, mine);
  cp_async_commit();
  while (b < total) {
    int64_t bn = b + gridDim.x, gn = gi + step_g, cn = c + step_c;
    if (cn >= nch) cn -= nch, ++gn;
    if (bn < total && row_of(gn) < m) issue_digits<Q>(Y, plane, ldy, row_of(gn), col_of(cn), n, mine + (slot ^ 1) * Q * 256);
    cp_async_commit();
    cp_async_wait1();                       // this task's copies have landed
    const int64_t i = row_of(gi), j0 = col_of(c);
    if (i < m && j0 < n) rec4_groups<NT, NP2, NQ4>(T, kP, mine + slot * Q * 256, i, j0, n, __ldg(s + i), t, C, ldc);
    slot ^= 1;
    b = bn, gi = gn, c = cn;
  }
}

// As reconstruct_groups_kernel with eight entries per thread and task (a
// task covers 256 / tpr rows of one chunk of 8 tpr entries): one 8-byte copy
// per modulus per eight entries. The two digit buffers are dynamic shared
// memory, [2][Q][256 threads][2 words].
template <int NT, int NP2, int NQ4>
__global__ void __launch_bounds__(256, 2) reconstruct_groups8_kernel(const __grid_constant__ OzTables T, int64_t m,
                                                                     int64_t n, const uint8_t* __restrict__ Y,
                                                                     int64_t ldy, const int32_t* __restrict__ s,
                                                                     const int32_t* __restrict__ t,
                                                                     double* __restrict__ C, int64_t ldc,
                                                                     int64_t nch, int tpr_log2) {
  constexpr int Q = 3 * NT + 2 * NP2 + 4 * NQ4;
  __shared__ uint4 kP[16];
  extern __shared__ uint32_t dbuf[];
  fill_kP(T, kP);
  __syncthreads();
  const int tpr = 1 << tpr_log2, rows = 256 >> tpr_log2;
  const int r_in = threadIdx.x >> tpr_log2, c_in = threadIdx.x & (tpr - 1);
  const int64_t plane = m * ldy;
  const int64_t ngroups = (m + rows - 1) / rows, total = ngroups * nch;
  const int64_t step_g = gridDim.x / nch, step_c = gridDim.x % nch;
  int64_t b = blockIdx.x, gi = b / nch, c = b % nch;
  uint32_t* const mine = dbuf + 2 * threadIdx.x;    // slot s: mine + s * Q * 512
  int slot = 0;
  auto row_of = [&](int64_t g) { return g * rows + r_in; };
  auto col_of = [&](int64_t cc) { return (cc * tpr + c_in) * 8; };
  if (b < total && row_of(gi) < m) issue_digits8<Q>(Y, plane, ldy, row_of(gi), col_of(c), n, mine);
  cp_async_commit();
  while (b < total) {
    int64_t bn = b + gridDim.x, gn = gi + step_g, cn = c + step_c;
    if (cn >= nch) cn -= nch, ++gn;
    if (bn < total && row_of(gn) < m)
      issue_digits8<Q>(Y, plane, ldy, row_of(gn), col_of(cn), n, mine + (slot ^ 1) * Q * 512);
    cp_async_commit();
    cp_async_wait1();                       // this task's copies have landed
    const int64_t i = row_of(gi), j0 = col_of(c);
    if (i < m && j0 < n) {
      const int32_t si = __ldg(s + i);
      const uint32_t* w = mine + slot * Q * 512;
      rec4_groups<NT, NP2, NQ4, 512>(T, kP, w, i, j0, n, si, t, C, ldc);
      if (j0 + 4 < n) rec4_groups<NT, NP2, NQ4, 512>(T, kP, w + 1, i, j0 + 4, n, si, t, C, ldc);
    }
    slot ^= 1;
    b = bn, gi = gn, c = cn;
  }
}

// Grouped products: one block per task (256 / tpr rows of one column chunk
// of 8 tpr entries of problem map[b], tpr = rec_tpr threads per row chunk, so
// that short rows share a block; eight entries per thread, as in
// reconstruct_groups8_kernel), with the groups' sum. (A persistent form with a
// task of lookahead, as reconstruct_groups_kernel, ran the 256-product batch
// 3-8 % slower at four entries per thread.)
template <int NT, int NP2, int NQ4>
__global__ void __launch_bounds__(256) reconstruct_groups_grouped_kernel(const __grid_constant__ OzTables T,
                                                                         const OzGroupProblem* __restrict__ probs,
                                                                         const int32_t* __restrict__ map) {
  constexpr int Q = 3 * NT + 2 * NP2 + 4 * NQ4;
  __shared__ uint4 kP[16];
  extern __shared__ uint32_t dbuf[];                   // [Q][256 threads][2 words]
  fill_kP(T, kP);
  __syncthreads();
  const int64_t b = blockIdx.x;
  const OzGroupProblem& P = probs[__ldg(map + b)];
  const int tpr = P.rec_tpr, rows = 256 / tpr;
  const int64_t l = b - P.rec_begin, nch = (P.n + 8 * tpr - 1) / (8 * tpr);
  const int64_t i = (l / nch) * rows + threadIdx.x / tpr;
  const int64_t j0 = ((l % nch) * tpr + threadIdx.x % tpr) * 8;
  if (i >= P.m || j0 >= P.n) return;
  uint32_t* const mine = dbuf + 2 * threadIdx.x;
  issue_digits8<Q>(P.Y, P.m * P.ldy, P.ldy, i, j0, P.n, mine);
  cp_async_commit();
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  const int32_t si = __ldg(P.s + i);
  rec4_groups<NT, NP2, NQ4, 512>(T, kP, mine, i, j0, P.n, si, P.t, P.C, P.ldc);
  if (j0 + 4 < P.n) rec4_groups<NT, NP2, NQ4, 512>(T, kP, mine + 1, i, j0 + 4, P.n, si, P.t, P.C, P.ldc);
}

// Grouped: a block covers 256 / tpr rows of one column chunk of 4 tpr entries
// (tpr = rec_tpr threads per row chunk, so short rows share a block); block b
// is row group l / nch, chunk l % nch of its problem, l = b - rec_begin.
template <int NP>
__global__ void __launch_bounds__(256) reconstruct128_grouped_kernel(const __grid_constant__ OzTables T,
                                                                     const OzGroupProblem* __restrict__ probs,
                                                                     const int32_t* __restrict__ map) {
  const int64_t b = blockIdx.x;
  const OzGroupProblem& P = probs[__ldg(map + b)];
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

template <int L>
cudaError_t launch_L16(const OzTables& T, int64_t m, int64_t n, const uint16_t* Y, int64_t ldy, const int32_t* s,
                       const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  constexpr int EPT = 4;
  dim3 grid((unsigned)m, (unsigned)((n + 256 * EPT - 1) / (256 * EPT)));
  reconstruct_kernel<L, EPT, uint16_t><<<grid, 256, 0, st>>>(T, m, n, Y, ldy, s, t, C, ldc);
  return cudaGetLastError();
}

// CTAs of a kernel resident per SM, times the SM count (cached per device)
template <typename K>
int persistent_grid(K kernel, int threads) {
  static int cache[64][2];                    // [device] = {kernel-independent SM count, CTAs per SM}
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess) return 0;
  (void)cache;
  return sms * (per > 0 ? per : 1);
}

template <int NT, int NP2, int NQ4>
cudaError_t launch_groups(const OzTables& T, int64_t m, int64_t n, const uint8_t* Y, int64_t ldy, const int32_t* s,
                          const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  constexpr int Q = 3 * NT + 2 * NP2 + 4 * NQ4;
  if ((ldy & 7) == 0 && (reinterpret_cast<uintptr_t>(Y) & 7) == 0) {   // eight entries per thread
    int tpr_log2 = 5;                                // 32 .. 256 threads per row chunk of 8 tpr entries
    while (tpr_log2 < 8 && ((int64_t)8 << tpr_log2) < n) ++tpr_log2;
    const int64_t rows = 256 >> tpr_log2;
    const int64_t nch = (n + (8 << tpr_log2) - 1) / (8 << tpr_log2);
    const int64_t total = ((m + rows - 1) / rows) * nch;
    const int smem = 2 * Q * 256 * 8;
    cudaError_t e = cudaFuncSetAttribute(reconstruct_groups8_kernel<NT, NP2, NQ4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, reconstruct_groups8_kernel<NT, NP2, NQ4>, 256, smem) !=
            cudaSuccess)
      return cudaErrorInvalidValue;
    int64_t grid = (int64_t)sms * (per > 0 ? per : 1);
    if (grid > total) grid = total;
    reconstruct_groups8_kernel<NT, NP2, NQ4><<<(unsigned)grid, 256, smem, st>>>(T, m, n, Y, ldy, s, t, C, ldc, nch,
                                                                               tpr_log2);
    return cudaGetLastError();
  }
  int tpr_log2 = 5;                                  // 32 .. 256 threads per row chunk of 4 tpr entries
  while (tpr_log2 < 8 && ((int64_t)4 << tpr_log2) < n) ++tpr_log2;
  const int64_t rows = 256 >> tpr_log2;
  const int64_t nch = (n + (4 << tpr_log2) - 1) / (4 << tpr_log2);
  const int64_t total = ((m + rows - 1) / rows) * nch;
  int grid = persistent_grid(reconstruct_groups_kernel<NT, NP2, NQ4>, 256);
  if (grid <= 0) return cudaErrorInvalidValue;
  if ((int64_t)grid > total) grid = (int)total;
  reconstruct_groups_kernel<NT, NP2, NQ4><<<grid, 256, 0, st>>>(T, m, n, Y, ldy, s, t, C, ldc, nch, tpr_log2);
  return cudaGetLastError();
}

// The group shape of a plan (oz_plan.cpp, fill_group_tables), as a switch
// over the shapes Q = 9 .. 16 give: -1 if the plan has none.
int group_shape(const OzTables& T) {
  const int key = T.rg_nt * 100 + T.rg_np2 * 10 + T.rg_nq4;
  switch (key) {
    case 300: case 220: case 310: case 400: case 301: case 320: case 410: case 500: case 401: case 420:
      return key;
    default: return -1;
  }
}

template <typename F>
cudaError_t with_shape(int key, F f) {
  switch (key) {
    case 300: return f(std::integral_constant<int, 3>(), std::integral_constant<int, 0>(), std::integral_constant<int, 0>());
    case 220: return f(std::integral_constant<int, 2>(), std::integral_constant<int, 2>(), std::integral_constant<int, 0>());
    case 310: return f(std::integral_constant<int, 3>(), std::integral_constant<int, 1>(), std::integral_constant<int, 0>());
    case 400: return f(std::integral_constant<int, 4>(), std::integral_constant<int, 0>(), std::integral_constant<int, 0>());
    case 301: return f(std::integral_constant<int, 3>(), std::integral_constant<int, 0>(), std::integral_constant<int, 1>());
    case 320: return f(std::integral_constant<int, 3>(), std::integral_constant<int, 2>(), std::integral_constant<int, 0>());
    case 410: return f(std::integral_constant<int, 4>(), std::integral_constant<int, 1>(), std::integral_constant<int, 0>());
    case 500: return f(std::integral_constant<int, 5>(), std::integral_constant<int, 0>(), std::integral_constant<int, 0>());
    case 401: return f(std::integral_constant<int, 4>(), std::integral_constant<int, 0>(), std::integral_constant<int, 1>());
    case 420: return f(std::integral_constant<int, 4>(), std::integral_constant<int, 2>(), std::integral_constant<int, 0>());
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Whether the grouped reconstruct of a plan's products takes the groups'
// kernel (eight entries per thread) rather than the pairs' (four).
bool reconstruct_grouped_eight(const OzTables& T) { return group_shape(T) >= 0; }

// 16-bit digits with P of five or six 32-bit limbs (widened float-format plans)
cudaError_t launch_reconstruct16_wide(const OzTables& T, int64_t m, int64_t n, const uint16_t* Y, int64_t ldy,
                                      const int32_t* s, const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (ldy < n || T.npairs > (OZ_TABLE_CAP + 1) / 2) return cudaErrorInvalidValue;
  switch (T.limbs) {
    case 5: return launch_L16<5>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 6: return launch_L16<6>(T, m, n, Y, ldy, s, t, C, ldc, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_reconstruct(const OzTables& T, int64_t m, int64_t n, const uint8_t* Y, int64_t ldy,
                               const int32_t* s, const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (ldy < n) return cudaErrorInvalidValue;
  // byte digits in groups: whole 4-byte digit words need a row pitch and base
  // that are multiples of 4
  const int shape = group_shape(T);
  if (shape >= 0 && (ldy & 3) == 0 && (reinterpret_cast<uintptr_t>(Y) & 3) == 0) {
    return with_shape(shape, [&](auto nt, auto np2, auto nq4) {
      return launch_groups<decltype(nt)::value, decltype(np2)::value, decltype(nq4)::value>(T, m, n, Y, ldy, s, t, C,
                                                                                            ldc, st);
    });
  }
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

namespace {

// Y[0] += Y[1] + ... + Y[nsplit - 1] modulo the plane's modulus, 16 bytes per
// thread (byte-wise modular adds; bytes past n in a row are summed too and
// never read).
__global__ void __launch_bounds__(256) combine_digits_kernel(const __grid_constant__ OzTables T, int64_t plane16,
                                                             int64_t total16, uint8_t* __restrict__ Y, int nsplit,
                                                             int64_t ysplit) {
  const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (c >= total16) return;
  const int q = (int)(c / plane16);
  const uint32_t mm = T.m[q] * 0x01010101u;
  uint4* dst = reinterpret_cast<uint4*>(Y) + c;
  uint4 a = *dst;
  for (int j = 1; j < nsplit; ++j) {
    const uint4 b = __ldcs(reinterpret_cast<const uint4*>(Y + j * ysplit) + c);
    a.x = addmod_bytes(a.x, b.x, mm);
    a.y = addmod_bytes(a.y, b.y, mm);
    a.z = addmod_bytes(a.z, b.z, mm);
    a.w = addmod_bytes(a.w, b.w, mm);
  }
  *dst = a;
}

}  // namespace

cudaError_t launch_combine_digits(const OzTables& T, int64_t m, int64_t ldy, uint8_t* Y, int nsplit, int64_t ysplit,
                                  cudaStream_t st) {
  if (nsplit <= 1 || m == 0) return cudaSuccess;
  if ((ldy & 15) || (ysplit & 15) || (reinterpret_cast<uintptr_t>(Y) & 15)) return cudaErrorInvalidValue;
  const int64_t plane16 = m * ldy / 16, total16 = plane16 * T.Q;
  const int64_t blocks = (total16 + 255) / 256;
  if (blocks > INT32_MAX) return cudaErrorInvalidValue;
  combine_digits_kernel<<<(unsigned)blocks, 256, 0, st>>>(T, plane16, total16, Y, nsplit, ysplit);
  return cudaGetLastError();
}

cudaError_t launch_reconstruct_grouped(const OzTables& T, const OzGroupProblem* probs, const GroupMaps& maps,
                                       int64_t total_rec, cudaStream_t st) {
  if (total_rec == 0) return cudaSuccess;
  if (total_rec > INT32_MAX) return cudaErrorInvalidValue;
  // every grouped problem's digit rows have a pitch of a multiple of 16 bytes
  const int shape = group_shape(T);
  if (shape >= 0) {
    return with_shape(shape, [&](auto nt, auto np2, auto nq4) {
      constexpr int Q = 3 * decltype(nt)::value + 2 * decltype(np2)::value + 4 * decltype(nq4)::value;
      auto kernel = reconstruct_groups_grouped_kernel<decltype(nt)::value, decltype(np2)::value, decltype(nq4)::value>;
      const int smem = Q * 256 * 8;
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      kernel<<<(unsigned)total_rec, 256, smem, st>>>(T, probs, maps.rec);
      return cudaGetLastError();
    });
  }
  if (T.limbs > 4) return cudaErrorInvalidValue;
  switch (T.npairs) {
    case 5: reconstruct128_grouped_kernel<5><<<(unsigned)total_rec, 256, 0, st>>>(T, probs, maps.rec); break;
    case 6: reconstruct128_grouped_kernel<6><<<(unsigned)total_rec, 256, 0, st>>>(T, probs, maps.rec); break;
    case 7: reconstruct128_grouped_kernel<7><<<(unsigned)total_rec, 256, 0, st>>>(T, probs, maps.rec); break;
    case 8: reconstruct128_grouped_kernel<8><<<(unsigned)total_rec, 256, 0, st>>>(T, probs, maps.rec); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace oz
