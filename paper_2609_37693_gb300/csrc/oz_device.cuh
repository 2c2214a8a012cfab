// oz_device.cuh -- device helpers shared by the kernels: the IEEE-field view
// of eq. convert (split kernels, INT8 and float-format planes) and the
// modular byte sum of the blocked call's epilogues.
#pragma once

#include <stdint.h>

namespace oz {

constexpr uint64_t kAbsMask = 0x7fffffffffffffffull;

// Shift s from the largest |x| bit pattern.
static __device__ __forceinline__ int32_t shift_from_maxbits(uint64_t mb, int beta) {
  if (mb == 0) return 0;
  int eb = (int)(mb >> 52);
  int e = eb ? eb - 1022 : (64 - __clzll((long long)mb)) - 1074;  // frexp exponent
  return beta - e;
}

// Decoded truncated integer of one entry: |a'| and its sign.
struct Trunc {
  uint64_t mag;
  uint32_t neg;
};

static __device__ __forceinline__ Trunc truncate(uint64_t bits, int32_t s) {
  Trunc t;
  t.neg = (uint32_t)(bits >> 63);
  int eb = (int)((bits >> 52) & 0x7ff);
  uint64_t f = bits & ((1ull << 52) - 1);
  uint64_t mant = eb ? (f | (1ull << 52)) : f;
  int sh = (eb ? eb - 1075 : -1074) + s;   // a' = mant * 2^sh, |a'| < 2^beta <= 2^64
  if (sh >= 0) t.mag = mant << sh;         // sh <= 11 when beta <= 64 (wider: truncate_wide)
  else t.mag = (-sh) >= 64 ? 0ull : (mant >> (-sh));
  return t;
}

// The same for a widened budget (beta up to 84): |a'| < 2^84 needs 128 bits.
struct TruncWide {
  unsigned __int128 mag;
  uint32_t neg;
};

static __device__ __forceinline__ TruncWide truncate_wide(uint64_t bits, int32_t s) {
  TruncWide t;
  t.neg = (uint32_t)(bits >> 63);
  int eb = (int)((bits >> 52) & 0x7ff);
  uint64_t f = bits & ((1ull << 52) - 1);
  uint64_t mant = eb ? (f | (1ull << 52)) : f;
  int sh = (eb ? eb - 1075 : -1074) + s;   // a' = mant * 2^sh, |a'| < 2^beta <= 2^84
  if (sh >= 0) t.mag = (unsigned __int128)mant << sh;   // sh <= 31
  else t.mag = (-sh) >= 64 ? 0 : (unsigned __int128)(mant >> (-sh));
  return t;
}

// 64-bit max across a warp.
static __device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// (a + b) mod m in each byte, for bytes a, b in [0, m) and m < 256 given as
// mm = m * 0x01010101: a - (m - b), plus m in the bytes where that borrows.
// The GEMM epilogues of a blocked call add a slab's digits into the earlier
// slabs' this way.
static __device__ __forceinline__ uint32_t addmod_bytes(uint32_t a, uint32_t b, uint32_t mm) {
  const uint32_t c = __vsub4(mm, b);
  const uint32_t lt = __vcmpltu4(a, c);
  return __vadd4(__vsub4(a, c), lt & mm);
}

}  // namespace oz
