// oz_internal.h -- plan constants shared by the host planner and the kernels.
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

#include "../../include/oz.h"

#define OZ_MAX_LIMBS 6     // 32-bit limbs of the CRT sum: Q P < 2^192 for Q <= 20

// Everything a kernel needs about a configuration. Passed by value as a kernel
// parameter, so it lives in the constant bank and every access indexed by a
// compile-time or warp-uniform modulus index is a uniform load.
struct OzTables {
  int Q;                                  // number of moduli (one GEMM each)
  int bits;                               // beta: |A'| < 2^beta
  int limbs;                              // 32-bit limbs for X in the reconstruct phase
  int pad_;
  uint32_t m[OZ_MAX_MODULI];              // moduli, decreasing
  uint32_t half[OZ_MAX_MODULI];           // ceil(m/2): residues >= half map to r - m
  uint32_t magic[OZ_MAX_MODULI];          // floor(2^32 / m), Barrett constant
  uint32_t c18[OZ_MAX_MODULI];            // 2^18 mod m
  uint32_t c36[OZ_MAX_MODULI];            // 2^36 mod m
  uint32_t c54[OZ_MAX_MODULI];            // 2^54 mod m
  uint32_t inv[OZ_MAX_MODULI];            // (P/m)^-1 mod m: CRT coefficient
  float invm[OZ_MAX_MODULI];              // 1/m rounded to fp32: quotient estimate
  float mf[OZ_MAX_MODULI];                // m as fp32
  float hif[OZ_MAX_MODULI];               // ceil(m/2): a residue >= this maps to r - m
  float lof[OZ_MAX_MODULI];               // -floor(m/2): a residue below this maps to r + m
  float c15f[OZ_MAX_MODULI];              // 2^15 mod m, 2^30, 2^45, 2^60 mod m, each as the
  float c30f[OZ_MAX_MODULI];              // representative nearest zero (|c| <= 119)
  float c45f[OZ_MAX_MODULI];
  float c60f[OZ_MAX_MODULI];
  uint32_t Mk[OZ_MAX_MODULI][OZ_MAX_LIMBS];  // P/m as 32-bit limbs, least significant first
  uint32_t P[OZ_MAX_LIMBS];               // P = product of the moduli, 32-bit limbs
  // Moduli taken in pairs (a, b) = (2p, 2p+1) for the reconstruct phase; an odd
  // Q ends with a pair whose second modulus is 1 (digit 0).
  int npairs;
  uint32_t pa[(OZ_MAX_MODULI + 1) / 2];   // m_a
  uint32_t pb[(OZ_MAX_MODULI + 1) / 2];   // m_b (1 for a lone last modulus)
  float pinv[(OZ_MAX_MODULI + 1) / 2];    // 1 / (m_a m_b) rounded to fp32
  uint32_t Np[(OZ_MAX_MODULI + 1) / 2][OZ_MAX_LIMBS];  // P / (m_a m_b), 32-bit limbs
};

struct oz_plan_s {
  int Q;
  int bits;
  int engine;        // resolved engine (never AUTO)
  int64_t k_max;
  OzTables tab;
};

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

inline int64_t round_up(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

// Launchers (defined in the .cu files). Each returns cudaGetLastError().
cudaError_t launch_split_rows(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld,
                              int64_t nvec_pad, int64_t k_pad, int32_t* shifts, void* planes, int bf16,
                              int32_t* flag, cudaStream_t st);
cudaError_t launch_split_cols(const OzTables& t, int64_t nvec, int64_t len, const double* X, int64_t ld,
                              int64_t nvec_pad, int64_t k_pad, int32_t* shifts, void* planes, int bf16,
                              int32_t* flag, uint64_t* colmax, cudaStream_t st);
cudaError_t launch_gemm_imma(const OzTables& t, int64_t m, int64_t n, int64_t k_pad, const int8_t* U,
                             int64_t u_plane, const int8_t* V, int64_t v_plane, uint8_t* Y, int raw,
                             cudaStream_t st);
cudaError_t launch_gemm_tc(const OzTables& t, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                           const void* U, const void* V, uint8_t* Y, int raw, int32_t* status, cudaStream_t st);
cudaError_t launch_reconstruct(const OzTables& t, int64_t m, int64_t n, const uint8_t* Y, const int32_t* s,
                               const int32_t* tt, double* C, int64_t ldc, cudaStream_t st);

}  // namespace oz
