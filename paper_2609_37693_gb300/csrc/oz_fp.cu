// oz_fp.cu -- the five phases on a low-precision float configuration
// (Sec. "Forms and Channels"; oz_plan_fp.cpp builds the configuration).
//
// Reduce: for every entry and channel, the class c = a' mod m in [0, m)
// (a' = trunc(x 2^s) from the IEEE fields, cut into 16-bit pieces, one 32-bit
// Barrett step), then the channel's code word of c from the plan's tables:
// byte q of the word is the code of the plane value the form assigns to c in
// plane q (the sign of a' selects the second half of the table, where entry r
// holds the word of class (m - r) mod m). Planes are K-major rows: 8-bit codes
// one per byte; 6-bit codes packed little-endian 16 to a 16-byte chunk whose
// last 4 bytes are zero (the shared-memory layout kind::f8f6f4 reads for 6-bit
// types, so a K = 32 step is 32 bytes for 8- and 6-bit formats); 4-bit codes
// two per byte, densely (the block-scaled kind::mxf4 layout, K = 64 per 32
// bytes).
//
// GEMMs and epilogue: tcgen05.mma.kind::f8f6f4 on the codes (E4M3, E5M2, E2M3,
// E3M2 or E2M1) into FP32 accumulators in tensor memory. The work unit is a
// (channel, 128 x 256 tile); its GEMMs run one after another, each over the
// whole inner dimension in one accumulator (every plane value is at most
// floor(sqrt(2^24 / K)), eq. ov-accgen), and the epilogue folds GEMM k as
//   r <- r + lambda_k (W_k mod m)  (mod m)                 (order R>C)
// in exact fp32 arithmetic, keeping r (|r| < 0.51 m) as a 16-bit field per
// entry in registers; at the end of the unit it writes the CRT digit
// (W mod m) (P/m)^-1 mod m, or W mod m, as uint16.
//
// Reconstruct: the CRT of Sec. "Around the GEMMs" on 16-bit digits, moduli
// taken in pairs as in oz_reconstruct.cu.
#include <cuda.h>
#include <stdint.h>

#include "oz_device.cuh"
#include "oz_internal.h"
#include "oz_sync.cuh"
#include "oz_pair.cuh"

namespace oz {
namespace {

// =========================================================================
// Reduce
// =========================================================================

struct ChConst {
  uint32_t m, magic, c16, c32, c48, c64;
};

__device__ __forceinline__ ChConst ch_const(const OzFpTables& F, int c) {
  ChConst k;
  k.m = F.m[c];
  k.magic = F.magic[c];
  k.c16 = F.c16[c];
  k.c32 = F.c32[c];
  k.c48 = F.c48[c];
  k.c64 = F.c64[c];
  return k;
}

// 16-bit pieces of |a'| (the sign is kept apart, one bit per entry); p4 (bits
// 64..79) only for a widened budget, beta > 64
struct Pieces16 {
  uint32_t p0, p1, p2, p3, p4;
};

__device__ __forceinline__ Pieces16 pieces16(uint64_t mag, uint32_t top = 0) {
  Pieces16 P;
  P.p0 = (uint32_t)mag & 0xffffu;
  P.p1 = (uint32_t)(mag >> 16) & 0xffffu;
  P.p2 = (uint32_t)(mag >> 32) & 0xffffu;
  P.p3 = (uint32_t)(mag >> 48);
  P.p4 = top;
  return P;
}

// Index of the code word of a' = +-|a'|: the class r of |a'| (y < 2^16 (1 + 4 * 4095)
// < 2^32, one Barrett step), plus m for a negative entry, whose class is (m - r) mod m.
template <bool WIDE>
__device__ __forceinline__ uint32_t word_index(const ChConst& k, const Pieces16& P, uint32_t neg) {
  uint32_t y = P.p0 + P.p1 * k.c16 + P.p2 * k.c32 + P.p3 * k.c48;
  if (WIDE) y += P.p4 * k.c64;
  return mod_barrett(y, k.m, k.magic) + (neg ? k.m : 0u);
}

// byte q of each of w0..w3, as the bytes of one word
__device__ __forceinline__ uint32_t gather4(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, int q) {
  const uint32_t sel = (uint32_t)q | ((uint32_t)(q + 4) << 4);
  return __byte_perm(__byte_perm(w0, w1, sel), __byte_perm(w2, w3, sel), 0x5410);
}

// four codes held one per byte -> 6-bit fields packed little-endian (24 bits)
__device__ __forceinline__ uint32_t pack6(uint32_t g) {
  return (g & 0x3Fu) | ((g >> 2) & 0xFC0u) | ((g >> 4) & 0x3F000u) | ((g >> 6) & 0xFC0000u);
}
// four codes held one per byte -> 4-bit fields packed little-endian (16 bits)
__device__ __forceinline__ uint32_t pack4(uint32_t g) {
  const uint32_t t = (g | (g >> 4)) & 0x00FF00FFu;
  return (t | (t >> 8)) & 0xFFFFu;
}

// Plane q's bits for 8 consecutive entries whose code words are w[0..7]:
// 8-bit codes: 64 bits; 6-bit: 48 bits; 4-bit: 32 bits (little-endian).
template <int CB>
__device__ __forceinline__ uint64_t plane_bits8(const uint32_t (&w)[8], int q) {
  const uint32_t g0 = gather4(w[0], w[1], w[2], w[3], q);
  const uint32_t g1 = gather4(w[4], w[5], w[6], w[7], q);
  if constexpr (CB == 8) return (uint64_t)g0 | ((uint64_t)g1 << 32);
  else if constexpr (CB == 6) return (uint64_t)pack6(g0) | ((uint64_t)pack6(g1) << 24);
  else return (uint64_t)(pack4(g0) | (pack4(g1) << 16));
}

// The 16-byte chunk of 16 entries of 6-bit codes from the 48-bit fields of
// entries 0..7 (a) and 8..15 (b); bytes 12..15 zero.
__device__ __forceinline__ uint4 chunk6(uint64_t a, uint64_t b) {
  return make_uint4((uint32_t)a, (uint32_t)(a >> 32) | ((uint32_t)b << 16), (uint32_t)(b >> 16), 0u);
}

// Entry bits: |a'| pieces and sign of x (non-finite entries count as 0);
// WIDE: |a'| < 2^80 in 128 bits (beta up to 72).
template <bool WIDE>
__device__ __forceinline__ Pieces16 load_entry(uint64_t b, int32_t s, uint32_t& neg) {
  if (((b >> 52) & 0x7ff) == 0x7ff) b = 0;
  if constexpr (WIDE) {
    const TruncWide t = truncate_wide(b, s);
    neg = t.neg && t.mag != 0;
    return pieces16((uint64_t)t.mag, (uint32_t)(t.mag >> 64) & 0xffffu);
  } else {
    const Trunc t = truncate(b, s);
    neg = t.neg && t.mag;
    return pieces16(t.mag);
  }
}

// Contiguous vectors: one CTA of 256 threads per vector, 8 entries per thread
// and pass; planes [nplanes][nvec_pad][row bytes of k_pad entries]. For 6-bit
// codes the two threads of a 16-entry chunk meet by a shuffle.
template <int CB, bool WIDE>
__global__ void __launch_bounds__(256) split_fp_rows_kernel(const __grid_constant__ OzFpTables F, int bits,
                                                            int64_t nvec, int64_t len, const double* __restrict__ X,
                                                            int64_t ld, int64_t nvec_pad, int64_t k_pad,
                                                            int32_t* __restrict__ shifts, uint8_t* __restrict__ planes,
                                                            int32_t* __restrict__ flag, bool given) {
  __shared__ uint64_t red[8];
  __shared__ int32_t s_sh;
  const int64_t v = blockIdx.x;
  const int tid = threadIdx.x;
  const bool live = v < nvec;
  const uint64_t* row = reinterpret_cast<const uint64_t*>(X) + (live ? v * ld : 0);
  int32_t s;
  if (given) {                      // the shift of the whole row is known (blocked call)
    s = live ? shifts[v] : 0;
  } else {
    uint64_t mx = 0;
    uint32_t bad = 0;
    if (live) {
      for (int64_t h = tid; h < len; h += 256) {
        uint64_t b = __ldg(row + h) & kAbsMask;
        bad |= (uint32_t)((b >> 52) == 0x7ff);
        mx = b > mx ? b : mx;
      }
    }
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
      int32_t s0 = live ? shift_from_maxbits(anybad ? 0 : m, bits) : 0;
      s_sh = s0;
      if (live) shifts[v] = s0;
    }
    __syncthreads();
    s = s_sh;
  }
  const int64_t row_bytes = CB == 4 ? k_pad / 2 : k_pad;
  const int64_t plane = nvec_pad * row_bytes;
  uint8_t* out_row = planes + v * row_bytes;
  // every thread runs every pass (the shuffle of the 6-bit path needs both lanes)
  for (int64_t base = 0; base < k_pad; base += 256 * 8) {
    const int64_t h0 = base + (int64_t)tid * 8;
    const bool active = h0 < k_pad;
    Pieces16 P[8];
    uint32_t negm = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint64_t b = (live && h0 + e < len) ? __ldg(row + h0 + e) : 0ull;
      uint32_t ng;
      P[e] = load_entry<WIDE>(b, s, ng);
      negm |= ng << e;
    }
    for (int c = 0; c < F.nch; ++c) {
      const ChConst k = ch_const(F, c);
      const uint32_t* tw = F.words + F.ch_woff[c];
      uint32_t w[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) w[e] = __ldg(tw + word_index<WIDE>(k, P[e], (negm >> e) & 1u));
      const int p0 = F.ch_plane0[c], np = F.ch_nplanes[c];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q >= np) break;
        uint8_t* dst = out_row + (int64_t)(p0 + q) * plane;
        const uint64_t pb = plane_bits8<CB>(w, q);
        if constexpr (CB == 8) {
          if (active) *reinterpret_cast<uint2*>(dst + h0) = make_uint2((uint32_t)pb, (uint32_t)(pb >> 32));
        } else if constexpr (CB == 4) {
          if (active) *reinterpret_cast<uint32_t*>(dst + h0 / 2) = (uint32_t)pb;
        } else {
          const uint64_t other = __shfl_xor_sync(0xffffffffu, pb, 1);
          if (active && (tid & 1) == 0) *reinterpret_cast<uint4*>(dst + h0) = chunk6(pb, other);
        }
      }
    }
  }
}

// Strided vectors (columns of B, or of A^T): 64 (vector) x 32 (h) tiles; lane
// groups of 4 take the 32 entries of one vector, 8 each, so that a vector's
// plane bits leave the group as one 32-, 24- (two chunks) or 16-byte piece of
// its plane row; 6-bit pairs meet by a shuffle. No shared memory.
template <int CB, bool WIDE>
__global__ void __launch_bounds__(256) split_fp_cols_kernel(const __grid_constant__ OzFpTables F, int64_t nvec,
                                                            int64_t len, const double* __restrict__ X, int64_t ld,
                                                            int64_t nvec_pad, int64_t k_pad,
                                                            const int32_t* __restrict__ shifts,
                                                            uint8_t* __restrict__ planes) {
  const int tid = threadIdx.x;
  const int hg = tid & 3;                              // entries hbase + 8 hg .. + 7
  const int jl = tid >> 2;
  const int64_t j = (int64_t)blockIdx.x * 64 + jl;
  const int64_t hbase = (int64_t)blockIdx.y * 32;
  const bool live = j < nvec;
  const int32_t s = live ? shifts[j] : 0;
  Pieces16 P[8];
  uint32_t negm = 0;
  const uint64_t* Xb = reinterpret_cast<const uint64_t*>(X);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t h = hbase + hg * 8 + e;
    const uint64_t b = (live && h < len) ? __ldg(Xb + h * ld + j) : 0ull;
    uint32_t ng;
    P[e] = load_entry<WIDE>(b, s, ng);
    negm |= ng << e;
  }
  const int64_t row_bytes = CB == 4 ? k_pad / 2 : k_pad;
  const int64_t plane = nvec_pad * row_bytes;
  uint8_t* out = planes + j * row_bytes + (CB == 4 ? (hbase + hg * 8) / 2 : hbase + hg * 8);
  for (int c = 0; c < F.nch; ++c) {
    const ChConst k = ch_const(F, c);
    const uint32_t* tw = F.words + F.ch_woff[c];
    uint32_t w[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) w[e] = __ldg(tw + word_index<WIDE>(k, P[e], (negm >> e) & 1u));
    const int p0 = F.ch_plane0[c], np = F.ch_nplanes[c];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q >= np) break;
      uint8_t* dst = out + (int64_t)(p0 + q) * plane;
      const uint64_t pb = plane_bits8<CB>(w, q);
      if constexpr (CB == 8) {
        *reinterpret_cast<uint2*>(dst) = make_uint2((uint32_t)pb, (uint32_t)(pb >> 32));
      } else if constexpr (CB == 4) {
        *reinterpret_cast<uint32_t*>(dst) = (uint32_t)pb;
      } else {
        const uint64_t other = __shfl_xor_sync(0xffffffffu, pb, 1);
        if ((hg & 1) == 0) *reinterpret_cast<uint4*>(dst) = chunk6(pb, other);
      }
    }
  }
}

// =========================================================================
// GEMMs + epilogue (tcgen05, kind::f8f6f4)
// =========================================================================

constexpr int BM = 128, BK = 128;                  // BK = 128 bytes of a plane row per stage
constexpr int kBand = 8;
constexpr int A_BYTES = BM * BK;                   // 16 KiB
constexpr int kEpiWarps = 8;
constexpr int kThreads = (2 + kEpiWarps) * 32;
constexpr int kTmemCols = 512;
constexpr uint32_t kSfaCol = 448, kSfbCol = 480;   // unit block scales (block-scaled FP4 only)

// Two configurations of the GEMM kernel:
//  * kind::f8f6f4 (E4M3, E5M2, E2M3, E3M2): 128 x 256 tiles, a stage holds 128
//    entries per row (four K = 32 MMAs), two 256-column accumulators fill TMEM;
//  * kind::mxf4 block-scaled (E2M1 at the 4-bit rate, every scale 1): codes two
//    per byte, a stage holds 256 entries per row (four K = 64 MMAs); 128 x 192
//    tiles so that two accumulators (384 columns) leave room for the scales.
template <bool MX>
struct Cfg {
  static constexpr int BN = MX ? 192 : 256;
  static constexpr int HC = BN / 2;                 // columns per epilogue warp
  static constexpr int NCH = HC / 32;               // 32-column TMEM loads per warp
  static constexpr int STAGES = MX ? 5 : 4;
  static constexpr int B_BYTES = BN * BK;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int kSmemBytes = STAGES * STAGE_BYTES + 256 + 1024;
  static constexpr int KSTAGE = MX ? 2 * BK : BK;   // entries per stage row
};

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma_f8f6f4(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_mxf4(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tmem_st32_fill(uint32_t taddr, uint32_t u) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
      "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(taddr),
      "r"(u)
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// K-major 128-byte-swizzled operand (rows of 128 bytes, groups of 8 rows 1024 B apart)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct Unit {
  int c, tm, tn;
};

__device__ __forceinline__ Unit unit_coord(int t, int tiles_m, int tiles_n) {
  const int per_c = tiles_m * tiles_n;
  Unit u;
  u.c = t / per_c;
  const int r = t - u.c * per_c;
  const int band = r / (tiles_m * kBand);
  const int rb = r - band * tiles_m * kBand;
  const int bw = min(kBand, tiles_n - band * kBand);
  u.tm = rb / bw;
  u.tn = band * kBand + (rb - u.tm * bw);
  return u;
}

struct FpParams {
  int m, n, tiles_m, tiles_n, num_units, kblocks, m_pad, n_pad, raw;
  int acc;           // add into the digits already in Y, modulo the channel's m (blocked call)
  uint32_t idesc;
  uint16_t* Y;
  int64_t ldy;       // row pitch of Y (entries)
  int32_t* status;
};

// ---- epilogue pieces shared by the one-CTA and the CTA-pair kernels ----

// Fold one GEMM of a channel into the running residues: this warp's 32 TMEM
// lanes, columns taddr0 .. + 32 NCH - 1 of the accumulator, W = acc 2^e2 (an
// exact integer, |W| <= 2^24), r <- r + lambda (W mod m) (mod m), r kept as
// r + 2048 in 16-bit fields. The accumulator is released (tempty: this CTA's
// barrier, or the leader's for a pair) once its last columns are loaded.
template <int NCH, bool PAIR>
__device__ __forceinline__ void fold_gemm(uint32_t (&acc16)[NCH * 16], uint32_t taddr0, uint32_t tempty, float lam,
                                          float wscale, float mf, float invm) {
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    uint32_t v[32];
    tmem_ld32(taddr0 + ch * 32, v);
    tmem_ld_wait();
    if (ch == NCH - 1) {                  // one arrival per warp, after every lane's loads
      tc_fence_before();
      __syncwarp();
      if ((threadIdx.x & 31) == 0) {
        if (PAIR) mbar_arrive_cluster(tempty);
        else mbar_arrive(tempty);
      }
    }
    // the two entries of a word of acc16 go through each packed fp32
    // operation together (f32x2: each half rounded as the scalar form)
    const float2 kC = make_float2(12582912.0f, 12582912.0f), kCn = make_float2(-12582912.0f, -12582912.0f);
    const float2 ws2 = make_float2(wscale, wscale), inv2 = make_float2(invm, invm), nm2 = make_float2(-mf, -mf);
    const float2 lam2 = make_float2(lam, lam), off2 = make_float2(8390656.0f, 8390656.0f);
    const float2 noff2 = make_float2(-8390656.0f, -8390656.0f);
#pragma unroll
    for (int w = 0; w < 16; ++w) {
      const uint32_t a = acc16[ch * 16 + w];
      // previous residues r from their 16-bit fields r + 2048
      const float2 prev = __fadd2_rn(make_float2(__int_as_float(__byte_perm(a, 0x4B000000u, 0x7410u)),
                                                 __int_as_float(__byte_perm(a, 0x4B000000u, 0x7432u))),
                                     noff2);
      const float2 W = __fmul2_rn(make_float2(__uint_as_float(v[2 * w]), __uint_as_float(v[2 * w + 1])),
                                  ws2);                                         // exact integers, |W| <= 2^24
      const float2 wq = __fadd2_rn(__ffma2_rn(W, inv2, kC), kCn);
      const float2 wm = __ffma2_rn(wq, nm2, W);                                  // W mod m, |wm| < 0.65 m
      const float2 tsum = __ffma2_rn(lam2, wm, prev);                            // exact: < 2^24
      const float2 q2 = __fadd2_rn(__ffma2_rn(tsum, inv2, kC), kCn);
      const float2 o = __fadd2_rn(__ffma2_rn(q2, nm2, tsum), off2);              // |r| < 0.51 m; r + 2048
      acc16[ch * 16 + w] = __byte_perm(__float_as_uint(o.x), __float_as_uint(o.y), 0x5410u);
    }
  }
}

// The unit's HC entries of row `row` from column col0 on, as W mod m or the
// CRT digit (W mod m) (P/m)^-1 mod m, 16 bits each, to channel c's plane of Y;
// acc: added modulo m to the digits already there (blocked call).
template <int HC>
__device__ __forceinline__ void store_unit(const OzFpTables& F, int c, const uint32_t (&acc16)[HC / 2],
                                           uint16_t* Y, int64_t ldy, int m, int n, int row, int col0, int raw,
                                           int acc) {
  if (row >= m || col0 >= n) return;
  const float mf = F.mf[c], invm = F.invm[c];
  const float inv = (float)F.inv[c];
  uint16_t* dst = Y + (size_t)c * m * ldy + (size_t)row * ldy + col0;
  const bool vec = col0 + HC <= n && (ldy & 7) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
#pragma unroll
  for (int i4 = 0; i4 < HC / 8; ++i4) {
    uint32_t o4[4];
    uint32_t prev[4] = {0u, 0u, 0u, 0u};
    if (acc) {                       // the digits of the earlier slabs
      if (vec) {
        const uint4 w = reinterpret_cast<const uint4*>(dst)[i4];
        prev[0] = w.x;
        prev[1] = w.y;
        prev[2] = w.z;
        prev[3] = w.w;
      } else {
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int j = 0; j < 2; ++j)
            if (col0 + 8 * i4 + 2 * ii + j < n) prev[ii] |= (uint32_t)dst[8 * i4 + 2 * ii + j] << (16 * j);
      }
    }
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      uint32_t o = 0;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float r = __int_as_float(0x4B000000u | ((acc16[4 * i4 + ii] >> (16 * j)) & 0xffffu)) - 8390656.0f;
        r = r < 0.f ? r + mf : r;                                            // W mod m in [0, m)
        float y = r;
        if (!raw) {
          const float tt = r * inv;                                          // < m^2 < 2^24: exact
          const float q = fmaf(tt, invm, 12582912.0f) - 12582912.0f;
          y = fmaf(-q, mf, tt);
          y = y < 0.f ? y + mf : y;
        }
        if (acc) {
          y += (float)((prev[ii] >> (16 * j)) & 0xffffu);
          y = y >= mf ? y - mf : y;
        }
        o |= (__float_as_uint(y + 8388608.0f) & 0xffffu) << (16 * j);
      }
      o4[ii] = o;
    }
    if (vec) {
      reinterpret_cast<uint4*>(dst)[i4] = make_uint4(o4[0], o4[1], o4[2], o4[3]);
    } else {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int j = 0; j < 2; ++j)
          if (col0 + 8 * i4 + 2 * ii + j < n) dst[8 * i4 + 2 * ii + j] = (uint16_t)(o4[ii] >> (16 * j));
    }
  }
}

template <bool MX>
__global__ void __launch_bounds__(kThreads, 1)
gemm_fp_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ OzFpTables F, const FpParams p) {
  using C = Cfg<MX>;
  constexpr int BN = C::BN, STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_base = smem_u32(smem_raw);
  const uint32_t base = (raw_base + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw_base);
  const uint32_t bar0 = base + STAGES * STAGE_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
  // barriers (2 STAGES + 5 of them) below 192; then the TMEM address and the abort flag
  static_assert((2 * STAGES + 5) * 8 <= 192, "barriers overlap the TMEM address");
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gbase + STAGES * STAGE_BYTES + 192);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + STAGES * STAGE_BYTES + 200);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), kEpiWarps);        // one arrival per epilogue warp
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  if constexpr (MX) {
    // every byte of columns 448..511 = 0x7F, the UE8M0 scale 2^0, so the block
    // scales leave every product unchanged whatever scale layout the MMA reads
    if (warp >= 2) {
      const uint32_t lane_q = (uint32_t)((warp & 3) * 32) << 16;
      tmem_st32_fill(tmem_base + lane_q + kSfaCol + ((warp - 2) >> 2) * 32, 0x7F7F7F7Fu);
      tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued_parity[STAGES];
      bool outstanding[STAGES];
      for (int i = 0; i < STAGES; ++i) outstanding[i] = false, issued_parity[i] = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < p.num_units && ok; t += gridDim.x) {
        const Unit u = unit_coord(t, p.tiles_m, p.tiles_n);
        const int g0 = F.ch_gemm0[u.c], ng = F.ch_ngemm[u.c];
        for (int g = g0; g < g0 + ng && ok; ++g) {
          const int ya = (int)F.g_pa[g] * p.m_pad + u.tm * BM;
          const int yb = (int)F.g_pb[g] * p.n_pad + u.tn * BN;
          for (int kb = 0; kb < p.kblocks; ++kb) {
            if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, p.status)) { ok = false; break; }
            outstanding[s] = false;
            const uint32_t sa = base + s * STAGE_BYTES;
            mbar_expect_tx(full_bar(s), STAGE_BYTES);
            tma_load_2d(sa, &tmA, full_bar(s), kb * BK, ya);
            tma_load_2d(sa + A_BYTES, &tmB, full_bar(s), kb * BK, yb);
            outstanding[s] = true;
            issued_parity[s] = ph;
            if (++s == STAGES) { s = 0; ph ^= 1u; }
          }
        }
      }
      if (!ok) {
        for (int i = 0; i < STAGES; ++i)
          if (outstanding[i]) mbar_drain(full_bar(i), issued_parity[i]);
      }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t g_ctr = 0;  // accumulations issued (one per GEMM of a unit)
      bool ok = true;
      for (int t = blockIdx.x; t < p.num_units && ok; t += gridDim.x) {
        const Unit u = unit_coord(t, p.tiles_m, p.tiles_n);
        const int ng = F.ch_ngemm[u.c];
        for (int gi = 0; gi < ng && ok; ++gi, ++g_ctr) {
          const uint32_t b = g_ctr & 1u, use = g_ctr >> 1;
          if (!mbar_wait(tempty_bar(b), (use & 1u) ^ 1u, abort_flag, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dtm = tmem_base + b * BN;
          for (int kb = 0; kb < p.kblocks; ++kb) {
            if (!mbar_wait(full_bar(s), ph, abort_flag, p.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = base + s * STAGE_BYTES;
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 32; ++kk) {
              if constexpr (MX)
                umma_mxf4(dtm, sdesc(sa + kk * 32), sdesc(sb + kk * 32), p.idesc, tmem_base + kSfaCol,
                          tmem_base + kSfbCol, (kb > 0 || kk > 0) ? 1u : 0u);
              else
                umma_f8f6f4(dtm, sdesc(sa + kk * 32), sdesc(sb + kk * 32), p.idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit(empty_bar(s));
            if (++s == STAGES) { s = 0; ph ^= 1u; }
          }
          if (!ok) break;
          umma_commit(tfull_bar(b));
        }
      }
      if (!ok) {
        umma_commit(drain_bar);
        mbar_drain(drain_bar, 0);
      }
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    const int e = warp - 2;
    const int quarter = warp & 3;
    const int half = e >> 2;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    const float wscale = __int_as_float((127 + F.e2) << 23);      // 2^e2: accumulator -> W
    uint32_t g_ctr = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < p.num_units && ok; t += gridDim.x) {
      const Unit u = unit_coord(t, p.tiles_m, p.tiles_n);
      const int g0 = F.ch_gemm0[u.c], ng = F.ch_ngemm[u.c];
      const float mf = F.mf[u.c], invm = F.invm[u.c];
      uint32_t acc16[C::HC / 2];             // running residue + 2048, 16 bits per column
#pragma unroll
      for (int i = 0; i < C::HC / 2; ++i) acc16[i] = 0x08000800u;
      for (int gi = 0; gi < ng; ++gi, ++g_ctr) {
        const uint32_t b = g_ctr & 1u, use = g_ctr >> 1;
        if (!mbar_wait(tfull_bar(b), use & 1u, abort_flag, p.status)) { ok = false; break; }
        tc_fence_after();
        fold_gemm<C::NCH, false>(acc16, tmem_base + lane_addr + b * BN + half * C::HC, tempty_bar(b),
                                 F.g_lam[g0 + gi], wscale, mf, invm);
      }
      if (!ok) break;
      // ---- unit done: W mod m or the CRT digit, 16 bits per entry ----
      store_unit<C::HC>(F, u.c, acc16, p.Y, p.ldy, p.m, p.n, u.tm * BM + quarter * 32 + lane,
                        u.tn * BN + half * C::HC, p.raw, p.acc);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// The same GEMMs on CTA pairs (cluster of 2, cta_group::2): a pair computes a
// 256 x BN tile (BN = 256 for kind::f8f6f4; 192 for the block-scaled 4-bit
// kind, whose two accumulators leave TMEM room for the scales); each CTA
// stages its 128 rows of A and BN / 2 rows of B, so that per product a CTA
// reads a quarter (f8f6f4) or an eighth (4-bit) less shared memory than one
// CTA on a 128 x BN tile, and the leader issues M = 256 products that write
// 128 rows into each CTA's tensor memory. Barriers as in the INT8 pair kernel:
//   full[s]   leader only: both CTAs' copies of stage s;
//   empty[s]  each CTA: its stage s may be refilled (multicast commit);
//   tfull[b]  each CTA: accumulator b holds a GEMM (multicast commit);
//   tempty[b] leader only: both CTAs' epilogues have loaded accumulator b.
// Every wait is bounded, as in the one-CTA kernel.
// ---------------------------------------------------------------------------
template <bool MX>
struct PairCfg {
  static constexpr int BN = MX ? 192 : 256;         // N of a pair's products
  static constexpr int BNC = BN / 2;                // rows of B per CTA
  static constexpr int HC = BN / 2;                 // columns per epilogue warp (two halves)
  static constexpr int NCH = HC / 32;
  static constexpr int STAGE_BYTES = A_BYTES + BNC * BK;
  static constexpr int STAGES = MX ? 7 : 6;
  static constexpr int kSmemBytes = STAGES * STAGE_BYTES + 256 + 1024;
};

__device__ __forceinline__ void umma_f8f6f4_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                 uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_mxf4_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
      : "memory");
}

template <bool MX>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
gemm_fp_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ OzFpTables F, const FpParams p) {
  using C = PairCfg<MX>;
  constexpr int BN = C::BN, BNC = C::BNC, STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_base = smem_u32(smem_raw);
  const uint32_t base = (raw_base + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw_base);
  const uint32_t bar0 = base + STAGES * STAGE_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
  static_assert((2 * STAGES + 5) * 8 <= 192, "barriers overlap the TMEM address");
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gbase + STAGES * STAGE_BYTES + 192);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + STAGES * STAGE_BYTES + 200);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 2 * kEpiWarps);    // one arrival per epilogue warp of the pair
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 1) {                          // one warp of each CTA: the pair's allocation
    tmem_alloc_pair(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  if constexpr (MX) {
    // every byte of columns 448..511 of both CTAs = 0x7F, the UE8M0 scale 2^0:
    // the products are unscaled whichever scale layout the pair's MMA reads
    if (warp >= 2) {
      const uint32_t lane_q = (uint32_t)((warp & 3) * 32) << 16;
      tmem_st32_fill(tmem_base + lane_q + kSfaCol + ((warp - 2) >> 2) * 32, 0x7F7F7F7Fu);
      tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  cluster_sync();                           // both CTAs' barriers and scales exist before any remote use
  tc_fence_after();

  if (warp == 0) {
    // ------------------------------ TMA producer (both CTAs) ------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued_parity[STAGES];
      bool outstanding[STAGES];
      for (int i = 0; i < STAGES; ++i) outstanding[i] = false, issued_parity[i] = 0;
      bool ok = true;
      for (int t = pair; t < p.num_units && ok; t += npairs) {
        const Unit u = unit_coord(t, p.tiles_m, p.tiles_n);
        const int g0 = F.ch_gemm0[u.c], ng = F.ch_ngemm[u.c];
        for (int g = g0; g < g0 + ng && ok; ++g) {
          const int ya = (int)F.g_pa[g] * p.m_pad + u.tm * 2 * BM + (int)rank * BM;
          const int yb = (int)F.g_pb[g] * p.n_pad + u.tn * BN + (int)rank * BNC;
          for (int kb = 0; kb < p.kblocks; ++kb) {
            if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, p.status)) { ok = false; break; }
            outstanding[s] = false;
            const uint32_t sa = base + s * STAGE_BYTES;
            if (leader) mbar_expect_tx(full_bar(s), 2 * STAGE_BYTES);
            const uint32_t fb = mapa(full_bar(s), 0);
            tma_load_2d_pair(sa, &tmA, fb, kb * BK, ya);
            tma_load_2d_pair(sa + A_BYTES, &tmB, fb, kb * BK, yb);
            outstanding[s] = true;
            issued_parity[s] = ph;
            if (++s == STAGES) { s = 0; ph ^= 1u; }
          }
        }
      }
      // both CTAs' copies complete on the leader's barriers: the leader waits
      // (bounded) for every stage it expected before the pair may exit
      if (!ok && leader) {
        for (int i = 0; i < STAGES; ++i)
          if (outstanding[i]) mbar_drain(full_bar(i), issued_parity[i]);
      }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer (leader) ------------------------------
    if (lane == 0 && leader) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t g_ctr = 0;
      bool ok = true;
      for (int t = pair; t < p.num_units && ok; t += npairs) {
        const Unit u = unit_coord(t, p.tiles_m, p.tiles_n);
        const int ng = F.ch_ngemm[u.c];
        for (int gi = 0; gi < ng && ok; ++gi, ++g_ctr) {
          const uint32_t b = g_ctr & 1u, use = g_ctr >> 1;
          if (!mbar_wait(tempty_bar(b), (use & 1u) ^ 1u, abort_flag, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dtm = tmem_base + b * BN;
          for (int kb = 0; kb < p.kblocks; ++kb) {
            if (!mbar_wait(full_bar(s), ph, abort_flag, p.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = base + s * STAGE_BYTES;
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 32; ++kk) {
              if constexpr (MX)
                umma_mxf4_pair(dtm, sdesc(sa + kk * 32), sdesc(sb + kk * 32), p.idesc, tmem_base + kSfaCol,
                               tmem_base + kSfbCol, (kb > 0 || kk > 0) ? 1u : 0u);
              else
                umma_f8f6f4_pair(dtm, sdesc(sa + kk * 32), sdesc(sb + kk * 32), p.idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit_pair_both(empty_bar(s));
            if (++s == STAGES) { s = 0; ph ^= 1u; }
          }
          if (!ok) break;
          umma_commit_pair_both(tfull_bar(b));
        }
      }
      if (!ok) {
        umma_commit_pair_self(drain_bar);
        mbar_drain(drain_bar, 0);
      }
    }
  } else {
    // ------------------------------ epilogue (both CTAs) ------------------------------
    const int e = warp - 2;
    const int quarter = warp & 3;
    const int half = e >> 2;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    const float wscale = __int_as_float((127 + F.e2) << 23);      // 2^e2: accumulator -> W
    uint32_t g_ctr = 0;
    bool ok = true;
    for (int t = pair; t < p.num_units && ok; t += npairs) {
      const Unit u = unit_coord(t, p.tiles_m, p.tiles_n);
      const int g0 = F.ch_gemm0[u.c], ng = F.ch_ngemm[u.c];
      const float mf = F.mf[u.c], invm = F.invm[u.c];
      uint32_t acc16[C::HC / 2];             // running residue + 2048, 16 bits per column
#pragma unroll
      for (int i = 0; i < C::HC / 2; ++i) acc16[i] = 0x08000800u;
      for (int gi = 0; gi < ng; ++gi, ++g_ctr) {
        const uint32_t b = g_ctr & 1u, use = g_ctr >> 1;
        if (!mbar_wait(tfull_bar(b), use & 1u, abort_flag, p.status)) { ok = false; break; }
        tc_fence_after();
        fold_gemm<C::NCH, true>(acc16, tmem_base + lane_addr + b * BN + half * C::HC, mapa(tempty_bar(b), 0),
                                F.g_lam[g0 + gi], wscale, mf, invm);
      }
      if (!ok) break;
      store_unit<C::HC>(F, u.c, acc16, p.Y, p.ldy, p.m, p.n, u.tm * 2 * BM + (int)rank * BM + quarter * 32 + lane,
                        u.tn * BN + half * C::HC, p.raw, p.acc);
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();                           // neither CTA leaves while the pair may touch its memory
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, kTmemCols);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}

bool make_map8(CUtensorMap* map, const void* planes, int64_t rows, int64_t k_pad, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)k_pad};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(planes), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// kind::f8f6f4 operand type codes of the instruction descriptor
uint32_t f8f6f4_code(int fmt) {
  switch (fmt) {
    case OZ_FMT_E4M3: return 0;
    case OZ_FMT_E5M2: return 1;
    case OZ_FMT_E2M3: return 3;
    case OZ_FMT_E3M2: return 4;
    case OZ_FMT_E2M1: return 5;
    default: return 0xffffffffu;
  }
}

// =========================================================================
// Reconstruct on 16-bit digits
// =========================================================================

typedef unsigned __int128 u128;

__device__ __forceinline__ uint64_t round128b(u128 mag, uint32_t neg, int e) {
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
    q = lo << (-sh);
  } else if (sh > nb) {
    q = 0;
  } else if (sh == nb) {
    q = (mag & ~((u128)1 << (nb - 1))) != 0 ? 1 : 0;
  } else {
    q = (uint64_t)(mag >> sh);
    const bool half = (mag >> (sh - 1)) & 1;
    const bool sticky = (mag & (((u128)1 << (sh - 1)) - 1)) != 0;
    if (half && (sticky || (q & 1ull))) q += 1ull;
  }
  uint64_t b = E >= -1022 ? ((uint64_t)(E + 1022) << 52) + q : q;
  if (b >= 0x7ff0000000000000ull) b = 0x7ff0000000000000ull;
  return sign | b;
}

// P < 2^125; digits y_c < m_c < 2^12; pairs z = y_a m_b + y_b m_a < 2^25.
template <int NP>
__global__ void __launch_bounds__(256) reconstruct16_kernel(const __grid_constant__ OzTables T, int64_t m, int64_t n,
                                                            const uint16_t* __restrict__ Y, int64_t ldy,
                                                            const int32_t* __restrict__ s,
                                                            const int32_t* __restrict__ t,
                                                            double* __restrict__ C, int64_t ldc) {
  constexpr int EPT = 4;
  const int64_t i = blockIdx.x;
  const int64_t j0 = ((int64_t)blockIdx.y * 256 + threadIdx.x) * EPT;
  if (i >= m || j0 >= n) return;
  const int Q = T.Q;
  const int64_t plane = m * ldy;
  const uint16_t* yp = Y + i * ldy + j0;
  const bool vec = (j0 + 4 <= n) && ((reinterpret_cast<uintptr_t>(yp) & 7) == 0) && ((plane & 3) == 0);
  uint64_t wa[NP], wb[NP];
#pragma unroll
  for (int pi = 0; pi < NP; ++pi) {
    if (vec) {
      wa[pi] = __ldg(reinterpret_cast<const unsigned long long*>(yp + (2 * pi) * plane));
      wb[pi] = (2 * pi + 1 < Q) ? __ldg(reinterpret_cast<const unsigned long long*>(yp + (2 * pi + 1) * plane)) : 0ull;
    } else {
      uint64_t a = 0, b = 0;
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (j0 + e < n) {
          a |= (uint64_t)__ldg(yp + (2 * pi) * plane + e) << (16 * e);
          if (2 * pi + 1 < Q) b |= (uint64_t)__ldg(yp + (2 * pi + 1) * plane + e) << (16 * e);
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
      const uint32_t ya = (uint32_t)(wa[pi] >> (16 * e)) & 0xffffu, yb = (uint32_t)(wb[pi] >> (16 * e)) & 0xffffu;
      const uint32_t z = ya * mb + yb * ma;
      f[e] = fmaf(__uint2float_rn(z), pinv, f[e]);
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
    const uint64_t c0 = acc[e][0];
    const uint64_t c1 = acc[e][1] + (c0 >> 32);
    const uint64_t c2 = acc[e][2] + (c1 >> 32);
    const uint64_t c3 = acc[e][3] + (c2 >> 32);
    const uint64_t lo = (c0 & 0xffffffffull) | (c1 << 32);
    const uint64_t hi = (c2 & 0xffffffffull) | (c3 << 32);
    const float qf = rintf(f[e]);
    __int128 X = (__int128)((((u128)hi) << 64 | lo) - (u128)(uint32_t)qf * P);
    if (fabsf(f[e] - qf) > 0.499f) {
      if (2 * X >= (__int128)P) X -= (__int128)P;
      else if (2 * X < -(__int128)P) X += (__int128)P;
    }
    const uint32_t neg = X < 0;
    const u128 mag = neg ? (u128)(-X) : (u128)X;
    const int64_t j = j0 + e;
    const int ex = j < n ? -(si + t[j]) : 0;
    out[e] = __longlong_as_double((long long)round128b(mag, neg, ex));
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

template <int NP>
cudaError_t launch16(const OzTables& T, int64_t m, int64_t n, const uint16_t* Y, int64_t ldy, const int32_t* s,
                     const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  dim3 grid((unsigned)m, (unsigned)((n + 1023) / 1024));
  reconstruct16_kernel<NP><<<grid, 256, 0, st>>>(T, m, n, Y, ldy, s, t, C, ldc);
  return cudaGetLastError();
}

template <int CB, bool WIDE>
cudaError_t split_fp_w(const OzTables& t, const OzFpTables& f, int contiguous, int64_t nvec, int64_t len,
                       const double* X, int64_t ld, int64_t nvec_pad, int64_t k_pad, int32_t* shifts,
                       uint8_t* planes, int32_t* flag, uint64_t* colmax, cudaStream_t st, bool given) {
  if (contiguous) {
    split_fp_rows_kernel<CB, WIDE><<<(unsigned)nvec_pad, 256, 0, st>>>(f, t.bits, nvec, len, X, ld, nvec_pad,
                                                                       k_pad, shifts, planes, flag, given);
    return cudaGetLastError();
  }
  if (!given) {
    cudaError_t e = launch_shifts_cols(t.bits, nvec, len, X, ld, shifts, flag, colmax, st);
    if (e != cudaSuccess) return e;
  }
  dim3 g((unsigned)(nvec_pad / 64), (unsigned)(k_pad / 32));
  split_fp_cols_kernel<CB, WIDE><<<g, 256, 0, st>>>(f, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes);
  return cudaGetLastError();
}

// beta > 64: |a'| in 128 bits and a fifth 16-bit piece
template <int CB>
cudaError_t split_fp(const OzTables& t, const OzFpTables& f, int contiguous, int64_t nvec, int64_t len,
                     const double* X, int64_t ld, int64_t nvec_pad, int64_t k_pad, int32_t* shifts, uint8_t* planes,
                     int32_t* flag, uint64_t* colmax, cudaStream_t st, bool given) {
  if (t.bits > 64)
    return split_fp_w<CB, true>(t, f, contiguous, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, colmax,
                                st, given);
  return split_fp_w<CB, false>(t, f, contiguous, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, colmax,
                               st, given);
}

}  // namespace

cudaError_t launch_split_fp(const OzTables& t, const OzFpTables& f, int contiguous, int64_t nvec, int64_t len,
                            const double* X, int64_t ld, int64_t nvec_pad, int64_t k_pad, int32_t* shifts,
                            uint8_t* planes, int32_t* flag, uint64_t* colmax, cudaStream_t st, bool given) {
  if (nvec_pad == 0) return cudaSuccess;
  switch (f.code_bits) {
    case 8:
      return split_fp<8>(t, f, contiguous, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, colmax, st, given);
    case 6:
      return split_fp<6>(t, f, contiguous, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, colmax, st, given);
    case 4:
      return split_fp<4>(t, f, contiguous, nvec, len, X, ld, nvec_pad, k_pad, shifts, planes, flag, colmax, st, given);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

// Float-format GEMMs run one CTA per tile (gemm_fp_kernel). The CTA-pair
// form (gemm_fp_pair_kernel) gives the same bits but was slower at 8192 on
// one box: E4M3 GEMMs 10.07 against 9.75 ms, E2M1 12.29 against 11.35 ms.
constexpr bool kFpPairs = false;

template <bool MX>
cudaError_t gemm_fp(const OzFpTables& f, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                    const uint8_t* U, const uint8_t* V, uint16_t* Y, int64_t ldy, int raw, int32_t* status,
                    cudaStream_t st) {
  using C = Cfg<MX>;
  using PC = PairCfg<MX>;
  const bool pairs = kFpPairs && m_pad % (2 * BM) == 0;
  const int tile_m = pairs ? 2 * BM : BM, tile_n = pairs ? PC::BN : C::BN;
  const int64_t tiles_m = (m + tile_m - 1) / tile_m, tiles_n = (n + tile_n - 1) / tile_n;
  const int64_t units = tiles_m * tiles_n * f.nch;
  if (units > INT32_MAX || (int64_t)f.nplanes * m_pad > INT32_MAX || (int64_t)f.nplanes * n_pad > INT32_MAX)
    return cudaErrorInvalidValue;
  const int64_t row_bytes = fp_row_bytes(f, k_pad);
  CUtensorMap mapA, mapB;
  // B tiles of the last plane may run past its rows: the map's bound fills zeros;
  // elsewhere they read the next plane's rows into columns the epilogue drops
  if (!make_map8(&mapA, U, (int64_t)f.nplanes * m_pad, row_bytes, BM)) return cudaErrorInvalidValue;
  if (!make_map8(&mapB, V, (int64_t)f.nplanes * n_pad, row_bytes, pairs ? PC::BNC : C::BN))
    return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  FpParams p;
  p.m = (int)m;
  p.n = (int)n;
  p.tiles_m = (int)tiles_m;
  p.tiles_n = (int)tiles_n;
  p.num_units = (int)units;
  p.kblocks = (int)(k_pad / C::KSTAGE);
  p.m_pad = (int)m_pad;
  p.n_pad = (int)n_pad;
  p.raw = raw & kEpiRaw;
  p.acc = (raw & kEpiAccumulate) != 0;
  const uint32_t mbits = (uint32_t)(tile_m >> 4) << 24, nbits = (uint32_t)(tile_n >> 3) << 17;
  if (MX) {
    // block-scaled: scale factor ids 0, A = B = E2M1 (1), both K-major, N >> 3,
    // UE8M0 scales (bit 23), M >> 4, K = 64 per instruction
    p.idesc = (1u << 7) | (1u << 10) | nbits | (1u << 23) | mbits;
  } else {
    // D = F32, A and B of the format, both K-major, N >> 3, M >> 4
    const uint32_t code = f8f6f4_code(f.fmt);
    if (code == 0xffffffffu) return cudaErrorInvalidValue;
    p.idesc = (1u << 4) | (code << 7) | (code << 10) | nbits | mbits;
  }
  p.Y = Y;
  p.ldy = ldy;
  p.status = status;
  if (pairs) {
    // as the INT8 pair kernel: each CTA of a pair claims all the shared memory a block may have
    int smem_optin = 0;
    e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int smem_bytes = smem_optin > PC::kSmemBytes ? smem_optin : PC::kSmemBytes;
    e = cudaFuncSetAttribute(gemm_fp_pair_kernel<MX>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    const int64_t npairs = units < sms / 2 ? units : sms / 2;
    gemm_fp_pair_kernel<MX><<<(unsigned)(2 * npairs), kThreads, smem_bytes, st>>>(mapA, mapB, f, p);
    return cudaGetLastError();
  }
  e = cudaFuncSetAttribute(gemm_fp_kernel<MX>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  if (e != cudaSuccess) return e;
  const int grid = (int)(units < sms ? units : sms);
  gemm_fp_kernel<MX><<<grid, kThreads, C::kSmemBytes, st>>>(mapA, mapB, f, p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_fp(const OzFpTables& f, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                           const uint8_t* U, const uint8_t* V, uint16_t* Y, int64_t ldy, int raw,
                           int32_t* status, cudaStream_t st) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (ldy < n) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(U) & 127) || (reinterpret_cast<uintptr_t>(V) & 127) || k_pad % fp_k_align(f) ||
      m_pad % BM || n_pad % kPadRows)
    return cudaErrorInvalidValue;
  if (f.code_bits == 4) return gemm_fp<true>(f, m, n, m_pad, n_pad, k_pad, U, V, Y, ldy, raw, status, st);
  return gemm_fp<false>(f, m, n, m_pad, n_pad, k_pad, U, V, Y, ldy, raw, status, st);
}

cudaError_t launch_reconstruct16(const OzTables& T, int64_t m, int64_t n, const uint16_t* Y, int64_t ldy,
                                 const int32_t* s, const int32_t* t, double* C, int64_t ldc, cudaStream_t st) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (ldy < n) return cudaErrorInvalidValue;
  if (T.limbs > 4) return launch_reconstruct16_wide(T, m, n, Y, ldy, s, t, C, ldc, st);   // widened budgets
  switch (T.npairs) {
    case 5: return launch16<5>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 6: return launch16<6>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 7: return launch16<7>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 8: return launch16<8>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 9: return launch16<9>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 10: return launch16<10>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 11: return launch16<11>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 12: return launch16<12>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 13: return launch16<13>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 14: return launch16<14>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 15: return launch16<15>(T, m, n, Y, ldy, s, t, C, ldc, st);
    case 16: return launch16<16>(T, m, n, Y, ldy, s, t, C, ldc, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace oz
