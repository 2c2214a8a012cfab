// oz_gemm_tc.cu -- phases 3 (GEMMs) and 4 (Epilogue) of Sec. "Structure" on
// the 5th-generation tensor cores: W_q = U_q V_q^T with the residues held
// exactly in BF16 (integers of magnitude <= 119 need 7 significand bits), one
// tcgen05.mma.kind::f16 stream into FP32 accumulators in tensor memory.
//
// Exactness (Sec. "Exactness Constraints and K_max", eq. ov-accgen with the
// FP32 bound Lambda = 2^24): one FP32 accumulator may sum K_t products of
// magnitude <= 119^2 only while K_t 119^2 <= 2^24, i.e. K_t <= 1184. The inner
// dimension is therefore cut into slabs of 1024 terms (Sec. "Slabs"); each
// slab's accumulator is drained and reduced modulo m into a running residue
// (order R>C, eq. ov-comrtc: the running residue and the slab sum stay below
// 2^24). Whether the tensor core adds such integers without rounding is the
// undocumented behaviour of Sec. "Exactness May Rely on Undocumented
// Accumulation"; the parity tests drive every accumulator to 1024 * 119^2 and
// compare bit for bit with exact integer products.
//
// Two kernels: gemm_tc_pair_kernel (the default; CTA pairs, cta_group::2,
// 256 x 256 tiles, described before it) and gemm_tc_kernel (one CTA per
// 128 x 256 tile). Both are persistent, one CTA per SM, 2 + E warps:
//   warp 0      TMA producer: bf16 tiles, 128-byte swizzle, a ring of
//               mbarrier-tracked shared-memory stages;
//   warp 1      allocates all 512 TMEM columns (two 256-column FP32
//               accumulators) and, from one thread, issues tcgen05.mma
//               (K = 16) and tcgen05.commit;
//   warps 2..   E epilogue warps (16 in the one-CTA kernels; 4 or 16 in the
//               pair kernel, see kPairEpiWarps): drain an accumulator with
//               tcgen05.ld while the MMAs fill the other; each slab's sums
//               are reduced modulo m and written back into the accumulator,
//               on which the slab after next accumulates; the last two slabs
//               of a tile give the CRT digit (or W mod m) of each entry, one
//               byte, stored in 16-byte runs. Their arithmetic runs on packed
//               f32x2 pairs.
// Every wait is bounded (about 2 s of %globaltimer); a wait that runs out sets
// bit 1 of the status word, makes every role stop issuing work, waits (again
// bounded) for the copies and products already in flight, frees the tensor
// memory and returns.
#include <cuda.h>
#include <stdint.h>

#include "oz_internal.h"
#include "oz_sync.cuh"
#include "oz_pair.cuh"
#include "oz_device.cuh"

namespace oz {
namespace {

constexpr int BM = 128, BN = 256, BK = 64;        // BK in bf16 entries = 128 bytes
constexpr int STAGES = 4;
constexpr int kSlabBlocks = 16;                    // k-blocks per FP32 slab: 1024 terms
constexpr int kBand = 8;                           // n-tiles per band of the tile order
constexpr int A_BYTES = BM * BK * 2;               // 16 KiB
constexpr int B_BYTES = BN * BK * 2;               // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;     // 48 KiB
constexpr int kEpiWarps = 16;                      // epilogue warps of the one-CTA kernels
constexpr int CPW1 = 1024 / kEpiWarps;             // columns of a 256-column tile per epilogue warp
constexpr int kThreads = (2 + kEpiWarps) * 32;
constexpr int kTmemCols = 512;
constexpr int kBarBytes = 256;                     // barriers, then the TMEM address and the abort flag
constexpr int kHolderOff = 192;                    // offsets in that area (past every barrier)
constexpr int kAbortOff = 200;
constexpr int kSmemBytes = STAGES * STAGE_BYTES + kBarBytes + 1024;

// Instruction descriptor of tcgen05.mma.kind::f16: D = F32 (bits 4-5 = 1),
// A = B = BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

// ---- tcgen05 ----
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

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// M = 256 across the pair (128 rows of A in each CTA), N = 256 (128 rows of B in each)
constexpr uint32_t kIdescPair = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                                ((uint32_t)(256 >> 4) << 24);
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescPair), "r"(accumulate)
      : "memory");
}

// 32 lanes x 32 columns of 32-bit words: thread i gets row (lane base + i),
// columns taddr.col .. +31.
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
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: start address,
// leading offset 16 B (unused for this layout), stride 1024 B between groups of
// eight 128-byte rows, descriptor version 1 (bit 46), swizzle mode 2 (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct Coord {
  int q, tm, tn;
};

// Tile order: modulus by modulus; within a modulus, bands of kBand n-tiles;
// within a band, row-major over (tm, tn), so a wave of CTAs shares the B strip
// of its band and each A panel across kBand neighbours (Sec. "Tile order").
__device__ __forceinline__ Coord tile_coord(int t, int tiles_m, int tiles_n) {
  const int per_q = tiles_m * tiles_n;
  Coord c;
  c.q = t / per_q;
  const int r = t - c.q * per_q;
  const int band = r / (tiles_m * kBand);
  const int rb = r - band * tiles_m * kBand;
  const int bw = min(kBand, tiles_n - band * kBand);
  c.tm = rb / bw;
  c.tn = band * kBand + (rb - c.tm * bw);
  return c;
}

// The epilogue's arithmetic, two accumulator values per packed fp32
// operation (the f32x2 fma, add and mul of sm_100 and later round each half
// as the scalar operation would, so the results are those of the scalar form
// at half the issued instructions). Per unit: the modulus m, fl(1/m), the
// factor f of the digit ((P/m)^-1 mod m, or 1 for raw W mod m) and
// bias = -1/2 + 1/(2m), each in both halves.
struct EpiConst {
  float2 invm, nm, f, bias;
};

__device__ __forceinline__ EpiConst epi_const(float mf, float invm, float f) {
  const float b = fmaf(0.5f, invm, -0.5f);
  return EpiConst{make_float2(invm, invm), make_float2(-mf, -mf), make_float2(f, f), make_float2(b, b)};
}

constexpr float kRint = 12582912.0f;      // 1.5 * 2^23: t + kRint - kRint = rint(t) for |t| < 2^22
constexpr float kTwo23 = 8388608.0f;      // 2^23 + y, 0 <= y < 256: y in the low byte
constexpr float kTwo23p128 = 8388736.0f;  // 2^23 + 128

// r = t - m rint(t / m) for two accumulator values (|t| < 2^24): exact,
// |r| <= 120.
__device__ __forceinline__ float2 residue2(float2 t, const EpiConst& k) {
  const float2 qf = __fadd2_rn(__ffma2_rn(t, k.invm, make_float2(kRint, kRint)), make_float2(-kRint, -kRint));
  return __ffma2_rn(qf, k.nm, t);
}

// The byte of two residues r: y = r f mod m in [0, m), as 2^23 + y. r f is
// an exact integer (|r f| <= 120 * 238 < 2^15), and floor(r f / m) =
// rint(r f / m - 1/2 + 1/(2m)): the fraction of r f / m is a multiple of
// 1/m, so the argument lies at least 1/(2m) from a half-integer, far beyond
// the rounding of fl(1/m), of the bias and of the fma (together below 2^-14).
// Equal to the balanced CRT digit moved into [0, m).
__device__ __forceinline__ float2 digit2(float2 r, const EpiConst& k) {
  const float2 y = __fmul2_rn(r, k.f);
  const float2 q = __fadd2_rn(__fadd2_rn(__ffma2_rn(y, k.invm, k.bias), make_float2(kRint, kRint)),
                              make_float2(-kRint, -kRint));
  return __fadd2_rn(__ffma2_rn(q, k.nm, y), make_float2(kTwo23, kTwo23));
}

// A write-back slab: the 32 values of v reduced modulo m in place.
__device__ __forceinline__ void residues32(uint32_t (&v)[32], const EpiConst& k) {
#pragma unroll
  for (int j = 0; j < 32; j += 2) {
    const float2 r = residue2(make_float2(__uint_as_float(v[j]), __uint_as_float(v[j + 1])), k);
    v[j] = __float_as_uint(r.x);
    v[j + 1] = __float_as_uint(r.y);
  }
}

// Four values v[0..3] of a slab that is not written back, as four bytes:
// the last slab's digits (after adding, when chain, the residue of the other
// chain of slabs held as r + 128 in the bytes of a8), else r + 128.
__device__ __forceinline__ uint32_t bytes4(const uint32_t* v, uint32_t a8, bool last, bool chain, const EpiConst& k) {
  float2 t0 = make_float2(__uint_as_float(v[0]), __uint_as_float(v[1]));
  float2 t1 = make_float2(__uint_as_float(v[2]), __uint_as_float(v[3]));
  if (last && chain) {
    const float2 nb = make_float2(-kTwo23p128, -kTwo23p128);
    const float2 p0 = make_float2(__int_as_float(__byte_perm(a8, 0x4B000000u, 0x7540u)),
                                  __int_as_float(__byte_perm(a8, 0x4B000000u, 0x7541u)));
    const float2 p1 = make_float2(__int_as_float(__byte_perm(a8, 0x4B000000u, 0x7542u)),
                                  __int_as_float(__byte_perm(a8, 0x4B000000u, 0x7543u)));
    t0 = __fadd2_rn(t0, __fadd2_rn(p0, nb));
    t1 = __fadd2_rn(t1, __fadd2_rn(p1, nb));
  }
  const float2 r0 = residue2(t0, k), r1 = residue2(t1, k);
  float2 o0, o1;
  if (last) {
    o0 = digit2(r0, k);
    o1 = digit2(r1, k);
  } else {
    o0 = __fadd2_rn(r0, make_float2(kTwo23p128, kTwo23p128));
    o1 = __fadd2_rn(r1, make_float2(kTwo23p128, kTwo23p128));
  }
  return __byte_perm(__byte_perm(__float_as_uint(o0.x), __float_as_uint(o0.y), 0x0040u),
                     __byte_perm(__float_as_uint(o1.x), __float_as_uint(o1.y), 0x0040u), 0x5410u);
}

// One thread's 128 digits of a tile row (one byte each, packed in words) to
// Y: whole 16-byte runs up to `left` (the columns of the row from here to n)
// rounded up to 16 when the row pitch is a multiple of 16 (bytes past n are
// never read), byte stores otherwise. acc: add into the digits in Y modulo m.
template <int NW>
__device__ __forceinline__ void store_digits(uint8_t* dst, const uint32_t* w, int left, bool runs, int acc,
                                             uint32_t m) {
  static_assert(NW == 32 || NW == 16, "128 or 64 digits");
  if (runs) {
    const int chunks = min(NW / 4, (left + 15) >> 4);
    const uint32_t mm = m * 0x01010101u;
#pragma unroll
    for (int i = 0; i < NW / 4; ++i) {
      if (i < chunks) {
        uint4 o = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
        if (acc) {
          const uint4 old = reinterpret_cast<const uint4*>(dst)[i];
          o.x = addmod_bytes(o.x, old.x, mm);
          o.y = addmod_bytes(o.y, old.y, mm);
          o.z = addmod_bytes(o.z, old.z, mm);
          o.w = addmod_bytes(o.w, old.w, mm);
        }
        reinterpret_cast<uint4*>(dst)[i] = o;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < NW; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * i + j < left) {
          uint32_t y = (w[i] >> (8 * j)) & 0xffu;
          if (acc) {
            y += dst[4 * i + j];
            y = y >= m ? y - m : y;
          }
          dst[4 * i + j] = (uint8_t)y;
        }
  }
}

// The drain of a unit that is one slab (a kernel launched for K of at most
// 1024 terms, unsplit): every chunk of this warp's columns is loaded first and
// the accumulator released at once (one arrival per warp: each thread's
// release-ordered arrival cost a memory barrier per unit), so that the
// products of the unit after next start while this warp forms the digits
// (W mod m reduced exactly, then the CRT digit, or W mod m when raw), one byte
// per entry in acc8.
template <int NCH, typename R>
__device__ __forceinline__ void drain_one_slab(uint32_t taddr0, uint32_t (&acc8)[NCH * 8], const EpiConst& k,
                                               R release) {
  uint32_t v[NCH][32];
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) tmem_ld32(taddr0 + ch * 32, v[ch]);
  tmem_ld_wait();
  tc_fence_before();
  release();
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
    for (int w = 0; w < 8; ++w) acc8[ch * 8 + w] = bytes4(v[ch] + 4 * w, 0u, true, false, k);
}

struct Params {
  int m, n, tiles_m, tiles_n, num_tiles, kblocks, m_pad, n_pad, raw;
  int acc;           // add into the digits already in Y, modulo m (blocked call)
  uint8_t* Y;
  int64_t ldy;       // row pitch of Y
  int32_t* status;
  // split-K: the inner dimension in nsplit ranges of kbps k-blocks (whole
  // slabs); unit u is split u / num_tiles of tile u % num_tiles, and split j
  // writes its digits to Y + j ysplit
  int nsplit, kbps;
  int64_t ysplit;
};

// The tile, split and k-block range [kb0, kb1) of unit u.
struct Unit {
  Coord c;
  int ks, kb0, kb1, nslabs;
};
__device__ __forceinline__ Unit unit_of(const Params& p, int u) {
  Unit w;
  w.ks = u / p.num_tiles;
  w.c = tile_coord(u - w.ks * p.num_tiles, p.tiles_m, p.tiles_n);
  w.kb0 = w.ks * p.kbps;
  w.kb1 = min(p.kblocks, w.kb0 + p.kbps);
  w.nslabs = (w.kb1 - w.kb0 + kSlabBlocks - 1) / kSlabBlocks;
  return w;
}

// ONE: every unit is one slab (K <= 1024, unsplit); see drain_one_slab.
template <bool ONE>
__global__ void __launch_bounds__(kThreads, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ OzTables T, const Params p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_base = smem_u32(smem_raw);
  const uint32_t base = (raw_base + 1023u) & ~1023u;                  // 1024-aligned stages
  uint8_t* gbase = smem_raw + (base - raw_base);
  const uint32_t bar0 = base + STAGES * STAGE_BYTES;
  // barriers: full[STAGES], empty[STAGES], tfull[2], tempty[2]
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gbase + STAGES * STAGE_BYTES + kHolderOff);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + STAGES * STAGE_BYTES + kAbortOff);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), ONE ? kEpiWarps : kEpiWarps * 32);   // one-slab: one arrival per warp
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

  const int num_units = p.num_tiles * p.nsplit;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued_parity[STAGES];
      bool outstanding[STAGES];
      for (int i = 0; i < STAGES; ++i) outstanding[i] = false, issued_parity[i] = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < num_units && ok; t += gridDim.x) {
        const Unit u = unit_of(p, t);
        const int ya = u.c.q * p.m_pad + u.c.tm * BM;
        const int yb = u.c.q * p.n_pad + u.c.tn * BN;
        for (int kb = u.kb0; kb < u.kb1; ++kb) {
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
      if (!ok) {  // wait for our own copies in flight before the CTA exits
        for (int i = 0; i < STAGES; ++i)
          if (outstanding[i]) mbar_drain(full_bar(i), issued_parity[i]);
      }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t g = 0;  // slab counter across tiles
      bool ok = true;
      for (int t = blockIdx.x; t < num_units && ok; t += gridDim.x) {
        const Unit u = unit_of(p, t);
        for (int sl = 0; sl < u.nslabs && ok; ++sl, ++g) {
          const uint32_t b = g & 1u, use = g >> 1;
          if (!mbar_wait(tempty_bar(b), (use & 1u) ^ 1u, abort_flag, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dtm = tmem_base + b * BN;
          const int kb0 = u.kb0 + sl * kSlabBlocks;
          const int kb1 = min(u.kb1, kb0 + kSlabBlocks);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(full_bar(s), ph, abort_flag, p.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = base + s * STAGE_BYTES;
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              umma_bf16(dtm, sdesc(sa + kk * 32), sdesc(sb + kk * 32), (sl >= 2 || kb > kb0 || kk > 0) ? 1u : 0u);
            umma_commit(empty_bar(s));  // frees the stage once these products have read it
            if (++s == STAGES) { s = 0; ph ^= 1u; }
          }
          if (!ok) break;
          umma_commit(tfull_bar(b));    // accumulator b holds the slab's sums
        }
      }
      if (!ok) {                        // wait for every product this thread issued
        umma_commit(drain_bar);
        mbar_drain(drain_bar, 0);
      }
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    // As in the pair kernel: slab sl lands in accumulator sl & 1 on top of what
    // it holds; the epilogue writes each residue r (|r| <= 120) back while slab
    // sl + 2 accumulates on it, keeps the residue of slab nsl - 2 as a byte,
    // and turns the last slab's sum into the digit in fp32.
    const int e = warp - 2;
    const int quarter = warp & 3;            // TMEM lanes 32*quarter .. +31
    const int cbase = (e >> 2) * CPW1;       // columns cbase .. cbase + CPW1 - 1
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint32_t g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < num_units && ok; t += gridDim.x) {
      const Unit u = unit_of(p, t);
      const Coord c = u.c;
      const int nslabs = u.nslabs;
      const EpiConst k = epi_const((float)T.m[c.q], T.invm[c.q], p.raw ? 1.0f : (float)T.inv[c.q]);
      uint32_t acc8[CPW1 / 4];
#pragma unroll
      for (int i = 0; i < CPW1 / 4; ++i) acc8[i] = 0x80808080u;
      for (int sl = 0; sl < nslabs; ++sl, ++g) {
        const uint32_t b = g & 1u, use = g >> 1;
        if (!mbar_wait(tfull_bar(b), use & 1u, abort_flag, p.status)) { ok = false; break; }
        tc_fence_after();
        if constexpr (ONE) {
          const uint32_t tb = tempty_bar(b);
          drain_one_slab<CPW1 / 32>(tmem_base + lane_addr + b * BN + cbase, acc8, k,
                                    [&] {
                                      __syncwarp();
                                      if (lane == 0) mbar_arrive(tb);
                                    });
          continue;
        }
        const bool write_back = sl + 2 < nslabs;
        const bool last = sl + 1 == nslabs;
#pragma unroll
        for (int ch = 0; ch < CPW1 / 32; ++ch) {
          const uint32_t taddr = tmem_base + lane_addr + b * BN + cbase + ch * 32;
          uint32_t v[32];
          tmem_ld32(taddr, v);
          tmem_ld_wait();
          if (write_back) {
            residues32(v, k);
            tmem_st32(taddr, v);
          } else {
#pragma unroll
            for (int w = 0; w < 8; ++w) acc8[ch * 8 + w] = bytes4(v + 4 * w, acc8[ch * 8 + w], last, nslabs > 1, k);
          }
        }
        if (write_back) tmem_st_wait();
        tc_fence_before();
        mbar_arrive(tempty_bar(b));
      }
      if (!ok) break;
      // ---- tile done: acc8 holds the digits (or W mod m), one byte per entry ----
      const int row = c.tm * BM + quarter * 32 + lane;
      const int col0 = c.tn * BN + cbase;
      if (row < p.m && col0 < p.n) {
        uint8_t* dst = p.Y + (size_t)u.ks * p.ysplit + (size_t)c.q * p.m * p.ldy + (size_t)row * p.ldy + col0;
        store_digits<CPW1 / 4>(dst, acc8, p.n - col0, (p.ldy & 15) == 0 && (reinterpret_cast<uintptr_t>(p.Y) & 15) == 0,
                               p.acc, T.m[c.q]);
      }
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
// The same product on CTA pairs (cluster of 2, tcgen05 cta_group::2): a pair
// computes a 256 x 256 output tile; each CTA stages its 128 rows of A and its
// 128 rows of B (a third less shared-memory and L2 traffic per SM than the
// 128 x 256 tile of one CTA), the leader (rank 0) issues M = 256 products that
// read both CTAs' stages and write 128 rows into each CTA's tensor memory.
//   full[s]   leader only: counts both CTAs' copies of stage s;
//   empty[s]  each CTA: its stage s may be refilled (multicast commit);
//   tfull[b]  each CTA: accumulator b holds a slab (multicast commit);
//   tempty[b] leader only: both CTAs' epilogues have drained accumulator b.
// ---------------------------------------------------------------------------
constexpr int P_BM = 128;                          // rows of A per CTA
constexpr int P_BN = 128;                          // rows of B per CTA (N = 256 per pair)
constexpr int P_STAGES = 7;
constexpr int P_A_BYTES = P_BM * BK * 2;           // 16 KiB
constexpr int P_STAGE_BYTES = P_A_BYTES + P_BN * BK * 2;   // 32 KiB
constexpr int P_SMEM_BYTES = P_STAGES * P_STAGE_BYTES + kBarBytes + 1024;
// full and empty barriers per stage, two tfull, two tempty, one drain: all below kHolderOff
static_assert((2 * P_STAGES + 5) * 8 <= kHolderOff, "pair kernel barriers overlap the TMEM address");
static_assert((2 * STAGES + 5) * 8 <= kHolderOff, "barriers overlap the TMEM address");
// Epilogue warps of the pair kernel: sixteen when every unit is one slab
// (the epilogue then bounds the kernel) and for grouped products; four for a
// product of several slabs, where fewer warps beside the MMA-issuing thread
// leave it more issue slots: with the packed epilogue arithmetic one warp
// drains its 256 columns of a slab well within the slab's products.
constexpr int kPairEpiWarps = 16;
constexpr int kPairEpiWarpsMulti = 4;

// What a CTA pair needs to know about one unit of work: the tensor maps and
// first plane rows of its 256 x 256 tile, its k-block range, its modulus and
// where its digits go.
struct PairUnit {
  const CUtensorMap* mA;
  const CUtensorMap* mB;
  int ya, yb;               // first rows of the pair tile in the stacked planes of A and B
  int kb0, kb1, nslabs;     // k blocks [kb0, kb1) in nslabs slabs
  int q;                    // modulus index
  uint8_t* Y;               // digit plane of this unit (row pitch ldy, m rows, n columns)
  int64_t ldy;
  int m, n, row0, col0;     // the output's size and the tile's first row and column
  int acc, raw;
};

// One product (oz_dgemm): units are (split, modulus, tile), as unit_of orders them.
struct PairSingle {
  CUtensorMap mapA, mapB;
  Params p;
  __device__ __forceinline__ int units() const { return p.num_tiles * p.nsplit; }
  __device__ __forceinline__ int32_t* status() const { return p.status; }
  __device__ __forceinline__ int first(int) const { return 0; }
  __device__ __forceinline__ void prefetch() const {
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapB) : "memory");
  }
  __device__ __forceinline__ PairUnit unit(int t, int&) const {
    const Unit u = unit_of(p, t);
    PairUnit w;
    w.mA = &mapA;
    w.mB = &mapB;
    w.ya = u.c.q * p.m_pad + u.c.tm * 2 * P_BM;
    w.yb = u.c.q * p.n_pad + u.c.tn * 2 * P_BN;
    w.kb0 = u.kb0;
    w.kb1 = u.kb1;
    w.nslabs = u.nslabs;
    w.q = u.c.q;
    w.Y = p.Y + (size_t)u.ks * p.ysplit + (size_t)u.c.q * p.m * p.ldy;
    w.ldy = p.ldy;
    w.m = p.m;
    w.n = p.n;
    w.row0 = u.c.tm * 2 * P_BM;
    w.col0 = u.c.tn * 2 * P_BN;
    w.acc = p.acc;
    w.raw = p.raw;
    return w;
  }
};

// Grouped products (oz_group_run): unit t belongs to the problem whose unit
// range holds it (problems in decreasing order of k, so the longest units go
// first); a role carries the index of its current problem forward, since a
// pair visits its units in increasing order. Tensor maps in global memory,
// 128-row boxes for both operands.
struct PairGrouped {
  const OzGroupProblem* probs;
  int count, total;
  int32_t* st;
  __device__ __forceinline__ int units() const { return total; }
  __device__ __forceinline__ int32_t* status() const { return st; }
  __device__ __forceinline__ int first(int t) const {
    return group_find(probs, count, (int64_t)(t < total ? t : 0), [](const OzGroupProblem& q) { return q.unit_begin; });
  }
  __device__ __forceinline__ void prefetch() const {}
  __device__ __forceinline__ PairUnit unit(int t, int& pi) const {
    while (pi + 1 < count && probs[pi + 1].unit_begin <= t) ++pi;
    const OzGroupProblem& P = probs[pi];
    const int tiles_m = (int)((P.m + 2 * P_BM - 1) / (2 * P_BM));
    const Coord c = tile_coord(t - (int)P.unit_begin, tiles_m, P.tiles_n);
    PairUnit w;
    w.mA = &P.mapA;
    w.mB = &P.mapB;
    w.ya = c.q * (int)P.m_pad + c.tm * 2 * P_BM;
    w.yb = c.q * (int)P.n_pad + c.tn * 2 * P_BN;
    w.kb0 = 0;
    w.kb1 = P.kblocks;
    w.nslabs = (P.kblocks + kSlabBlocks - 1) / kSlabBlocks;
    w.q = c.q;
    w.Y = P.Y + (size_t)c.q * P.m * P.ldy;
    w.ldy = P.ldy;
    w.m = (int)P.m;
    w.n = (int)P.n;
    w.row0 = c.tm * 2 * P_BM;
    w.col0 = c.tn * 2 * P_BN;
    w.acc = 0;
    w.raw = 0;
    return w;
  }
};

// EW epilogue warps (4, 8 or 16): every warp drains the 32 TMEM lanes of its
// quarter (warp index mod 4), over CPW = 256 / (EW / 4) columns.
// S: the unit scheduler (PairSingle or PairGrouped).
template <int EW, typename S, bool ONE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__((2 + EW) * 32, 1)
gemm_tc_pair_kernel(const __grid_constant__ S sched, const __grid_constant__ OzTables T) {
  constexpr int CPW = 1024 / EW;            // columns per epilogue warp
  static_assert(EW == 4 || EW == 8 || EW == 16, "4, 8 or 16 epilogue warps");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_base = smem_u32(smem_raw);
  const uint32_t base = (raw_base + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw_base);
  const uint32_t bar0 = base + P_STAGES * P_STAGE_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (P_STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * P_STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * P_STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * P_STAGES + 4);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gbase + P_STAGES * P_STAGE_BYTES + kHolderOff);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + P_STAGES * P_STAGE_BYTES + kAbortOff);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), ONE ? 2 * EW : 2 * EW * 32);        // one-slab: one arrival per warp
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sched.prefetch();
  }
  if (warp == 1) {                          // one warp of each CTA: the pair's allocation
    tmem_alloc_pair(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();                           // both CTAs' barriers exist before any remote use
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  const int num_units = sched.units();
  int32_t* const status = sched.status();

  if (warp == 0) {
    // ------------------------------ TMA producer (both CTAs) ------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued_parity[P_STAGES];
      bool outstanding[P_STAGES];
      for (int i = 0; i < P_STAGES; ++i) outstanding[i] = false, issued_parity[i] = 0;
      bool ok = true;
      int pi = sched.first(pair);
      for (int t = pair; t < num_units && ok; t += npairs) {
        const PairUnit u = sched.unit(t, pi);
        const int ya = u.ya + (int)rank * P_BM;
        const int yb = u.yb + (int)rank * P_BN;
        for (int kb = u.kb0; kb < u.kb1; ++kb) {
          if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, status)) { ok = false; break; }
          outstanding[s] = false;
          const uint32_t sa = base + s * P_STAGE_BYTES;
          if (leader) mbar_expect_tx(full_bar(s), 2 * P_STAGE_BYTES);
          const uint32_t fb = mapa(full_bar(s), 0);
          tma_load_2d_pair(sa, u.mA, fb, kb * BK, ya);
          tma_load_2d_pair(sa + P_A_BYTES, u.mB, fb, kb * BK, yb);
          outstanding[s] = true;
          issued_parity[s] = ph;
          if (++s == P_STAGES) { s = 0; ph ^= 1u; }
        }
      }
      // both CTAs' copies complete on the leader's barriers: the leader waits
      // (bounded) for every stage it expected before the pair may exit
      if (!ok && leader) {
        for (int i = 0; i < P_STAGES; ++i)
          if (outstanding[i]) mbar_drain(full_bar(i), issued_parity[i]);
      }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer (leader) ------------------------------
    if (lane == 0 && leader) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t g = 0;
      bool ok = true;
      int pi = sched.first(pair);
      for (int t = pair; t < num_units && ok; t += npairs) {
        const PairUnit u = sched.unit(t, pi);
        for (int sl = 0; sl < u.nslabs && ok; ++sl, ++g) {
          const uint32_t b = g & 1u, use = g >> 1;
          if (!mbar_wait(tempty_bar(b), (use & 1u) ^ 1u, abort_flag, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dtm = tmem_base + b * 256;
          const int kb0 = u.kb0 + sl * kSlabBlocks;
          const int kb1 = min(u.kb1, kb0 + kSlabBlocks);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(full_bar(s), ph, abort_flag, status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = base + s * P_STAGE_BYTES;
            const uint32_t sb = sa + P_A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              umma_bf16_pair(dtm, sdesc(sa + kk * 32), sdesc(sb + kk * 32), (sl >= 2 || kb > kb0 || kk > 0) ? 1u : 0u);
            umma_commit_pair_both(empty_bar(s));
            if (++s == P_STAGES) { s = 0; ph ^= 1u; }
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
    // Slab sl of a tile lands in accumulator sl & 1 on top of what that
    // accumulator holds. The epilogue reduces each value t (|t| < 2^24) to
    // r = t - m rint(t / m), |r| <= 120, and writes r back when slab sl + 2
    // accumulates on it; the residue of slab nsl - 2 is kept as one byte per
    // entry and added to that of the last slab (eq. ov-comrtc: every partial
    // sum stays below 2^24, so the FP32 arithmetic is exact). Each warp drains
    // the 32 TMEM lanes of its quarter (warp index mod 4) over CPW columns.
    const int e = warp - 2;
    const int quarter = warp & 3;
    const int cbase = (e >> 2) * CPW;          // first column this warp drains
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint32_t g = 0;
    bool ok = true;
    int pi = sched.first(pair);
    for (int t = pair; t < num_units && ok; t += npairs) {
      const PairUnit u = sched.unit(t, pi);
      const int nslabs = u.nslabs;
      const EpiConst k = epi_const((float)T.m[u.q], T.invm[u.q], u.raw ? 1.0f : (float)T.inv[u.q]);
      uint32_t acc8[CPW / 4];                // residue + 128 of the chain of slab nsl - 2, one byte per column
#pragma unroll
      for (int i = 0; i < CPW / 4; ++i) acc8[i] = 0x80808080u;
      for (int sl = 0; sl < nslabs; ++sl, ++g) {
        const uint32_t b = g & 1u, use = g >> 1;
        if (!mbar_wait(tfull_bar(b), use & 1u, abort_flag, status)) { ok = false; break; }
        tc_fence_after();
        if constexpr (ONE) {
          const uint32_t tb = mapa(tempty_bar(b), 0);
          drain_one_slab<CPW / 32>(tmem_base + lane_addr + b * 256 + cbase, acc8, k,
                                   [&] {
                                     __syncwarp();
                                     if (lane == 0) mbar_arrive_cluster(tb);
                                   });
          continue;
        }
        const bool write_back = sl + 2 < nslabs;
        const bool last = sl + 1 == nslabs;
#pragma unroll
        for (int ch = 0; ch < CPW / 32; ++ch) {
          const uint32_t taddr = tmem_base + lane_addr + b * 256 + cbase + ch * 32;
          uint32_t v[32];
          tmem_ld32(taddr, v);
          tmem_ld_wait();
          if (write_back) {
            residues32(v, k);
            tmem_st32(taddr, v);
          } else {
#pragma unroll
            for (int w = 0; w < 8; ++w) acc8[ch * 8 + w] = bytes4(v + 4 * w, acc8[ch * 8 + w], last, nslabs > 1, k);
          }
        }
        if (write_back) tmem_st_wait();
        tc_fence_before();
        mbar_arrive_cluster(mapa(tempty_bar(b), 0));
      }
      if (!ok) break;
      // ---- tile done: acc8 holds the digits (or W mod m), one byte per entry ----
      const int row = u.row0 + (int)rank * P_BM + quarter * 32 + lane;
      const bool runs = (u.ldy & 15) == 0 && (reinterpret_cast<uintptr_t>(u.Y) & 15) == 0;
#pragma unroll
      for (int part = 0; part < (CPW + 127) / 128; ++part) {
        const int col0 = u.col0 + cbase + part * 128;
        if (row < u.m && col0 < u.n) {
          uint8_t* dst = u.Y + (size_t)row * u.ldy + col0;
          store_digits<(CPW < 128 ? CPW : 128) / 4>(dst, acc8 + part * 32, u.n - col0, runs, u.acc, T.m[u.q]);
        }
      }
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

// ---------------------------------------------------------------------------
// Grouped products (oz_group_run): the one-CTA kernel over the units of many
// products of one plan. Unit t belongs to the problem whose unit range holds
// it (problems in decreasing order of k, so the longest units go first); that
// problem's descriptor gives its tensor maps (in global memory), padding, k
// blocks and output. Roles and barriers as in gemm_tc_kernel.
// ---------------------------------------------------------------------------
template <bool ONE>
__global__ void __launch_bounds__(kThreads, 1)
gemm_tc_grouped_kernel(const __grid_constant__ OzTables T, const OzGroupProblem* __restrict__ probs, int count,
                       int64_t total_units, int32_t* status) {
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
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gbase + STAGES * STAGE_BYTES + kHolderOff);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + STAGES * STAGE_BYTES + kAbortOff);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  auto unit_begin = [](const OzGroupProblem& q) { return q.unit_begin; };
  // a CTA visits its units in increasing order, so each role carries the
  // index of the current problem forward instead of searching per unit
  auto advance = [&](int pi, int64_t t) {
    while (pi + 1 < count && probs[pi + 1].unit_begin <= t) ++pi;
    return pi;
  };
  const int pi0 = group_find(probs, count, (int64_t)blockIdx.x < total_units ? (int64_t)blockIdx.x : 0, unit_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), ONE ? kEpiWarps : kEpiWarps * 32);   // one-slab: one arrival per warp
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued_parity[STAGES];
      bool outstanding[STAGES];
      for (int i = 0; i < STAGES; ++i) outstanding[i] = false, issued_parity[i] = 0;
      bool ok = true;
      int pi = pi0;
      for (int64_t t = blockIdx.x; t < total_units && ok; t += gridDim.x) {
        pi = advance(pi, t);
        const OzGroupProblem& P = probs[pi];
        const Coord c = tile_coord((int)(t - P.unit_begin), P.tiles_m, P.tiles_n);
        const int ya = c.q * (int)P.m_pad + c.tm * BM;
        const int yb = c.q * (int)P.n_pad + c.tn * BN;
        for (int kb = 0; kb < P.kblocks; ++kb) {
          if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, status)) { ok = false; break; }
          outstanding[s] = false;
          const uint32_t sa = base + s * STAGE_BYTES;
          mbar_expect_tx(full_bar(s), STAGE_BYTES);
          tma_load_2d(sa, &P.mapA, full_bar(s), kb * BK, ya);
          tma_load_2d(sa + A_BYTES, &P.mapB, full_bar(s), kb * BK, yb);
          outstanding[s] = true;
          issued_parity[s] = ph;
          if (++s == STAGES) { s = 0; ph ^= 1u; }
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
      uint32_t g = 0;
      bool ok = true;
      int pi = pi0;
      for (int64_t t = blockIdx.x; t < total_units && ok; t += gridDim.x) {
        pi = advance(pi, t);
        const OzGroupProblem& P = probs[pi];
        const int kblocks = P.kblocks;
        const int nslabs = (kblocks + kSlabBlocks - 1) / kSlabBlocks;
        for (int sl = 0; sl < nslabs && ok; ++sl, ++g) {
          const uint32_t b = g & 1u, use = g >> 1;
          if (!mbar_wait(tempty_bar(b), (use & 1u) ^ 1u, abort_flag, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dtm = tmem_base + b * BN;
          const int kb0 = sl * kSlabBlocks;
          const int kb1 = min(kblocks, kb0 + kSlabBlocks);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(full_bar(s), ph, abort_flag, status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = base + s * STAGE_BYTES;
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              umma_bf16(dtm, sdesc(sa + kk * 32), sdesc(sb + kk * 32), (sl >= 2 || kb > kb0 || kk > 0) ? 1u : 0u);
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
    const int cbase = (e >> 2) * CPW1;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint32_t g = 0;
    bool ok = true;
    int pi = pi0;
      for (int64_t t = blockIdx.x; t < total_units && ok; t += gridDim.x) {
      pi = advance(pi, t);
        const OzGroupProblem& P = probs[pi];
      const Coord c = tile_coord((int)(t - P.unit_begin), P.tiles_m, P.tiles_n);
      const int nslabs = (P.kblocks + kSlabBlocks - 1) / kSlabBlocks;
      const EpiConst k = epi_const((float)T.m[c.q], T.invm[c.q], (float)T.inv[c.q]);
      uint32_t acc8[CPW1 / 4];
#pragma unroll
      for (int i = 0; i < CPW1 / 4; ++i) acc8[i] = 0x80808080u;
      for (int sl = 0; sl < nslabs; ++sl, ++g) {
        const uint32_t b = g & 1u, use = g >> 1;
        if (!mbar_wait(tfull_bar(b), use & 1u, abort_flag, status)) { ok = false; break; }
        tc_fence_after();
        if constexpr (ONE) {
          const uint32_t tb = tempty_bar(b);
          drain_one_slab<CPW1 / 32>(tmem_base + lane_addr + b * BN + cbase, acc8, k,
                                    [&] {
                                      __syncwarp();
                                      if (lane == 0) mbar_arrive(tb);
                                    });
          continue;
        }
        const bool write_back = sl + 2 < nslabs;
        const bool last = sl + 1 == nslabs;
#pragma unroll
        for (int ch = 0; ch < CPW1 / 32; ++ch) {
          const uint32_t taddr = tmem_base + lane_addr + b * BN + cbase + ch * 32;
          uint32_t v[32];
          tmem_ld32(taddr, v);
          tmem_ld_wait();
          if (write_back) {
            residues32(v, k);
            tmem_st32(taddr, v);
          } else {
#pragma unroll
            for (int w = 0; w < 8; ++w) acc8[ch * 8 + w] = bytes4(v + 4 * w, acc8[ch * 8 + w], last, nslabs > 1, k);
          }
        }
        if (write_back) tmem_st_wait();
        tc_fence_before();
        mbar_arrive(tempty_bar(b));
      }
      if (!ok) break;
      const int row = c.tm * BM + quarter * 32 + lane;
      const int col0 = c.tn * BN + cbase;
      if (row < P.m && col0 < P.n) {
        uint8_t* dst = P.Y + (size_t)c.q * P.m * P.ldy + (size_t)row * P.ldy + col0;
        store_digits<CPW1 / 4>(dst, acc8, P.n - col0, (P.ldy & 15) == 0 && (reinterpret_cast<uintptr_t>(P.Y) & 15) == 0,
                               0, T.m[c.q]);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
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

bool make_map(CUtensorMap* map, const void* planes, int64_t rows, int64_t k_pad, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)k_pad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(planes), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The split-K fields of the kernel parameters: one range (the whole K) or
// the ranges of ksplit_for, whole slabs each, none of them empty.
bool set_split(Params* p, KSplit split, int64_t ysplit) {
  if (split.nsplit <= 1) {
    p->nsplit = 1;
    p->kbps = p->kblocks;
    p->ysplit = 0;
    return true;
  }
  if (split.kbps <= 0 || split.kbps % kSlabBlocks || (int64_t)(split.nsplit - 1) * split.kbps >= p->kblocks ||
      (int64_t)split.nsplit * split.kbps < p->kblocks || (int64_t)p->num_tiles * split.nsplit > INT32_MAX ||
      ysplit <= 0)
    return false;
  p->nsplit = split.nsplit;
  p->kbps = split.kbps;
  p->ysplit = ysplit;
  return true;
}

}  // namespace

cudaError_t launch_gemm_tc(const OzTables& t, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                           const void* U, const void* V, uint8_t* Y, int64_t ldy, int raw, int32_t* status,
                           cudaStream_t st, KSplit split, int64_t ysplit) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (ldy < n) return cudaErrorInvalidValue;
  // pair tiles: 256 x 256 per CTA pair
  if ((reinterpret_cast<uintptr_t>(U) & 127) || (reinterpret_cast<uintptr_t>(V) & 127) || k_pad % BK ||
      m_pad % (2 * P_BM) || n_pad % (2 * P_BN))
    return cudaErrorInvalidValue;
  const int64_t tiles_m = (m + 2 * P_BM - 1) / (2 * P_BM), tiles_n = (n + 2 * P_BN - 1) / (2 * P_BN);
  const int64_t num_tiles = tiles_m * tiles_n * t.Q;
  if (num_tiles > INT32_MAX || (int64_t)t.Q * m_pad > INT32_MAX || (int64_t)t.Q * n_pad > INT32_MAX)
    return cudaErrorInvalidValue;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, U, (int64_t)t.Q * m_pad, k_pad, P_BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, V, (int64_t)t.Q * n_pad, k_pad, P_BN)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // A pair's CTA takes all the shared memory a block may have, so that no CTA
  // of another kernel shares its SM: CTA-pair GEMMs running beside other
  // kernels' CTAs on several streams were seen to stall.
  int smem_optin = 0;
  e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const int smem_bytes = smem_optin > P_SMEM_BYTES ? smem_optin : P_SMEM_BYTES;
  // every unit one slab (K <= 1024, unsplit): the kernel whose epilogue
  // releases each accumulator before forming its digits
  const bool one = k_pad <= (int64_t)kSlabBlocks * BK && split.nsplit <= 1;
  auto kernel = one ? gemm_tc_pair_kernel<kPairEpiWarps, PairSingle, true>
                    : gemm_tc_pair_kernel<kPairEpiWarpsMulti, PairSingle, false>;
  const int epi_warps = one ? kPairEpiWarps : kPairEpiWarpsMulti;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  PairSingle sched;
  sched.mapA = mapA;
  sched.mapB = mapB;
  Params& p = sched.p;
  p.m = (int)m;
  p.n = (int)n;
  p.tiles_m = (int)tiles_m;
  p.tiles_n = (int)tiles_n;
  p.num_tiles = (int)num_tiles;
  p.kblocks = (int)(k_pad / BK);
  p.m_pad = (int)m_pad;
  p.n_pad = (int)n_pad;
  p.raw = raw & kEpiRaw;
  p.acc = (raw & kEpiAccumulate) != 0;
  p.Y = Y;
  p.ldy = ldy;
  p.status = status;
  if (!set_split(&p, split, ysplit)) return cudaErrorInvalidValue;
  const int64_t units = num_tiles * p.nsplit;
  const int64_t pairs = units < sms / 2 ? units : sms / 2;
  kernel<<<(unsigned)(2 * pairs), (2 + epi_warps) * 32, smem_bytes, st>>>(sched, t);
  return cudaGetLastError();
}

// Tensor maps of one grouped problem's planes (rows of Q planes): 128-row
// boxes for A; for B 128-row boxes (CTA pairs) or 256-row boxes (the one-CTA
// kernel).
bool group_maps_tc(OzGroupProblem* pr, int Q, bool pairs) {
  return make_map(&pr->mapA, pr->U, (int64_t)Q * pr->m_pad, pr->k_pad, BM) &&
         make_map(&pr->mapB, pr->V, (int64_t)Q * pr->n_pad, pr->k_pad, pairs ? P_BN : BN);
}

cudaError_t launch_gemm_tc_grouped(const OzTables& t, const OzGroupProblem* probs, int count, int64_t total_units,
                                   int32_t* status, cudaStream_t st, bool pairs, bool one_slab) {
  if (count == 0 || total_units == 0) return cudaSuccess;
  if (total_units > INT32_MAX) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (pairs) {
    // as launch_gemm_tc: each CTA of a pair claims all the shared memory a block may have
    int smem_optin = 0;
    e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int smem_bytes = smem_optin > P_SMEM_BYTES ? smem_optin : P_SMEM_BYTES;
    auto kernel = one_slab ? gemm_tc_pair_kernel<kPairEpiWarps, PairGrouped, true>
                           : gemm_tc_pair_kernel<kPairEpiWarps, PairGrouped, false>;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    PairGrouped sched;
    sched.probs = probs;
    sched.count = count;
    sched.total = (int)total_units;
    sched.st = status;
    const int64_t pairs_n = total_units < sms / 2 ? total_units : sms / 2;
    kernel<<<(unsigned)(2 * pairs_n), (2 + kPairEpiWarps) * 32, smem_bytes, st>>>(sched, t);
    return cudaGetLastError();
  }
  auto kernel1 = one_slab ? gemm_tc_grouped_kernel<true> : gemm_tc_grouped_kernel<false>;
  e = cudaFuncSetAttribute(kernel1, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  const int grid = (int)(total_units < sms ? total_units : sms);
  kernel1<<<grid, kThreads, kSmemBytes, st>>>(t, probs, count, total_units, status);
  return cudaGetLastError();
}

// The one-CTA kernel (128 x 256 tiles), kept for comparison.
cudaError_t launch_gemm_tc_single(const OzTables& t, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad,
                                  int64_t k_pad, const void* U, const void* V, uint8_t* Y, int64_t ldy, int raw,
                                  int32_t* status, cudaStream_t st, KSplit split, int64_t ysplit) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (ldy < n) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(U) & 127) || (reinterpret_cast<uintptr_t>(V) & 127) || k_pad % BK ||
      m_pad % BM || n_pad % BN)
    return cudaErrorInvalidValue;
  const int64_t tiles_m = (m + BM - 1) / BM, tiles_n = (n + BN - 1) / BN;
  const int64_t num_tiles = tiles_m * tiles_n * t.Q;
  if (num_tiles > INT32_MAX || (int64_t)t.Q * m_pad > INT32_MAX || (int64_t)t.Q * n_pad > INT32_MAX)
    return cudaErrorInvalidValue;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, U, (int64_t)t.Q * m_pad, k_pad, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mapB, V, (int64_t)t.Q * n_pad, k_pad, BN)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const bool one = k_pad <= (int64_t)kSlabBlocks * BK && split.nsplit <= 1;
  auto kernel = one ? gemm_tc_kernel<true> : gemm_tc_kernel<false>;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  Params p;
  p.m = (int)m;
  p.n = (int)n;
  p.tiles_m = (int)tiles_m;
  p.tiles_n = (int)tiles_n;
  p.num_tiles = (int)num_tiles;
  p.kblocks = (int)(k_pad / BK);
  p.m_pad = (int)m_pad;
  p.n_pad = (int)n_pad;
  p.raw = raw & kEpiRaw;
  p.acc = (raw & kEpiAccumulate) != 0;
  p.Y = Y;
  p.ldy = ldy;
  p.status = status;
  if (!set_split(&p, split, ysplit)) return cudaErrorInvalidValue;
  const int64_t units = num_tiles * p.nsplit;
  const int grid = (int)(units < sms ? units : sms);
  kernel<<<grid, kThreads, kSmemBytes, st>>>(mapA, mapB, t, p);
  return cudaGetLastError();
}

}  // namespace oz
