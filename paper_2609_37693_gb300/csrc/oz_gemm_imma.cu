// oz_gemm_imma.cu -- phases 3 (GEMMs) and 4 (Epilogue) of Sec. "Structure" on
// the INT8 unit: W_q = U_q V_q^T with exact INT32 accumulation, then W_q
// reduced modulo m_q in the epilogue (order R>C of eq. ov-com; one accumulator
// and lambda = 1, so the epilogue is a single reduction).
//
// sm_103a has no tcgen05 INT8 kind, so this engine issues the warp-level
// mma.sync.m16n8k32 s8 x s8 -> s32. Exactness: every product is at most
// 119^2 in magnitude and K <= floor((2^31 - 1) / 119^2) (eq. ov-acc), so no
// partial sum leaves INT32 whatever the order of the additions.
//
// CTA tile 128 x 256 x 128 bytes, 8 warps as 2 x 4 (warp tile 64 x 64), a
// 4-stage cp.async pipeline, 128-byte XOR swizzle in shared memory, ldmatrix
// fragments. Grid: (n tiles, m tiles, Q); consecutive CTAs share the A panel
// of one modulus.
#include <stdint.h>

#include "oz_internal.h"
#include "oz_device.cuh"

namespace oz {
namespace {

constexpr int BM = 128, BN = 256, BK = 128, STAGES = 4;
constexpr int kStageBytes = (BM + BN) * BK;
constexpr int kSmemBytes = STAGES * kStageBytes;
constexpr int kOutPitch = BN + 16;  // epilogue staging row pitch (bytes)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_s8(int32_t* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// swizzled byte offset of (row, 16-byte chunk) in a tile with 128-byte rows
__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return (uint32_t)(row * BK + ((chunk ^ (row & 7)) << 4));
}

// Epilogue value of one INT32 product entry.
__device__ __forceinline__ uint32_t epilogue(int32_t w, uint32_t m, uint32_t magic, uint32_t inv, int raw) {
  uint32_t neg = w < 0;
  uint32_t u = neg ? (uint32_t)(-(int64_t)w) : (uint32_t)w;
  uint32_t r = mod_barrett(u, m, magic);   // |W| mod m
  if (raw) return neg ? (r ? m - r : 0u) : r;
  uint32_t mult = neg ? m - inv : inv;      // (+-1) * inv mod m
  return mod_barrett(r * mult, m, magic);
}

__global__ void __launch_bounds__(256, 1)
gemm_imma_kernel(const __grid_constant__ OzTables T, int64_t m, int64_t n, int64_t k_pad, const int8_t* __restrict__ U,
                 int64_t u_plane, const int8_t* __restrict__ V, int64_t v_plane, uint8_t* __restrict__ Y,
                 int64_t ldy, int mode) {
  const int raw = mode & kEpiRaw;
  const bool accum = (mode & kEpiAccumulate) != 0;   // blocked call: add into Y modulo m
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;
  const int q = blockIdx.z;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int8_t* Ub = U + (int64_t)q * u_plane + m0 * k_pad;
  const int8_t* Vb = V + (int64_t)q * v_plane + n0 * k_pad;
  const int KT = (int)(k_pad / BK);
  const uint32_t sbase = smem_u32(smem);

  auto load_stage = [&](int stage, int kt) {
    const uint32_t sa = sbase + stage * kStageBytes;
    const uint32_t sb = sa + BM * BK;
    const int64_t k0 = (int64_t)kt * BK;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      int c = tid + 256 * i;
      if (c < BM * 8) {
        int row = c >> 3, ch = c & 7;
        cp_async16(sa + swz(row, ch), Ub + row * k_pad + k0 + ch * 16);
      } else {
        c -= BM * 8;
        int row = c >> 3, ch = c & 7;
        cp_async16(sb + swz(row, ch), Vb + row * k_pad + k0 + ch * 16);
      }
    }
  };

  int32_t acc[4][8][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0;

#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < KT) load_stage(s, s);
    cp_async_commit();
  }

  for (int kt = 0; kt < KT; ++kt) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    {
      int nk = kt + STAGES - 1;
      if (nk < KT) load_stage(nk % STAGES, nk);
      cp_async_commit();
    }
    const uint32_t sa = sbase + (kt % STAGES) * kStageBytes;
    const uint32_t sb = sa + BM * BK;
#pragma unroll
    for (int ks = 0; ks < BK / 32; ++ks) {
      uint32_t a[4][4];
      uint32_t b[8][2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        int row = wm * 64 + mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
        int ch = ks * 2 + (lane >> 4);
        ldmatrix_x4(sa + swz(row, ch), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
      }
#pragma unroll
      for (int np = 0; np < 4; ++np) {
        int row = wn * 64 + np * 16 + (lane & 7) + ((lane >> 4) & 1) * 8;
        int ch = ks * 2 + ((lane >> 3) & 1);
        ldmatrix_x4(sb + swz(row, ch), b[2 * np][0], b[2 * np][1], b[2 * np + 1][0], b[2 * np + 1][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) mma_s8(acc[mt][nt], a[mt], b[nt][0], b[nt][1]);
    }
  }
  cp_async_wait<0>();
  __syncthreads();

  // Epilogue: reduce, stage the bytes in shared memory, store rows of 16 bytes.
  const uint32_t mq = T.m[q], magic = T.magic[q], inv = T.inv[q];
  uint8_t* so = smem;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int hlf = 0; hlf < 2; ++hlf) {
        int row = wm * 64 + mt * 16 + (lane >> 2) + hlf * 8;
        int col = wn * 64 + nt * 8 + (lane & 3) * 2;
        uint32_t y0 = epilogue(acc[mt][nt][2 * hlf], mq, magic, inv, raw);
        uint32_t y1 = epilogue(acc[mt][nt][2 * hlf + 1], mq, magic, inv, raw);
        *reinterpret_cast<uint16_t*>(so + row * kOutPitch + col) = (uint16_t)(y0 | (y1 << 8));
      }
  __syncthreads();
  uint8_t* Yq = Y + (int64_t)q * m * ldy;
  const bool vec_ok = (ldy % 16) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  for (int c = tid; c < BM * (BN / 16); c += 256) {
    int row = c / (BN / 16), cb = (c % (BN / 16)) * 16;
    int64_t gi = m0 + row, gj = n0 + cb;
    if (gi >= m || gj >= n) continue;
    const uint8_t* src = so + row * kOutPitch + cb;
    uint8_t* dst = Yq + gi * ldy + gj;
    if (vec_ok && gj + 16 <= n) {
      uint4 o = *reinterpret_cast<const uint4*>(src);
      if (accum) {
        const uint32_t mm = mq * 0x01010101u;
        const uint4 old = *reinterpret_cast<const uint4*>(dst);
        o.x = addmod_bytes(o.x, old.x, mm);
        o.y = addmod_bytes(o.y, old.y, mm);
        o.z = addmod_bytes(o.z, old.z, mm);
        o.w = addmod_bytes(o.w, old.w, mm);
      }
      *reinterpret_cast<uint4*>(dst) = o;
    } else {
      for (int e = 0; e < 16 && gj + e < n; ++e) {
        uint32_t y = src[e];
        if (accum) {
          y += dst[e];
          y = y >= mq ? y - mq : y;
        }
        dst[e] = (uint8_t)y;
      }
    }
  }
}

}  // namespace

cudaError_t launch_gemm_imma(const OzTables& t, int64_t m, int64_t n, int64_t k_pad, const int8_t* U,
                             int64_t u_plane, const int8_t* V, int64_t v_plane, uint8_t* Y, int64_t ldy, int raw,
                             cudaStream_t st) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (ldy < n) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(gemm_imma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM), (unsigned)t.Q);
  gemm_imma_kernel<<<grid, 256, kSmemBytes, st>>>(t, m, n, k_pad, U, u_plane, V, v_plane, Y, ldy, raw);
  return cudaGetLastError();
}

}  // namespace oz
