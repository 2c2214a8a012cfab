// oz_plan.cpp -- host-side configuration builder (Sec. "Implementation": a
// configuration is its moduli, its tables and its caps; building it checks the
// accumulator bound and refuses K above the reconstruction cap).
//
// The INT8 alphabet is complete modulo every m <= 256 (Sec. "Forms and
// Channels"), so each channel is one-limb with the balanced residue as both
// tables and lambda = 1; its cost is one GEMM. The moduli are the Q
// pairwise-coprime integers <= 239 of largest product; for 9 <= Q <= 20 these
// are the first Q entries of kModuli below (Sec. "INT4 and INT8" fixes 16
// moduli up to 239 with radius 119 and K_max = 151 647).
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "oz_internal.h"

namespace {

const uint32_t kModuli[OZ_MAX_MODULI] = {239, 237, 236, 235, 233, 229, 227, 223, 221, 217,
                                         211, 209, 199, 197, 193, 191, 181, 179, 173, 167};

// Unsigned big integer, 32-bit limbs, least significant first; 8 limbs = 256 bits.
struct Big {
  uint32_t w[8];
  Big() { memset(w, 0, sizeof w); }
  explicit Big(uint64_t v) {
    memset(w, 0, sizeof w);
    w[0] = (uint32_t)v;
    w[1] = (uint32_t)(v >> 32);
  }
  Big mul(uint64_t s) const {  // s < 2^32
    Big r;
    uint64_t carry = 0;
    for (int i = 0; i < 8; ++i) {
      uint64_t t = (uint64_t)w[i] * s + carry;
      r.w[i] = (uint32_t)t;
      carry = t >> 32;
    }
    return r;
  }
  Big mulbig(const Big& o) const {  // truncated to 256 bits
    Big r;
    for (int i = 0; i < 8; ++i) {
      uint64_t carry = 0;
      for (int j = 0; i + j < 8; ++j) {
        uint64_t t = (uint64_t)w[i] * o.w[j] + r.w[i + j] + carry;
        r.w[i + j] = (uint32_t)t;
        carry = t >> 32;
      }
    }
    return r;
  }
  uint32_t divmod(uint32_t d, Big* q) const {  // returns remainder
    uint64_t rem = 0;
    for (int i = 7; i >= 0; --i) {
      uint64_t cur = (rem << 32) | w[i];
      q->w[i] = (uint32_t)(cur / d);
      rem = cur % d;
    }
    return (uint32_t)rem;
  }
  int cmp(const Big& o) const {
    for (int i = 7; i >= 0; --i)
      if (w[i] != o.w[i]) return w[i] < o.w[i] ? -1 : 1;
    return 0;
  }
  int bitlen() const {
    for (int i = 7; i >= 0; --i)
      if (w[i]) return 32 * i + 32 - __builtin_clz(w[i]);
    return 0;
  }
};

Big product(int Q) {
  Big P(1);
  for (int i = 0; i < Q; ++i) P = P.mul(kModuli[i]);
  return P;
}

// 2 K (2^beta - 1)^2, beta <= 96, K < 2^63
Big window(int64_t K, int beta) {
  Big b;  // 2^beta - 1
  for (int i = 0; i < beta; ++i) b.w[i / 32] |= 1u << (i % 32);
  Big sq = b.mulbig(b);
  Big twoK((uint64_t)K * 2u);
  return sq.mulbig(twoK);
}

bool window_holds(const Big& P, int64_t K, int beta) { return window(K, beta).cmp(P) < 0; }

uint32_t inverse_mod(uint32_t a, uint32_t m) {  // extended Euclid, gcd(a, m) = 1
  int64_t t = 0, newt = 1, r = m, newr = a % m;
  while (newr) {
    int64_t q = r / newr;
    int64_t tmp = t - q * newt; t = newt; newt = tmp;
    tmp = r - q * newr; r = newr; newr = tmp;
  }
  if (t < 0) t += m;
  return (uint32_t)t;
}

uint32_t pow2_mod(int e, uint32_t m) {
  uint64_t r = 1 % m;
  for (int i = 0; i < e; ++i) r = (r * 2) % m;
  return (uint32_t)r;
}

// Largest K (capped at 2^62) with 2 K (2^beta - 1)^2 < P: the reconstruction cap.
int64_t kappa_rec(const Big& P, int beta) {
  int64_t lo = 0, hi = (int64_t)1 << 62;
  if (window_holds(P, hi, beta)) return hi;
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (window_holds(P, mid, beta)) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace

namespace oz {

// Groups of moduli for the reconstruct of byte digits (oz_reconstruct.cu): as
// many triples as fit, the remaining one or two moduli joined to the last
// groups as one quad (when its product is below 2^31) or as pairs. Left
// unset (rg_nt = rg_np2 = rg_nq4 = 0) unless every bound the kernel relies on
// holds: digits and moduli below 256 (dp2a takes bytes), weights below 2^16,
// the sum of the groups' largest t_g below 2^32 (each 64-bit limb
// accumulator then stays below 2^64), N_g below 2^128, the CRT sum below
// 15 P (its quotient fits the kernel's table of 16 multiples of P), and
// 3P / 2 below 2^127 (the two's-complement candidate X).
void fill_group_tables(OzTables* tp, const uint32_t* moduli, int Q, const Big& P) {
  OzTables& t = *tp;
  t.rg_nt = t.rg_np2 = t.rg_nq4 = 0;
  if (Q < 2 || Q > 16 || P.bitlen() > 125) return;
  for (int q = 0; q < Q; ++q)
    if (moduli[q] >= 256) return;
  int nt = Q / 3, np2 = 0, nq4 = 0;
  if (Q % 3 == 2) np2 = 1;
  if (Q % 3 == 1) {
    --nt;                                   // the last triple and the lone modulus: a quad, or two pairs
    const uint64_t m4 = (uint64_t)moduli[Q - 4] * moduli[Q - 3] * moduli[Q - 2] * moduli[Q - 1];
    if (m4 < ((uint64_t)1 << 31)) nq4 = 1; else np2 = 2;
  }
  if (nt < 0 || nt + np2 + nq4 > OZ_RG_MAX) return;
  double tsum = 0.0, ksum = 0.0;            // sum of the largest t_g, sum of t_max / M_g
  int q = 0;
  for (int g = 0; g < nt + np2 + nq4; ++g) {
    uint64_t Mg = 1;
    int size = g < nt ? 3 : g < nt + np2 ? 2 : 4;
    for (int i = 0; i < size; ++i) Mg *= moduli[q + i];
    const uint32_t ma = moduli[q], mb = moduli[q + 1];
    if (size == 3) {
      const uint32_t mc = moduli[q + 2];
      if ((uint64_t)mb * mc >= 65536 || (uint64_t)ma * mc >= 65536 || (uint64_t)ma * mb >= 65536) return;
      t.rg_w0[g] = (mb * mc) | ((ma * mc) << 16);        // y_a (m_b m_c) + y_b (m_a m_c)
      t.rg_w1[g] = ma * mb;                               // y_c (m_a m_b)
      tsum += 3.0 * (double)Mg;
      ksum += 3.0;
    } else if (size == 2) {
      t.rg_w0[g] = mb | (ma << 16);                       // y_a m_b + y_b m_a
      t.rg_w1[g] = 0;
      tsum += 2.0 * (double)Mg;
      ksum += 2.0;
    } else {
      const uint32_t mc = moduli[q + 2], md = moduli[q + 3];
      t.rg_w0[g] = mb | (ma << 16);
      t.rg_w1[g] = md | (mc << 16);
      t.rg_m2a[g] = ma * mb;
      t.rg_m2b[g] = mc * md;
      if (ma * mb >= 65536 || mc * md >= 65536 || Mg >= ((uint64_t)1 << 31)) return;
      tsum += 2.0 * (double)Mg;
      ksum += 2.0;
    }
    Big N;
    Big Mb(1);
    for (int i = 0; i < size; ++i) Mb = Mb.mul(moduli[q + i]);
    // N = P / M_g by two exact divisions (M_g may exceed 2^32)
    Big N1;
    P.divmod(moduli[q], &N1);
    N = N1;
    for (int i = 1; i < size; ++i) {
      Big N2;
      N.divmod(moduli[q + i], &N2);
      N = N2;
    }
    if (N.bitlen() > 128) return;
    for (int l = 0; l < 4; ++l) t.rg_N[g][l] = N.w[l];
    t.rg_invM[g] = (float)(1.0 / (double)Mg);
    q += size;
  }
  if (q != Q || tsum >= 4294967296.0 || ksum > 15.0) return;
  t.rg_nt = nt;
  t.rg_np2 = np2;
  t.rg_nq4 = nq4;
}

// Per-modulus constants and the CRT sum's limbs for moduli m[0..Q-1] (pairwise
// coprime, each below 2^12): Barrett and reduction constants for the split
// kernels, (P/m)^-1 mod m for the epilogue, and P, P/m, and the pair products
// P/(m_a m_b) as 32-bit limbs for the reconstruct kernels.
bool fill_crt_tables(OzTables* tp, const uint32_t* moduli, int Q, int bits) {
  if (Q < 1 || Q > OZ_TABLE_CAP) return false;
  OzTables& t = *tp;
  memset(&t, 0, sizeof t);
  Big P(1);
  for (int i = 0; i < Q; ++i) P = P.mul(moduli[i]);
  t.Q = Q;
  t.bits = bits;
  // The reconstruct phase works modulo 2^(32 limbs) in two's complement. Its
  // candidate X lies in (-1.5P, 1.5P) and it compares 2X with +-P, so 3P must
  // stay below 2^(32 limbs - 1).
  t.limbs = (P.bitlen() + 3 + 31) / 32;
  if (t.limbs > OZ_MAX_LIMBS) return false;
  for (int i = 0; i < OZ_MAX_LIMBS; ++i) t.P[i] = P.w[i];
  for (int q = 0; q < Q; ++q) {
    uint32_t m = moduli[q];
    t.m[q] = m;
    t.magic[q] = (uint32_t)((((uint64_t)1) << 32) / m);
    Big Mk;
    P.divmod(m, &Mk);
    Big dummy;
    uint32_t mk_mod_m = Mk.divmod(m, &dummy);
    t.inv[q] = inverse_mod(mk_mod_m, m);
    t.invm[q] = 1.0f / (float)m;
    t.mf[q] = (float)m;
    auto centred = [m](uint32_t c) { return (float)(c >= (m + 1) / 2 ? (int)c - (int)m : (int)c); };
    for (int i = 0; i < 4; ++i) t.c13f[i][q] = centred(pow2_mod(22 + 13 * i, m));
    for (int i = 0; i < 6; ++i) t.c12f[i][q] = centred(pow2_mod(22 + 12 * i, m));
    t.halfm[q] = (m & 1u) ? 0.0f : (float)(m / 2);
  }
  t.npairs = (Q + 1) / 2;
  for (int pi = 0; pi < t.npairs; ++pi) {
    uint32_t ma = moduli[2 * pi], mb = 2 * pi + 1 < Q ? moduli[2 * pi + 1] : 1u;
    t.pa[pi] = ma;
    t.pb[pi] = mb;
    t.pinv[pi] = (float)(1.0 / ((double)ma * (double)mb));
    Big Np;
    P.divmod(ma * mb, &Np);
    for (int i = 0; i < OZ_MAX_LIMBS; ++i) t.Np[pi][i] = Np.w[i];
  }
  fill_group_tables(&t, moduli, Q, P);
  return true;
}

}  // namespace oz

extern "C" oz_status oz_plan_create(oz_plan* out, int num_moduli, int bits, int64_t k_hint, int engine) {
  if (!out) return OZ_ERR_INVALID_ARG;
  *out = nullptr;
  if (k_hint < 1 || bits < 0 || bits > OZ_MAX_BITS) return OZ_ERR_INVALID_ARG;
  if (engine < OZ_ENGINE_AUTO || engine > OZ_ENGINE_TC1 || engine == OZ_ENGINE_FP)
    return OZ_ERR_INVALID_ARG;   // float formats: oz_plan_create_fp
  if (num_moduli != 0 && (num_moduli < OZ_MIN_MODULI || num_moduli > OZ_MAX_MODULI)) return OZ_ERR_UNSUPPORTED;

  int Q = num_moduli;
  if (Q == 0) {  // least Q meeting the window at beta = 53 (eq. ov-crtgen)
    for (Q = OZ_MIN_MODULI; Q <= OZ_MAX_MODULI; ++Q)
      if (window_holds(product(Q), k_hint, 53)) break;
    if (Q > OZ_MAX_MODULI) return OZ_ERR_K_TOO_LARGE;
  }
  Big P = product(Q);
  int beta = bits;
  if (beta == 0) {
    for (beta = OZ_MAX_BITS; beta >= 1; --beta)
      if (window_holds(P, k_hint, beta)) break;
    if (beta < 1) return OZ_ERR_K_TOO_LARGE;
  } else if (!window_holds(P, k_hint, beta)) {
    return OZ_ERR_K_TOO_LARGE;
  }
  int resolved = engine == OZ_ENGINE_AUTO ? OZ_ENGINE_TC : engine;

  oz_plan p = new (std::nothrow) oz_plan_s;
  if (!p) return OZ_ERR_INVALID_ARG;
  memset(p, 0, sizeof *p);
  p->Q = Q;
  p->bits = beta;
  p->engine = resolved;
  // eq. caps: K_max = min(kappa_rec, kappa_acc). On the IMMA engine one INT32
  // accumulator sums K products of two residues of magnitude <= r (eq. ov-acc).
  // The TC engine accumulates in FP32 slabs of 1024 terms and reduces each slab
  // modulo m (Sec. "Slabs"), so only kappa_rec limits K there.
  uint32_t r = 0;
  for (int i = 0; i < Q; ++i) r = kModuli[i] / 2 > r ? kModuli[i] / 2 : r;
  int64_t k_acc = oz::engine_bf16(resolved) ? (int64_t)INT32_MAX : (int64_t)2147483647 / ((int64_t)r * r);
  int64_t k_rec = kappa_rec(P, beta);
  p->k_max = k_acc < k_rec ? k_acc : k_rec;
  p->k_acc = k_acc;
  p->k_rec = k_rec;
  if (k_hint > p->k_max) { delete p; return OZ_ERR_K_TOO_LARGE; }

  if (!oz::fill_crt_tables(&p->tab, kModuli, Q, beta)) { delete p; return OZ_ERR_UNSUPPORTED; }
  // the split kernels map the tie +m/2 of an even modulus to -m/2 for the
  // modulus at index 2 only (236 in the list); every other modulus is odd
  for (int q = 0; q < Q; ++q)
    if (q != 2 && (kModuli[q] & 1u) == 0) { delete p; return OZ_ERR_UNSUPPORTED; }
  p->gemms = Q;
  *out = p;
  return OZ_OK;
}

extern "C" oz_status oz_plan_info(oz_plan plan, int* q, int* bits, int64_t* k_max, int* engine, uint32_t* moduli) {
  if (!plan) return OZ_ERR_INVALID_ARG;
  if (q) *q = plan->Q;
  if (bits) *bits = plan->bits;
  if (k_max) *k_max = plan->k_max;
  if (engine) *engine = plan->engine;
  if (moduli) {
    for (int i = 0; i < OZ_MAX_MODULI; ++i) moduli[i] = i < plan->Q ? plan->tab.m[i] : 0;
  }
  return OZ_OK;
}

extern "C" oz_status oz_plan_caps(oz_plan plan, int64_t* k_acc, int64_t* k_rec) {
  if (!plan) return OZ_ERR_INVALID_ARG;
  if (k_acc) *k_acc = plan->k_acc;
  if (k_rec) *k_rec = plan->k_rec;
  return OZ_OK;
}

extern "C" void oz_plan_destroy(oz_plan plan) {
  if (!plan) return;
  if (plan->d_words) cudaFree(plan->d_words);
  delete[] plan->h_values;
  delete plan;
}

extern "C" const char* oz_status_str(oz_status s) {
  switch (s) {
    case OZ_OK: return "ok";
    case OZ_ERR_INVALID_ARG: return "invalid argument";
    case OZ_ERR_K_TOO_LARGE: return "inner dimension above the configuration's K_max";
    case OZ_ERR_WORKSPACE: return "workspace missing or too small";
    case OZ_ERR_NONFINITE: return "non-finite entry in an operand";
    case OZ_ERR_UNSUPPORTED: return "configuration or engine not supported";
    case OZ_ERR_CUDA: return "CUDA error";
  }
  return "unknown status";
}
