// oz_plan_fp.cpp -- configurations on the low-precision float alphabets
// (Sec. "Forms and Channels", Sec. "Forms Built from Limbs", Sec.
// "Instantiation"): a set of pairwise-coprime channels, each a modulus with a
// one-limb, schoolbook or Toom form over the format's alphabet S.
//
// The channel lists are frozen (oz_fp_configs.inc, written by
// gen_fp_configs.py from the exact search of fpsearch.py): per format, the
// least configuration for K_cfg = 2^13, 2^14 and 2^16 at beta = 53, and a
// widened one (beta = 69 at K_cfg = 2^14, Example ex:widened). A plan takes
// the base configuration of the least K_cfg >= k_hint, or, for a requested
// budget its window does not hold, the first widened one that holds it.
// Building a plan makes the forms' tables, weights and codes from them:
//   * alphabet S: the format's finite values scaled by 2^e_S, the least power of
//     two making them integers; a plane value v is stored as the code of v 2^-e_S;
//   * every plane value is at most r = floor(sqrt(2^24 / K_cfg)) in magnitude, so
//     one FP32 accumulator per GEMM is exact up to K_cfg (eq. ov-accgen, rmax);
//   * a class c is encoded by the tuple whose largest plane magnitude is least;
//     ties go to the smaller |a1|, then the smaller a1, then the smaller a0;
//   * forms (base b): one limb: plane a0, GEMM (0,0) weight 1;
//     schoolbook with m | b^2: planes a0, a1, GEMMs (0,0) 1, (0,1) b, (1,0) b;
//     Toom at {0, 1, inf}: planes a0, a0 + a1, a1, GEMMs (0,0) 1 - b, (1,1) b,
//     (2,2) b^2 - b; schoolbook: planes a0, a1, GEMMs (0,0) 1, (0,1) b, (1,0) b,
//     (1,1) b^2. Weights enter reduced into [0, m) (order R>C, eq. ov-comrtc).
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <vector>

#include "oz_internal.h"

namespace {

struct FpChannel {
  uint32_t m;
  int form, base;
};
struct FpConfig {
  int fmt;
  int64_t K;
  int beta;          // the bit budget it was searched for (53: base; wider: widened)
  int Q, nch;
  FpChannel ch[OZ_TABLE_CAP];
};

const FpConfig kFpConfigs[] = {
#include "oz_fp_configs.inc"
};

enum { F_ONE = 1, F_SCHOOL3 = 2, F_TOOM3 = 3, F_SCHOOL4 = 4 };

struct FormatBits {
  int e_bits, m_bits, bias;
  bool ieee_top, nan_top;
  int code_bits;
};

bool format_bits(int fmt, FormatBits* f) {
  switch (fmt) {
    case OZ_FMT_E4M3: *f = {4, 3, 7, false, true, 8}; return true;
    case OZ_FMT_E5M2: *f = {5, 2, 15, true, false, 8}; return true;
    case OZ_FMT_E2M3: *f = {2, 3, 1, false, false, 6}; return true;
    case OZ_FMT_E3M2: *f = {3, 2, 3, false, false, 6}; return true;
    case OZ_FMT_E2M1: *f = {2, 1, 1, false, false, 4}; return true;
    default: return false;
  }
}

// scaled integer value -> code, and e_S
bool alphabet(int fmt, std::map<int64_t, int>* code_of, int* e_s) {
  FormatBits f;
  if (!format_bits(fmt, &f)) return false;
  // every finite value is k 2^(1 - bias - m_bits) for an integer k, so e_S = bias + m_bits - 1
  *e_s = f.bias + f.m_bits - 1;
  code_of->clear();
  for (int sign = 0; sign < 2; ++sign)
    for (int e = 0; e < (1 << f.e_bits); ++e)
      for (int mt = 0; mt < (1 << f.m_bits); ++mt) {
        if (f.ieee_top && e == (1 << f.e_bits) - 1) continue;
        if (f.nan_top && e == (1 << f.e_bits) - 1 && mt == (1 << f.m_bits) - 1) continue;
        int64_t k = e == 0 ? mt : (int64_t)((1 << f.m_bits) + mt) << (e - 1);   // value = k 2^(1-bias-m_bits)
        int64_t v = sign ? -k : k;
        int code = (sign << (f.e_bits + f.m_bits)) | (e << f.m_bits) | mt;
        if (!code_of->count(v) || (v == 0 && sign == 0)) (*code_of)[v] = code;
      }
  return true;
}

uint32_t pow2_mod(int e, uint32_t m) {
  uint64_t r = 1 % m;
  for (int i = 0; i < e; ++i) r = (r * 2) % m;
  return (uint32_t)r;
}

uint32_t mod_pos(int64_t x, uint32_t m) {
  int64_t r = x % (int64_t)m;
  return (uint32_t)(r < 0 ? r + m : r);
}

struct Tuple {
  int64_t a0, a1;
};

// Plane value tables of one channel: out[p][c] for plane p, class c.
bool channel_tables(const std::vector<int64_t>& Sr, uint32_t m, int form, int base,
                    std::vector<std::vector<int64_t>>* out) {
  const int np = form == F_ONE ? 1 : (form == F_TOOM3 ? 3 : 2);
  out->assign(np, std::vector<int64_t>(m, 0));
  std::vector<char> seen(m, 0);
  uint32_t covered = 0;
  if (form == F_ONE) {
    std::vector<int64_t> one(Sr);
    std::sort(one.begin(), one.end(), [](int64_t x, int64_t y) {
      int64_t ax = x < 0 ? -x : x, ay = y < 0 ? -y : y;
      return ax != ay ? ax < ay : x < y;
    });
    for (int64_t v : one) {
      uint32_t c = mod_pos(v, m);
      if (!seen[c]) { seen[c] = 1; (*out)[0][c] = v; ++covered; }
    }
    return covered == m;
  }
  std::vector<int64_t> sset(Sr);
  std::vector<Tuple> cand;
  for (int64_t x : Sr)
    for (int64_t y : Sr) {
      if (form == F_TOOM3 && !std::binary_search(sset.begin(), sset.end(), x + y)) continue;
      cand.push_back({x, y});
    }
  auto mx = [form](const Tuple& t) {
    int64_t a = t.a0 < 0 ? -t.a0 : t.a0, b = t.a1 < 0 ? -t.a1 : t.a1;
    int64_t r = a > b ? a : b;
    if (form == F_TOOM3) {
      int64_t s = t.a0 + t.a1;
      s = s < 0 ? -s : s;
      r = r > s ? r : s;
    }
    return r;
  };
  std::stable_sort(cand.begin(), cand.end(), [&](const Tuple& x, const Tuple& y) {
    int64_t kx = mx(x), ky = mx(y);
    if (kx != ky) return kx < ky;
    int64_t ax = x.a1 < 0 ? -x.a1 : x.a1, ay = y.a1 < 0 ? -y.a1 : y.a1;
    if (ax != ay) return ax < ay;
    if (x.a1 != y.a1) return x.a1 < y.a1;
    return x.a0 < y.a0;
  });
  for (const Tuple& t : cand) {
    uint32_t c = mod_pos(t.a0 + (int64_t)base * t.a1, m);
    if (seen[c]) continue;
    seen[c] = 1;
    ++covered;
    if (form == F_TOOM3) {
      (*out)[0][c] = t.a0;
      (*out)[1][c] = t.a0 + t.a1;
      (*out)[2][c] = t.a1;
    } else {
      (*out)[0][c] = t.a0;
      (*out)[1][c] = t.a1;
    }
  }
  return covered == m;
}

// 256-bit helpers for the window (the INT8 planner has its own copy).
struct U256 {
  uint32_t w[8];
};
void u_mul(U256* x, uint64_t s) {
  uint64_t carry = 0;
  for (int i = 0; i < 8; ++i) {
    uint64_t t = (uint64_t)x->w[i] * s + carry;
    x->w[i] = (uint32_t)t;
    carry = t >> 32;
  }
}
int u_cmp(const U256& a, const U256& b) {
  for (int i = 7; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}
U256 u_window(int64_t K, int beta) {  // 2 K (2^beta - 1)^2
  U256 b = {};
  for (int i = 0; i < beta; ++i) b.w[i / 32] |= 1u << (i % 32);
  U256 r = {};
  for (int i = 0; i < 8; ++i) {
    uint64_t carry = 0;
    for (int j = 0; i + j < 8; ++j) {
      uint64_t t = (uint64_t)b.w[i] * b.w[j] + r.w[i + j] + carry;
      r.w[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  u_mul(&r, (uint64_t)2);
  // multiply by K (< 2^62) in two 31-bit halves
  U256 lo = r, hi = r;
  u_mul(&lo, (uint64_t)(K & 0x7fffffff));
  u_mul(&hi, (uint64_t)(K >> 31));
  for (int s = 0; s < 31; ++s) u_mul(&hi, 2);
  U256 out = {};
  uint64_t carry = 0;
  for (int i = 0; i < 8; ++i) {
    uint64_t t = (uint64_t)lo.w[i] + hi.w[i] + carry;
    out.w[i] = (uint32_t)t;
    carry = t >> 32;
  }
  return out;
}

}  // namespace

// Builds the OzTables (CRT constants) for a list of moduli; defined in oz_plan.cpp.
namespace oz {
bool fill_crt_tables(OzTables* t, const uint32_t* moduli, int Q, int bits);
}

extern "C" oz_status oz_plan_create_fp(oz_plan* out, int format, int64_t k_hint, int bits) {
  if (!out) return OZ_ERR_INVALID_ARG;
  *out = nullptr;
  if (k_hint < 1 || bits < 0 || bits > OZ_MAX_BITS_FP) return OZ_ERR_INVALID_ARG;
  std::map<int64_t, int> code_of;
  int e_s = 0;
  if (!alphabet(format, &code_of, &e_s)) return OZ_ERR_UNSUPPORTED;
  // the configuration: the base one (beta = 53) of the least K_cfg >= k_hint
  // whose window holds the requested bits (bits = 0: the base one of the least
  // K_cfg), else the widened one of the least K_cfg >= k_hint that holds them
  const FpConfig* cfg = nullptr;
  auto holds = [&](const FpConfig& c) {
    if (bits == 0) return true;
    U256 P = {};
    P.w[0] = 1;
    for (int i = 0; i < c.nch; ++i) u_mul(&P, c.ch[i].m);
    return u_cmp(u_window(k_hint, bits), P) < 0;
  };
  auto better = [&](const FpConfig& c) {
    if (!cfg) return true;
    const bool cw = c.beta > 53, bw = cfg->beta > 53;
    if (cw != bw) return !cw;                    // base configurations first
    return c.K < cfg->K || (c.K == cfg->K && c.Q < cfg->Q);
  };
  for (const FpConfig& c : kFpConfigs)
    if (c.fmt == format && c.K >= k_hint && holds(c) && better(c)) cfg = &c;
  if (!cfg) return OZ_ERR_K_TOO_LARGE;
  const int64_t r = (int64_t)std::sqrt((double)((1ll << 24) / cfg->K));
  int64_t rr = r;
  while ((rr + 1) * (rr + 1) <= (1ll << 24) / cfg->K) ++rr;
  while (rr * rr > (1ll << 24) / cfg->K) --rr;
  std::vector<int64_t> Sr;
  for (auto& kv : code_of)
    if (kv.first >= -rr && kv.first <= rr) Sr.push_back(kv.first);
  std::sort(Sr.begin(), Sr.end());

  oz_plan p = new (std::nothrow) oz_plan_s;
  if (!p) return OZ_ERR_INVALID_ARG;
  memset(p, 0, sizeof *p);
  p->is_fp = 1;
  p->engine = OZ_ENGINE_FP;
  p->fp_kcfg = cfg->K;
  OzFpTables& f = p->fp;
  f.fmt = format;
  f.e2 = 2 * e_s;
  FormatBits fb;
  format_bits(format, &fb);
  f.code_bits = fb.code_bits;
  f.nch = cfg->nch;
  std::vector<uint32_t> moduli(cfg->nch);
  std::vector<std::vector<int64_t>> planes;      // value tables, one per plane
  int64_t rho = 0;
  int g = 0;
  for (int c = 0; c < cfg->nch; ++c) {
    const uint32_t m = cfg->ch[c].m;
    const int form = cfg->ch[c].form, base = cfg->ch[c].base;
    // the epilogue's fp32 steps and 16-bit fields assume 5 <= m <= 4000
    if (m < 5 || m > 4000) { delete p; return OZ_ERR_UNSUPPORTED; }
    moduli[c] = m;
    p->fp_form[c] = form;
    p->fp_base[c] = base;
    std::vector<std::vector<int64_t>> t;
    if (!channel_tables(Sr, m, form, base, &t)) { delete p; return OZ_ERR_UNSUPPORTED; }
    f.m[c] = m;
    f.magic[c] = (uint32_t)((((uint64_t)1) << 32) / m);
    f.c16[c] = pow2_mod(16, m);
    f.c32[c] = pow2_mod(32, m);
    f.c48[c] = pow2_mod(48, m);
    f.c64[c] = pow2_mod(64, m);
    f.mf[c] = (float)m;
    f.invm[c] = 1.0f / (float)m;
    f.ch_plane0[c] = (int)planes.size();
    f.ch_nplanes[c] = (int)t.size();
    for (auto& tab : t) {
      for (int64_t v : tab) rho = std::max(rho, v < 0 ? -v : v);
      planes.push_back(tab);
    }
    const int64_t b = base, P0 = f.ch_plane0[c];
    struct G { int pa, pb; int64_t lam; };
    std::vector<G> gs;
    if (form == F_ONE) gs = {{0, 0, 1}};
    else if (form == F_SCHOOL3) gs = {{0, 0, 1}, {0, 1, b}, {1, 0, b}};
    else if (form == F_TOOM3) gs = {{0, 0, 1 - b}, {1, 1, b}, {2, 2, b * b - b}};
    else gs = {{0, 0, 1}, {0, 1, b}, {1, 0, b}, {1, 1, b * b}};
    f.ch_gemm0[c] = g;
    f.ch_ngemm[c] = (int)gs.size();
    for (const G& x : gs) {
      if (g >= OZ_MAX_FP_GEMMS) { delete p; return OZ_ERR_UNSUPPORTED; }
      f.g_pa[g] = (uint8_t)(P0 + x.pa);
      f.g_pb[g] = (uint8_t)(P0 + x.pb);
      f.g_ch[g] = (uint8_t)c;
      f.g_lam[g] = (float)mod_pos(x.lam, m);
      ++g;
    }
  }
  f.ngemm = g;
  f.nplanes = (int)planes.size();
  if (f.nplanes > OZ_MAX_FP_PLANES || g != cfg->Q) { delete p; return OZ_ERR_UNSUPPORTED; }
  p->gemms = g;
  p->Q = cfg->nch;
  // bits: the largest beta <= 64 with the window at k_hint, or the caller's
  U256 P = {};
  P.w[0] = 1;
  for (uint32_t m : moduli) u_mul(&P, m);
  int beta = bits;
  if (beta == 0) {
    for (beta = OZ_MAX_BITS_FP; beta >= 1; --beta)
      if (u_cmp(u_window(k_hint, beta), P) < 0) break;
    if (beta < 1) { delete p; return OZ_ERR_K_TOO_LARGE; }
  } else if (u_cmp(u_window(k_hint, beta), P) >= 0) {
    delete p;
    return OZ_ERR_K_TOO_LARGE;
  }
  p->bits = beta;
  if (!oz::fill_crt_tables(&p->tab, moduli.data(), cfg->nch, beta)) { delete p; return OZ_ERR_UNSUPPORTED; }
  for (int c = 0; c < cfg->nch; ++c) f.inv[c] = p->tab.inv[c];
  // K_max: the window (eq. ov-crtgen) and the accumulation cap 2^24 / rho^2 (eq. caps)
  int64_t lo = 0, hi = (int64_t)1 << 40;
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (u_cmp(u_window(mid, beta), P) < 0) lo = mid; else hi = mid;
  }
  const int64_t k_acc = rho > 0 ? (1ll << 24) / (rho * rho) : (int64_t)1 << 40;
  p->k_max = std::min(lo, k_acc);
  p->k_acc = k_acc;
  p->k_rec = lo;
  if (k_hint > p->k_max) { delete p; return OZ_ERR_K_TOO_LARGE; }
  // codes: host values and device code tables (plane p, class c at plane_off[p] + c)
  size_t total = 0;
  for (int q = 0; q < f.nplanes; ++q) {
    f.plane_off[q] = (uint32_t)total;
    f.plane_ch[q] = 0;
    total += planes[q].size();
  }
  for (int c = 0; c < cfg->nch; ++c)
    for (int q = 0; q < f.ch_nplanes[c]; ++q) f.plane_ch[f.ch_plane0[c] + q] = (uint32_t)c;
  p->h_values = new (std::nothrow) int16_t[total];
  if (!p->h_values) { delete p; return OZ_ERR_INVALID_ARG; }
  for (int q = 0; q < f.nplanes; ++q)
    for (size_t c = 0; c < planes[q].size(); ++c) p->h_values[f.plane_off[q] + c] = (int16_t)planes[q][c];
  p->values_len = total;
  // code words: per channel 2 m words, class i then the class of its negation
  std::vector<uint32_t> words;
  for (int c = 0; c < cfg->nch; ++c) {
    const uint32_t m = f.m[c];
    f.ch_woff[c] = (uint32_t)words.size();
    for (uint32_t i = 0; i < 2 * m; ++i) {
      const uint32_t cls = i < m ? i : (m - (i - m)) % m;
      uint32_t w = 0;
      for (int q = 0; q < f.ch_nplanes[c]; ++q)
        w |= (uint32_t)code_of.at(planes[f.ch_plane0[c] + q][cls]) << (8 * q);
      words.push_back(w);
    }
  }
  // Without a CUDA device the plan still describes the configuration
  // (oz_plan_info_fp); products on it then return OZ_ERR_CUDA.
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
    const size_t nb = words.size() * sizeof(uint32_t);
    if (cudaMalloc(&p->d_words, nb) != cudaSuccess ||
        cudaMemcpy(p->d_words, words.data(), nb, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      oz_plan_destroy(p);
      return OZ_ERR_CUDA;
    }
  } else {
    cudaGetLastError();
  }
  f.words = p->d_words;
  *out = p;
  return OZ_OK;
}

extern "C" oz_status oz_plan_info_fp(oz_plan plan, int* channels, int* gemms, int64_t* k_cfg, uint32_t* moduli,
                                     int* forms, int* bases, int* plane_count, int16_t* plane_values,
                                     size_t values_len) {
  if (!plan || !plan->is_fp) return OZ_ERR_INVALID_ARG;
  if (channels) *channels = plan->Q;
  if (gemms) *gemms = plan->gemms;
  if (k_cfg) *k_cfg = plan->fp_kcfg;
  if (plane_count) *plane_count = plan->fp.nplanes;
  for (int c = 0; c < plan->Q; ++c) {
    if (moduli) moduli[c] = plan->fp.m[c];
    if (forms) forms[c] = plan->fp_form[c];
    if (bases) bases[c] = plan->fp_base[c];
  }
  if (plane_values) {
    if (values_len < plan->values_len) return OZ_ERR_INVALID_ARG;
    memcpy(plane_values, plan->h_values, plan->values_len * sizeof(int16_t));
  }
  return OZ_OK;
}
