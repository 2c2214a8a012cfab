/*
 * oz_oracle.c -- plain CPU oracle for Ozaki-II emulated FP64 GEMM on the INT8
 * residue path.
 *
 * TEST INFRASTRUCTURE. This file exists only to check the CUDA path. Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * it. It shares no code, header, table or constant with the CUDA library, and
 * it includes nothing from it.
 *
 * It follows the paper's definitions step by step, with no blocking and no
 * fusion:
 *   1. Scale     (Sec. "Emulation Problem", eq. convert): per row of A and per
 *                column of B, the exponent e with max|x| in [2^(e-1), 2^e) by
 *                frexp; shift s = beta - e (s = 0 for a zero vector).
 *   2. Truncate  (eq. convert): x' = trunc(x * 2^s), an exact integer with
 *                |x'| < 2^beta.
 *   3. Reduce    (Sec. "Ozaki II"): the representative of x' mod m nearest zero,
 *                in [-floor(m/2), ceil(m/2) - 1].
 *   4. GEMMs     (Sec. "Forms and Channels", one-limb INT8 form, rank 1):
 *                W = U V in 64-bit integers, then W mod m in [0, m).
 *   5. CRT       (Sec. "Ozaki II"; window eq. ov-crtgen): Garner's mixed-radix
 *                algorithm in 256-bit integers, then the representative in
 *                [-P/2, P/2).
 *   6. Round     (Sec. "Emulation Problem"): C = fl(X * 2^-(s_i + t_j)), one
 *                round-to-nearest-even rounding done on the integer X, with
 *                gradual underflow and overflow to +-inf.
 * The exact reference product used for error reports is a fixed-point
 * (Kulisch) accumulator over the whole binary64 product range, so that
 * |C - AB| is formed exactly and rounded once.
 *
 * Every function returns 0 on success and a negative code on bad arguments or
 * non-finite input. Matrices are row-major: A[i*lda + h], B[h*ldb + j].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OZO_MAXQ 32   /* moduli; their product must also stay below 2^254 (moduli_ok) */

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------------- */
/* 256-bit unsigned integers, little-endian 64-bit words.                  */
/* ---------------------------------------------------------------------- */
typedef struct { uint64_t w[4]; } u256;

static void u256_set_u64(u256* x, uint64_t v) { x->w[0] = v; x->w[1] = x->w[2] = x->w[3] = 0; }

static void u256_mul_small_add(u256* x, uint64_t mul, uint64_t add) {
  /* x = x * mul + add  (mul, add < 2^32) */
  u128 carry = add;
  for (int i = 0; i < 4; ++i) {
    u128 t = (u128)x->w[i] * mul + carry;
    x->w[i] = (uint64_t)t;
    carry = t >> 64;
  }
}

static int u256_cmp(const u256* a, const u256* b) {
  for (int i = 3; i >= 0; --i) {
    if (a->w[i] < b->w[i]) return -1;
    if (a->w[i] > b->w[i]) return 1;
  }
  return 0;
}

static void u256_sub(u256* r, const u256* a, const u256* b) { /* r = a - b mod 2^256 */
  uint64_t borrow = 0;
  for (int i = 0; i < 4; ++i) {
    uint64_t ai = a->w[i], bi = b->w[i];
    uint64_t d = ai - bi - borrow;
    borrow = (ai < bi) || (ai == bi && borrow) ? 1 : 0;
    r->w[i] = d;
  }
}

static int u256_bitlen(const u256* x) {
  for (int i = 3; i >= 0; --i)
    if (x->w[i]) return 64 * i + 64 - __builtin_clzll(x->w[i]);
  return 0;
}

static int u256_bit(const u256* x, int k) { return (int)((x->w[k >> 6] >> (k & 63)) & 1); }

/* bits [lo, lo+n) of x as an integer, n <= 64 */
static uint64_t u256_bits(const u256* x, int lo, int n) {
  uint64_t v = 0;
  for (int k = n - 1; k >= 0; --k) v = (v << 1) | (uint64_t)u256_bit(x, lo + k);
  return v;
}

static int u256_any_below(const u256* x, int k) { /* any bit with index < k set */
  for (int b = 0; b < k; ++b) if (u256_bit(x, b)) return 1;
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Step 1: scale.                                                          */
/* ---------------------------------------------------------------------- */
static int scale_shift(const double* x, int64_t len, int64_t stride, int beta, int32_t* s) {
  double mx = 0.0;
  for (int64_t h = 0; h < len; ++h) {
    double v = x[h * stride];
    if (!isfinite(v)) return -2;
    if (fabs(v) > mx) mx = fabs(v);
  }
  if (mx == 0.0) { *s = 0; return 0; }
  int e;
  frexp(mx, &e);          /* mx in [2^(e-1), 2^e) */
  *s = beta - e;
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Step 2: truncate to an integer with |x'| < 2^beta (beta <= 120).        */
/* ---------------------------------------------------------------------- */
static __int128 truncate_scaled(double x, int32_t s) {
  double v = trunc(ldexp(x, s));     /* scaling by a power of two is exact   */
  return (__int128)v;                /* v is an integer below 2^beta         */
}

/* Step 3: representative nearest zero, in [-floor(m/2), ceil(m/2) - 1]. */
static int32_t balanced_residue(__int128 x, int32_t m) {
  __int128 r = x % m;
  if (r < 0) r += m;                         /* r in [0, m) */
  if (r >= (m + 1) / 2) r -= m;              /* ceil(m/2) */
  return (int32_t)r;
}

/* ---------------------------------------------------------------------- */
/* Step 5: CRT by Garner's algorithm.                                      */
/* ---------------------------------------------------------------------- */
static int64_t inverse_mod(int64_t a, int64_t m) { /* a^{-1} mod m by brute force; gcd(a, m) = 1 */
  a %= m; if (a < 0) a += m;
  for (int64_t x = 1; x < m; ++x) if ((a * x) % m == 1) return x;
  return m == 1 ? 0 : -1;
}

/* w[k] in [0, m_k). Output: magnitude |X| and its sign, X in [-P/2, P/2). */
static void crt_garner(const int32_t* w, const int32_t* mod, int Q, u256* mag, int* neg) {
  int64_t v[OZO_MAXQ] = {0};
  for (int k = 0; k < Q; ++k) {
    int64_t mk = mod[k];
    /* value of v[0] + m0 (v[1] + m1 (... v[k-1])) modulo mk, by Horner */
    int64_t acc = 0, prod = 1;
    for (int j = k - 1; j >= 0; --j) acc = (acc * mod[j] + v[j]) % mk;
    for (int j = 0; j < k; ++j) prod = (prod * mod[j]) % mk;
    int64_t d = ((int64_t)w[k] - acc) % mk; if (d < 0) d += mk;
    v[k] = (d * inverse_mod(prod, mk)) % mk;
  }
  /* X = v[0] + m0 (v[1] + m1 (... + m_{Q-2} v[Q-1])), in [0, P) */
  u256 X;
  u256_set_u64(&X, (uint64_t)v[Q - 1]);
  for (int k = Q - 2; k >= 0; --k) u256_mul_small_add(&X, (uint64_t)mod[k], (uint64_t)v[k]);

  u256 P; u256_set_u64(&P, 1);
  for (int k = 0; k < Q; ++k) u256_mul_small_add(&P, (uint64_t)mod[k], 0);
  u256 twoX = X; u256_mul_small_add(&twoX, 2, 0);
  if (u256_cmp(&twoX, &P) >= 0) { u256_sub(mag, &P, &X); *neg = 1; }   /* X - P < 0 */
  else { *mag = X; *neg = 0; }
  if (u256_bitlen(mag) == 0) *neg = 0;
}

/* The moduli fit the 256-bit CRT: 1 <= Q <= OZO_MAXQ, every m >= 2, and the
 * sum of their bit lengths (a bound on that of P) at most 254, so that 2X < 2^256. */
static int moduli_ok(const int32_t* mod, int Q) {
  if (Q < 1 || Q > OZO_MAXQ) return 0;
  int bits = 0;
  for (int k = 0; k < Q; ++k) {
    if (mod[k] < 2) return 0;
    int b = 0;
    for (uint32_t m = (uint32_t)mod[k]; m; m >>= 1) ++b;
    bits += b;
  }
  return bits <= 254;
}

/* ---------------------------------------------------------------------- */
/* Step 6: round (-1)^neg * mag * 2^e to binary64, nearest-even.           */
/* ---------------------------------------------------------------------- */
static double round_scaled(const u256* mag, int neg, int64_t e) {
  int L = u256_bitlen(mag);
  if (L == 0) return 0.0;
  int64_t E = (int64_t)L - 1 + e;             /* exponent of the leading bit */
  int64_t lsb = (E >= -1022) ? E - 52 : -1074; /* exponent of the last kept bit */
  int64_t sh = lsb - e;                        /* low bits of mag dropped */
  double r;
  if (sh <= 0) {
    r = ldexp((double)u256_bits(mag, 0, L), (int)e);  /* at most 53 bits: exact */
  } else {
    uint64_t q = (sh >= L) ? 0 : u256_bits(mag, (int)sh, (int)(L - sh));
    int half = (sh - 1 < L) ? u256_bit(mag, (int)(sh - 1)) : 0;
    int sticky = u256_any_below(mag, (int)((sh - 1 < L) ? sh - 1 : L));
    if (half && (sticky || (q & 1))) q += 1;
    if (lsb > 2000) return neg ? -INFINITY : INFINITY;
    r = ldexp((double)q, (int)lsb);                      /* exact or overflow to inf */
  }
  return neg ? -r : r;
}

/* ---------------------------------------------------------------------- */
/* Public entry points.                                                    */
/* ---------------------------------------------------------------------- */

/* Per-vector shifts. Vector v has elements X[v*s_vec + h*s_elem], h < len. */
int ozo_scale(const double* X, int64_t nvec, int64_t len, int64_t s_vec, int64_t s_elem,
              int beta, int32_t* s_out) {
  if (nvec < 0 || len < 0 || beta < 1 || beta > 120) return -1;
  for (int64_t v = 0; v < nvec; ++v)
    if (scale_shift(X + v * s_vec, len, s_elem, beta, &s_out[v])) return -2;
  return 0;
}

/* Balanced residue planes out[k][v][h] of trunc(X * 2^s[v]) modulo mod[k]. */
int ozo_residue_planes(const double* X, int64_t nvec, int64_t len, int64_t s_vec, int64_t s_elem,
                       const int32_t* s, const int32_t* mod, int Q, int16_t* out) {
  if (!moduli_ok(mod, Q)) return -1;
  for (int64_t v = 0; v < nvec; ++v)
    for (int64_t h = 0; h < len; ++h) {
      double x = X[v * s_vec + h * s_elem];
      if (!isfinite(x)) return -2;
      __int128 xp = truncate_scaled(x, s[v]);
      for (int k = 0; k < Q; ++k) out[((int64_t)k * nvec + v) * len + h] = (int16_t)balanced_residue(xp, mod[k]);
    }
  return 0;
}

/* Full emulated product C = fl(diag(mu)^-1 (A'B') diag(nu)^-1), every entry.
 * Optional outputs (may be NULL): w_out[k][i][j] = (A'B')_ij mod m_k in [0, m_k),
 * s_out[M], t_out[N]. */
int ozo_dgemm(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
              const double* B, int64_t ldb, const int32_t* mod, int Q, int beta,
              double* C, int64_t ldc, uint16_t* w_out, int32_t* s_out, int32_t* t_out) {
  if (M < 0 || N < 0 || K < 0 || !moduli_ok(mod, Q) || beta < 1 || beta > 120) return -1;
  int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M + 1));
  int32_t* t = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N + 1));
  int16_t* U = (int16_t*)malloc(sizeof(int16_t) * (size_t)(Q * M * K + 1));
  int16_t* V = (int16_t*)malloc(sizeof(int16_t) * (size_t)(Q * N * K + 1)); /* V[k][j][h] */
  int32_t* W = (int32_t*)malloc(sizeof(int32_t) * (size_t)(Q * M * N + 1));
  int rc = 0;
  if (!s || !t || !U || !V || !W) { rc = -3; goto done; }
  /* 1-3: scale, truncate, reduce */
  if (ozo_scale(A, M, K, lda, 1, beta, s)) { rc = -2; goto done; }
  if (ozo_scale(B, N, K, 1, ldb, beta, t)) { rc = -2; goto done; }
  if (ozo_residue_planes(A, M, K, lda, 1, s, mod, Q, U)) { rc = -2; goto done; }
  if (ozo_residue_planes(B, N, K, 1, ldb, t, mod, Q, V)) { rc = -2; goto done; }
  /* 4: one integer GEMM per modulus, then W mod m in [0, m) */
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < Q; ++k)
    for (int64_t i = 0; i < M; ++i)
      for (int64_t j = 0; j < N; ++j) {
        const int16_t* u = U + ((int64_t)k * M + i) * K;
        const int16_t* v = V + ((int64_t)k * N + j) * K;
        int64_t acc = 0;
        for (int64_t h = 0; h < K; ++h) acc += (int64_t)u[h] * (int64_t)v[h];
        int64_t r = acc % mod[k]; if (r < 0) r += mod[k];
        W[((int64_t)k * M + i) * N + j] = (int32_t)r;
      }
  /* 5-6: CRT and one rounding */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i)
    for (int64_t j = 0; j < N; ++j) {
      int32_t w[OZO_MAXQ];
      for (int k = 0; k < Q; ++k) w[k] = W[((int64_t)k * M + i) * N + j];
      u256 mag; int neg;
      crt_garner(w, mod, Q, &mag, &neg);
      C[i * ldc + j] = round_scaled(&mag, neg, -((int64_t)s[i] + t[j]));
    }
  if (w_out)
    for (int64_t x = 0; x < (int64_t)Q * M * N; ++x) w_out[x] = (uint16_t)W[x];
  if (s_out) memcpy(s_out, s, sizeof(int32_t) * (size_t)M);
  if (t_out) memcpy(t_out, t, sizeof(int32_t) * (size_t)N);
done:
  free(s); free(t); free(U); free(V); free(W);
  return rc;
}

/* Selected entries (rows[e], cols[e]) of the same product, each computed on its
 * own from row rows[e] of A and column cols[e] of B. Optional x_out: the CRT
 * result X as four 64-bit words of a two's-complement 256-bit integer. */
int ozo_dgemm_entries(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                      const double* B, int64_t ldb, const int32_t* mod, int Q, int beta,
                      int64_t n_entries, const int64_t* rows, const int64_t* cols,
                      double* out, uint64_t* x_out) {
  if (M < 0 || N < 0 || K < 0 || !moduli_ok(mod, Q) || beta < 1 || beta > 120) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
  for (int64_t e = 0; e < n_entries; ++e) {
    int64_t i = rows[e], j = cols[e];
    if (i < 0 || i >= M || j < 0 || j >= N) { bad |= 1; continue; }
    int32_t si, tj;
    if (scale_shift(A + i * lda, K, 1, beta, &si) || scale_shift(B + j, K, ldb, beta, &tj)) { bad |= 2; continue; }
    int32_t w[OZO_MAXQ];
    for (int k = 0; k < Q; ++k) {
      int64_t acc = 0;
      for (int64_t h = 0; h < K; ++h) {
        int32_t ra = balanced_residue(truncate_scaled(A[i * lda + h], si), mod[k]);
        int32_t rb = balanced_residue(truncate_scaled(B[h * ldb + j], tj), mod[k]);
        acc += (int64_t)ra * rb;
      }
      int64_t r = acc % mod[k]; if (r < 0) r += mod[k];
      w[k] = (int32_t)r;
    }
    u256 mag; int neg;
    crt_garner(w, mod, Q, &mag, &neg);
    out[e] = round_scaled(&mag, neg, -((int64_t)si + tj));
    if (x_out) {
      u256 X = mag;
      if (neg) { u256 z; u256_set_u64(&z, 0); u256_sub(&X, &z, &mag); }
      for (int q = 0; q < 4; ++q) x_out[4 * e + q] = X.w[q];
    }
  }
  return bad ? -1 - bad : 0;
}

/* CRT alone: residues w[e][k] in [0, m_k) -> X as two's-complement 256-bit words. */
int ozo_crt(int64_t n, const int32_t* w, const int32_t* mod, int Q, uint64_t* x_out) {
  if (!moduli_ok(mod, Q)) return -1;
  for (int64_t e = 0; e < n; ++e) {
    u256 mag; int neg;
    crt_garner(w + e * Q, mod, Q, &mag, &neg);
    u256 X = mag;
    if (neg) { u256 z; u256_set_u64(&z, 0); u256_sub(&X, &z, &mag); }
    for (int q = 0; q < 4; ++q) x_out[4 * e + q] = X.w[q];
  }
  return 0;
}

/* Rounding alone: value = X * 2^e with X two's-complement 256-bit. */
int ozo_round(int64_t n, const uint64_t* x, const int64_t* e, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    u256 X; memcpy(X.w, x + 4 * i, sizeof X.w);
    int neg = (int)(X.w[3] >> 63);
    u256 mag = X;
    if (neg) { u256 z; u256_set_u64(&z, 0); u256_sub(&mag, &z, &X); }
    out[i] = round_scaled(&mag, neg, e[i]);
  }
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Exact reference: a fixed-point accumulator covering every product of    */
/* two finite doubles (bits 2^-2148 .. 2^2048) plus headroom for the sum.  */
/* ---------------------------------------------------------------------- */
#define KW 72                   /* 72 * 64 = 4608 bits */
#define KBIAS 2200              /* bit index of 2^0 */
typedef struct { uint64_t w[KW]; } kacc;

static void kacc_add_u128(kacc* a, u128 v, int bit, int negate) {
  /* add (or subtract) v * 2^(bit - KBIAS) */
  int wi = bit >> 6, off = bit & 63;
  uint64_t part[3];
  part[0] = (uint64_t)v << off;
  part[1] = off ? (uint64_t)(v >> (64 - off)) : (uint64_t)(v >> 64);
  part[2] = off ? (uint64_t)((v >> 64) >> (64 - off)) : 0;
  if (!negate) {
    uint64_t carry = 0;
    for (int q = 0; wi + q < KW; ++q) {
      uint64_t add = (q < 3) ? part[q] : 0;
      if (q >= 3 && !carry) break;
      uint64_t s1 = a->w[wi + q] + add; uint64_t c1 = s1 < add;
      uint64_t s2 = s1 + carry; uint64_t c2 = s2 < carry;
      a->w[wi + q] = s2; carry = c1 | c2;
    }
  } else {
    uint64_t borrow = 0;
    for (int q = 0; wi + q < KW; ++q) {
      uint64_t sub = (q < 3) ? part[q] : 0;
      if (q >= 3 && !borrow) break;
      uint64_t old = a->w[wi + q];
      uint64_t d1 = old - sub; uint64_t b1 = old < sub;
      uint64_t d2 = d1 - borrow; uint64_t b2 = d1 < borrow;
      a->w[wi + q] = d2; borrow = b1 | b2;
    }
  }
}

/* double -> (sign, integer significand, exponent) with x = sig * 2^ex */
static void decompose(double x, int* neg, uint64_t* sig, int* ex) {
  uint64_t b; memcpy(&b, &x, 8);
  *neg = (int)(b >> 63);
  int be = (int)((b >> 52) & 0x7ff);
  uint64_t f = b & ((1ULL << 52) - 1);
  if (be == 0) { *sig = f; *ex = -1074; }
  else { *sig = f | (1ULL << 52); *ex = be - 1075; }
}

static void kacc_add_product(kacc* a, double x, double y) {
  int nx, ny, ex, ey; uint64_t sx, sy;
  decompose(x, &nx, &sx, &ex); decompose(y, &ny, &sy, &ey);
  if (!sx || !sy) return;
  kacc_add_u128(a, (u128)sx * sy, ex + ey + KBIAS, nx ^ ny);
}

static void kacc_add_double(kacc* a, double x, int negate) {
  int nx, ex; uint64_t sx;
  decompose(x, &nx, &sx, &ex);
  if (!sx) return;
  kacc_add_u128(a, (u128)sx, ex + KBIAS, nx ^ negate);
}

/* |value| rounded to nearest double (value = accumulator, two's complement) */
static double kacc_abs_to_double(const kacc* a) {
  kacc m = *a;
  if (m.w[KW - 1] >> 63) { /* negate */
    uint64_t carry = 1;
    for (int q = 0; q < KW; ++q) { uint64_t v = ~m.w[q] + carry; carry = (carry && v == 0); m.w[q] = v; }
  }
  int top = -1;
  for (int q = KW - 1; q >= 0; --q) if (m.w[q]) { top = 64 * q + 63 - __builtin_clzll(m.w[q]); break; }
  if (top < 0) return 0.0;
  /* round the magnitude to 53 bits (the values here are far from the subnormal range) */
  int lo = top - 52 > 0 ? top - 52 : 0;
  uint64_t q = 0;
  for (int b = top; b >= lo; --b) q = (q << 1) | ((m.w[b >> 6] >> (b & 63)) & 1);
  if (lo > 0) {
    int half = (int)((m.w[(lo - 1) >> 6] >> ((lo - 1) & 63)) & 1);
    int sticky = 0;
    for (int b = 0; b < lo - 1 && !sticky; ++b) sticky = (int)((m.w[b >> 6] >> (b & 63)) & 1);
    if (half && (sticky || (q & 1))) q += 1;
  }
  return ldexp((double)q, lo - KBIAS);
}

/* For each selected entry: err_out = |C_ij - (AB)_ij|, the exact difference
 * rounded once (C may be NULL, giving |(AB)_ij|), and absprod_out = (|A||B|)_ij
 * summed in binary64. */
int ozo_exact_error(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                    const double* B, int64_t ldb, const double* C, int64_t ldc,
                    int64_t n_entries, const int64_t* rows, const int64_t* cols,
                    double* err_out, double* absprod_out) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
  for (int64_t e = 0; e < n_entries; ++e) {
    int64_t i = rows[e], j = cols[e];
    if (i < 0 || i >= M || j < 0 || j >= N) { bad = 1; continue; }
    kacc* acc = (kacc*)calloc(1, sizeof(kacc));
    double ab = 0.0;
    for (int64_t h = 0; h < K; ++h) {
      double x = A[i * lda + h], y = B[h * ldb + j];
      kacc_add_product(acc, x, y);
      ab += fabs(x) * fabs(y);
    }
    if (C) kacc_add_double(acc, C[i * ldc + j], 1);   /* acc = AB - C */
    err_out[e] = kacc_abs_to_double(acc);
    absprod_out[e] = ab;
    free(acc);
  }
  return bad ? -1 : 0;
}
