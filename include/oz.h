/*
 * oz.h -- C ABI of the GB300 (sm_103a) Ozaki-II emulated FP64 GEMM library.
 *
 * The library computes C = op(A) op(B) for FP64 row-major matrices by the
 * Ozaki-II scheme on the INT8 alphabet (Sec. "Ozaki II", Sec. "INT4 and INT8"),
 * or on a low-precision float alphabet (oz_plan_create_fp):
 *   1. Scale      one power-of-two shift per row of op(A) and per column of
 *                 op(B) (eq. convert);
 *   2. Reduce     truncate to integers below 2^bits and write the balanced
 *                 residue planes modulo each of Q pairwise-coprime moduli
 *                 (Sec. "Structure", phase 2);
 *   3. GEMMs      one exact integer product per modulus (phase 3);
 *   4. Epilogue   each product reduced modulo its modulus (phase 4, order R>C);
 *   5. Reconstruct CRT back to the integer product, one rounding to binary64,
 *                 unscale (phase 5).
 *
 * Conventions for every call below:
 *   - Matrices are row-major. op(X) = X if trans == 0, X^T if trans == 1.
 *     A is stored m x k (trans_a = 0) or k x m (trans_a = 1) with leading
 *     dimension lda >= its column count; likewise B (k x n or n x k), C (m x n).
 *   - A, B, C and the workspace are DEVICE pointers owned by the caller
 *     (oz_dgemm_host takes HOST A, B, C). The library never allocates device
 *     memory during a product call. An INT8 plan owns a small table of
 *     constants in host memory; a float-format plan also owns a small device
 *     table of codes; a grouped product (oz_group_create) owns a few streams
 *     and events; oz_dgemm_host keeps a pool of events per host thread and
 *     device, created on first use and reused by every later call of that
 *     thread (destroyed when the thread exits).
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream). Nothing synchronises the host
 *     except oz_query_status.
 *   - Errors come back as oz_status codes; the library never exits, aborts or
 *     traps. Argument errors are detected on the host before any launch.
 *     Non-finite input is detected on the device, leaves C unspecified, and is
 *     reported by the next oz_query_status on the same workspace.
 *   - A plan is immutable after creation and may be shared by threads; a
 *     workspace must not be used by two calls that overlap on the GPU. The
 *     only per-thread state is oz_dgemm_host's event pool.
 */
#ifndef OZ_H_
#define OZ_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OZ_API __attribute__((visibility("default")))
#else
#define OZ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define OZ_MAX_MODULI 20   /* largest Q the library accepts */
#define OZ_MIN_MODULI 9    /* smallest Q the library accepts */
#define OZ_MAX_BITS 80     /* largest bit budget beta (|A'| < 2^beta) of an INT8 plan */
#define OZ_MAX_BITS_FP 72  /* largest bit budget of a float-format plan (widened configurations) */
#define OZ_MAX_CHANNELS 32 /* most channels a float-format configuration has */

typedef enum {
  OZ_OK = 0,
  OZ_ERR_INVALID_ARG = 1,   /* bad size, leading dimension, pointer or flag */
  OZ_ERR_K_TOO_LARGE = 2,   /* k above the plan's K_max (eq. caps) */
  OZ_ERR_WORKSPACE = 3,     /* workspace NULL or shorter than oz_workspace_bytes */
  OZ_ERR_NONFINITE = 4,     /* NaN or Inf in A or B (reported by oz_query_status) */
  OZ_ERR_UNSUPPORTED = 5,   /* configuration or engine not available */
  OZ_ERR_CUDA = 6           /* a CUDA runtime call or launch failed */
} oz_status;

typedef enum {
  OZ_ENGINE_AUTO = 0,  /* the fastest engine available for the plan */
  OZ_ENGINE_IMMA = 1,  /* INT8 residue planes, warp-level mma.sync s8 -> s32 */
  OZ_ENGINE_TC = 2,    /* BF16-held residue planes, tcgen05.mma into TMEM, CTA pairs
                          (cta_group::2) on 256 x 256 output tiles */
  OZ_ENGINE_FP = 3,    /* float-format planes (oz_plan_create_fp), tcgen05.mma kind::f8f6f4 */
  OZ_ENGINE_TC1 = 4    /* as OZ_ENGINE_TC with one CTA per 128 x 256 tile (same bits) */
} oz_engine;

/* Low-precision float formats (OCP): FP8 E4M3 and E5M2, FP6 E2M3 and E3M2, FP4 E2M1. */
typedef enum {
  OZ_FMT_E4M3 = 1,
  OZ_FMT_E2M3 = 2,
  OZ_FMT_E3M2 = 3,
  OZ_FMT_E2M1 = 4,
  OZ_FMT_E5M2 = 5
} oz_format;

typedef struct oz_plan_s* oz_plan;

/*
 * oz_plan_create -- build an INT8 configuration (Sec. "Forms and Channels":
 * one one-limb channel per modulus; Sec. "INT4 and INT8": moduli up to 239).
 *   out          receives the plan (caller frees it with oz_plan_destroy).
 *   num_moduli   Q in [OZ_MIN_MODULI, OZ_MAX_MODULI]; 0 picks the least Q whose
 *                modulus product satisfies the window P > 2 K (2^53 - 1)^2
 *                (eq. ov-crtgen) at K = k_hint.
 *                The moduli are the Q pairwise-coprime integers <= 239 with the
 *                largest product (for Q >= 9 these are prefixes of one list).
 *   bits         beta, the bits kept per row/column maximum (eq. convert uses
 *                53). 0 picks the largest beta <= OZ_MAX_BITS with
 *                2 k_hint (2^beta - 1)^2 < P. Above 53 the operands are
 *                widened (Sec. "Not True Emulation of DGEMM", Example
 *                widened): rows and columns whose entries span at most
 *                2^(beta - 53) convert without loss, and the product is then
 *                fl(AB) exactly.
 *   k_hint       the largest inner dimension the caller intends to use (>= 1).
 *                The plan is refused with OZ_ERR_K_TOO_LARGE if the window
 *                does not hold at k_hint.
 *   engine       an oz_engine value.
 * Returns OZ_OK, OZ_ERR_INVALID_ARG, OZ_ERR_K_TOO_LARGE or OZ_ERR_UNSUPPORTED.
 */
OZ_API oz_status oz_plan_create(oz_plan* out, int num_moduli, int bits, int64_t k_hint, int engine);

/*
 * oz_plan_info -- report a plan: q = Q, bits = beta, k_max = K_max (the
 * minimum of the reconstruction and accumulation caps of eq. caps at this
 * beta), engine = the engine a call will use, moduli[0..Q-1] (decreasing).
 * Any output pointer may be NULL. moduli, if given, must hold OZ_MAX_MODULI.
 */
OZ_API oz_status oz_plan_info(oz_plan plan, int* q, int* bits, int64_t* k_max, int* engine, uint32_t* moduli);

/*
 * oz_plan_create_fp -- a configuration over a low-precision float alphabet
 * (Sec. "Forms and Channels", Sec. "Instantiation"): pairwise-coprime channels,
 * each a modulus with a one-limb, schoolbook or Toom (Karatsuba) form whose
 * tables take values in the format's alphabet S (its finite values scaled to
 * integers), found by an exact least-GEMM-count search (Sec. "Solving the
 * Program") and frozen in the library: for inner dimensions K_cfg = 8192,
 * 16384 and 65536 at beta = 53, and widened for K_cfg = 16384 at beta = 69
 * (Example ex:widened: E2M1 78 GEMMs, E4M3 / E2M3 39). The plan takes the
 * beta = 53 configuration of the least K_cfg >= k_hint whose window holds
 * `bits`, else the widened one. Every plane value is at most
 * floor(sqrt(2^24/K_cfg)), so each GEMM's FP32 accumulator is exact (eq.
 * ov-accgen).
 *   format   an oz_format value.
 *   k_hint   the largest inner dimension the caller intends to use.
 *   bits     as for oz_plan_create, up to OZ_MAX_BITS_FP (0: the largest beta
 *            the beta = 53 configuration's window allows, 53 to 55).
 * Returns OZ_ERR_K_TOO_LARGE when no configuration holds the window at
 * (k_hint, bits).
 * The plan owns a small device table of codes (allocated here on the current
 * device, freed by oz_plan_destroy). Without a CUDA device the plan is still
 * made and describes the configuration (oz_plan_info_fp), but products on it
 * return OZ_ERR_CUDA. Products run through oz_dgemm, oz_dgemm_batched,
 * oz_dgemm_host and the phase entry points as for INT8 plans; their residues
 * Y are uint16, one per entry and channel.
 */
OZ_API oz_status oz_plan_create_fp(oz_plan* out, int format, int64_t k_hint, int bits);

/*
 * oz_plan_info_fp -- describe a float-format plan: channel count, GEMM count
 * (the paper's Q), K_cfg, per channel its modulus, form (1 one limb,
 * 2 schoolbook with m | b^2, 3 Toom at {0, 1, inf}, 4 schoolbook) and base, the
 * plane count, and (if plane_values is given, values_len entries long) the
 * plane value tables: plane p (channels in order, planes of a channel in the
 * order a0 | a0, a1 | a0, a0 + a1, a1) holds m_c scaled alphabet values, one
 * per class. moduli, forms and bases, if given, must hold OZ_MAX_CHANNELS
 * entries. Any output pointer may be NULL.
 */
OZ_API oz_status oz_plan_info_fp(oz_plan plan, int* channels, int* gemms, int64_t* k_cfg, uint32_t* moduli,
                                 int* forms, int* bases, int* plane_count, int16_t* plane_values,
                                 size_t values_len);

/*
 * oz_plan_caps -- the two caps of eq. caps separately: k_acc, the largest
 * inner dimension one accumulation may take (INT32 accumulators on the IMMA
 * engine, FP32 accumulators of float-format plans; the TC engine drains its
 * FP32 slabs itself and has none below 2^31), and k_rec, the largest K the
 * CRT window admits at the plan's beta (eq. ov-crtgen). K_max of
 * oz_plan_info is their minimum; a blocked call (oz_dgemm_blocked) takes any
 * K <= k_rec in slabs of at most k_acc. Either output may be NULL.
 */
OZ_API oz_status oz_plan_caps(oz_plan plan, int64_t* k_acc, int64_t* k_rec);

/* Release a plan (NULL is accepted). */
OZ_API void oz_plan_destroy(oz_plan plan);

/*
 * oz_workspace_bytes -- device workspace a product of this shape needs: the
 * shifts, the residue planes of both operands (planes x (m_pad + n_pad) rows
 * of oz_plane_geometry's row bytes), the residues of the product (Q x m
 * rows of n entries, each row padded to a multiple of 16 bytes so that the
 * GEMM epilogue stores whole 16-byte runs; uint8, or uint16 per channel for
 * float-format plans) and, for the IMMA engine's int8 planes, B^T (n x k
 * doubles: with trans_b = 0 the columns of B are split as rows of its
 * transpose; the bf16 planes of the TC engines are split from B's columns in
 * place). Returns 0 for an invalid plan or shape.
 */
OZ_API size_t oz_workspace_bytes(oz_plan plan, int64_t m, int64_t n, int64_t k);

/*
 * oz_workspace_layout -- where oz_dgemm puts each part of its workspace, so
 * that the phase entry points below can run the same product step by step.
 * out[0..9] receives byte offsets of: flag (int32[4]), s (int32[m]),
 * t (int32[n]), colmax (uint64[max(m, n)]), U planes, V planes, Y residues
 * (Q x m rows, row pitch n rounded up to 16 bytes; the phase entry points
 * below take and give row pitch n, which fits in the same region), then m_pad,
 * n_pad, k_pad (entries, not bytes), and out[10] the byte offset of B^T
 * (n x k doubles; an IMMA-engine oz_dgemm with trans_b = 0 transposes B there
 * and splits its columns as rows; empty for the TC engines, which split B's
 * columns with oz_split(contiguous = 0), and for float-format plans). out
 * must hold 11 entries.
 */
OZ_API oz_status oz_workspace_layout(oz_plan plan, int64_t m, int64_t n, int64_t k, int64_t* out);

/*
 * oz_dgemm -- C = op(A) op(B) (Sec. "Emulation Problem"; five phases of
 * Sec. "Structure"). No alpha/beta: C is overwritten.
 *   m, n, k >= 0 (an empty product writes nothing; k = 0 writes zeros).
 *   k must not exceed the plan's K_max (OZ_ERR_K_TOO_LARGE).
 *   workspace: device memory of at least oz_workspace_bytes(plan, m, n, k)
 *   bytes, 256-byte aligned.
 * The result is C_ij = fl(2^-(s_i + t_j) (A'B')_ij), one round-to-nearest-even
 * rounding of the exact integer product of the truncated operands, with
 * gradual underflow and overflow to +-inf.
 */
OZ_API oz_status oz_dgemm(oz_plan plan, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k,
                   const double* A, int64_t lda, const double* B, int64_t ldb,
                   double* C, int64_t ldc, void* workspace, size_t workspace_bytes, void* stream);

/*
 * oz_query_status -- wait for the stream, then report OZ_ERR_NONFINITE if the
 * last oz_dgemm on this workspace met a NaN or Inf, OZ_ERR_CUDA if the stream
 * has a CUDA error or a bounded device wait of that call ran out, else OZ_OK.
 */
OZ_API oz_status oz_query_status(void* workspace, void* stream);

/* ---- Blocked call: the inner dimension in slabs (Sec. "Slabs"). ---- */

/*
 * oz_blocked_workspace_bytes -- device workspace of a blocked call: the
 * workspace of one product with inner dimension k_slab (the planes of one
 * slab of each operand) plus nothing else; the residues Y cover the whole
 * output as in oz_workspace_bytes. Returns 0 for an invalid plan or shape.
 */
OZ_API size_t oz_blocked_workspace_bytes(oz_plan plan, int64_t m, int64_t n, int64_t k_slab);

/*
 * oz_dgemm_blocked -- the product of oz_dgemm, with the inner dimension cut
 * into slabs of k_slab terms (the last one shorter), each accumulated on its
 * own and added into a running residue (Sec. "Slabs"):
 *   1. the shifts s, t are taken over the whole of each row of op(A) and
 *      column of op(B) (eq. convert), so the truncated operands A', B' are
 *      those of the unblocked call;
 *   2. per slab, the residue planes of that slab's columns of op(A) and rows
 *      of op(B) are formed, and each modulus' GEMM epilogue adds the slab's
 *      CRT digit into the digits of the earlier slabs, modulo m (digits are
 *      linear in W, and W is the sum of the slabs' products);
 *   3. one Reconstruct after the last slab.
 * The result is therefore bit for bit that of oz_dgemm whenever both apply.
 * The call serves K above the accumulation cap (k <= k_rec, k_slab <= k_acc
 * of oz_plan_caps, else OZ_ERR_K_TOO_LARGE) and operands whose planes for the
 * whole K would not fit in memory: the workspace holds one slab's planes,
 * oz_blocked_workspace_bytes(plan, m, n, k_slab) bytes, 256-byte aligned.
 * Other arguments, errors and asynchrony as for oz_dgemm; k_slab >= 1.
 */
OZ_API oz_status oz_dgemm_blocked(oz_plan plan, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k,
                                  int64_t k_slab, const double* A, int64_t lda, const double* B, int64_t ldb,
                                  double* C, int64_t ldc, void* workspace, size_t workspace_bytes, void* stream);

/* ---- Host-resident operands with the copies overlapped. ---- */

/*
 * oz_host_workspace_bytes / oz_dgemm_host -- C = A B (row-major, no
 * transposes) with A, B and C in HOST memory (pinned memory lets the copies
 * overlap; pageable memory works but serialises them). The product is the one
 * oz_dgemm computes. C is cut into blocks of rows_per_chunk rows by
 * cols_per_chunk columns (0 picks about a quarter of m or n, a multiple of
 * 256). The copy stream brings the first row chunk of A, then B column chunk
 * by column chunk, then the other row chunks of A; each column chunk of B is
 * split once, when it has arrived, and each row chunk of A when its block row
 * starts; each block's GEMMs and reconstruct run on `stream` and its copy back
 * on stream_d2h, under the next block's work. The first GEMMs thus wait for
 * one chunk of each operand only. When the call returns the work is queued;
 * once `stream` has finished, C holds the result (the copy streams join it
 * through events). The three streams must be distinct; the workspace (device,
 * 256-byte aligned) holds B, two A chunks, two C blocks, the planes of one A
 * chunk and of all of B, and the residues of one block row. Non-finite input
 * is reported by oz_query_status on this workspace.
 */
OZ_API size_t oz_host_workspace_bytes(oz_plan plan, int64_t m, int64_t n, int64_t k, int64_t rows_per_chunk,
                                      int64_t cols_per_chunk);
OZ_API oz_status oz_dgemm_host(oz_plan plan, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                               const double* B, int64_t ldb, double* C, int64_t ldc, int64_t rows_per_chunk,
                               int64_t cols_per_chunk, void* workspace, size_t workspace_bytes, void* stream,
                               void* stream_h2d, void* stream_d2h);

/* ---- Many products of uneven shapes in one call. ---- */

/*
 * oz_batched_workspace_bytes / oz_dgemm_batched -- count independent products
 * C_i = op(A_i) op(B_i) (the problem of Sec. "Emulation Problem" for each i),
 * each with its own plan (plans[i]; one plan may serve several problems) and
 * its own sizes mnk[3i..3i+2] = (m_i, n_i, k_i).
 * Scheduling: the problems go to the nstreams caller-owned streams (streams[0]
 * is the origin; the others join it through events, so the whole batch can be
 * captured into one CUDA graph on streams[0]), each problem to the stream with
 * the least estimated work so far, largest problems first. The problems of one
 * stream run one after another and share that stream's slice of the
 * workspace, so the workspace is nstreams times the largest single-problem
 * workspace of any stream's problems; oz_batched_workspace_bytes reports it
 * (0 for invalid arguments). With nstreams > 1, OZ_ENGINE_TC plans run their
 * GEMMs with one CTA per tile (as OZ_ENGINE_TC1): CTA-pair GEMMs of products
 * running at once on several streams were seen to stall one another.
 * Arrays (plans, mnk, trans, pointer and leading-dimension arrays, streams)
 * are host arrays of length count (streams: nstreams); the matrices and the
 * workspace are device memory. trans may be NULL (no transposes), else
 * trans[2i], trans[2i+1] = trans_a, trans_b of problem i.
 * Errors: as oz_dgemm, checked for every problem before anything launches.
 */
OZ_API size_t oz_batched_workspace_bytes(int count, const oz_plan* plans, const int64_t* mnk, int nstreams);
OZ_API oz_status oz_dgemm_batched(int count, const oz_plan* plans, const int64_t* mnk, const int* trans,
                                  const double* const* A, const int64_t* lda, const double* const* B,
                                  const int64_t* ldb, double* const* C, const int64_t* ldc, void* workspace,
                                  size_t workspace_bytes, void* const* streams, int nstreams);

/* ---- The phases on their own, for parity checks and profiling. ---- */

/*
 * oz_plane_geometry -- how a plan lays out the residue planes the phase entry
 * points exchange: k_align = the multiple k_pad must be (128 entries; 256 for
 * E2M1 plans), row_bytes = bytes of one plane row of k_pad entries: k_pad for
 * IMMA (int8) and for float formats other than E2M1 (one 8-bit code per entry,
 * or 6-bit codes packed 16 to a 16-byte chunk whose last 4 bytes are zero),
 * 2 k_pad for TC (bf16), k_pad / 2 for E2M1 (two 4-bit codes per byte, the
 * even entry in the low half). A plane of nvec_pad rows is nvec_pad row_bytes
 * bytes. k_pad must be a multiple of k_align. Outputs may be NULL.
 */
OZ_API oz_status oz_plane_geometry(oz_plan plan, int64_t k_pad, int64_t* k_align, int64_t* row_bytes);

/*
 * oz_split -- phases 1 and 2 for one operand (Sec. "Structure").
 * The operand is viewed as nvec vectors of len entries: vector v, entry h is
 * X[v*ld + h] if contiguous != 0 (rows of a row-major matrix: A, or B^T), else
 * X[h*ld + v] (columns: B, or A^T). Writes:
 *   shifts[v]  = beta - e_v, e_v the exponent with max_h |x| in [2^(e-1), 2^e)
 *                (0 for a zero vector), int32, device;
 *   planes     = Q planes of nvec_pad x k_pad entries, plane q row v entry h =
 *                the balanced residue of trunc(x 2^shift) modulo m_q in
 *                [-floor(m/2), ceil(m/2) - 1]; int8 for IMMA, bf16 for TC;
 *                padding (v >= nvec or h >= len) is zero. For a float-format
 *                plan: its plane count (oz_plan_info_fp) of codes of the
 *                form's plane values of the class of trunc(x 2^shift) modulo
 *                each channel's modulus, laid out as oz_plane_geometry states.
 * nvec_pad must be a multiple of 256 and k_pad of oz_plane_geometry's k_align.
 *   flag       (may be NULL) device int32; bit 0 set if an entry is not finite.
 *   colmax     device scratch of nvec uint64 words, used when contiguous == 0
 *              (may be NULL otherwise).
 * nvec_pad >= nvec and k_pad >= len.
 */
OZ_API oz_status oz_split(oz_plan plan, int contiguous, int64_t nvec, int64_t len, const double* X, int64_t ld,
                   int64_t nvec_pad, int64_t k_pad, int32_t* shifts, void* planes, int32_t* flag,
                   uint64_t* colmax, void* stream);

/*
 * oz_transpose -- Y = X^T for X of rows x cols doubles (row pitch ld >=
 * cols), Y of cols x rows (row pitch rows): the step an IMMA-engine oz_dgemm
 * takes before splitting the columns of B as contiguous rows (then
 * oz_split(contiguous = 1) on Y is that split). Device pointers, 8-byte
 * aligned; asynchronous on the stream.
 */
OZ_API oz_status oz_transpose(int64_t rows, int64_t cols, const double* X, int64_t ld, double* Y, void* stream);

/*
 * oz_residue_gemm -- phases 3 and 4: for each modulus q,
 * W_q = U_q V_q^T (exact, INT32) and
 *   raw == 0: Y[q][i][j] = (W mod m_q) * ((P/m_q)^-1 mod m_q) mod m_q, the CRT
 *             digit the reconstruct phase consumes;
 *   raw != 0: Y[q][i][j] = W mod m_q in [0, m_q) (the paper's epilogue value).
 * U, V: planes from oz_split (m_pad x k_pad and n_pad x k_pad per modulus),
 * Y: uint8, Q planes of m x n (row pitch n); uint16 for float-format plans,
 * one plane per channel, the residue folded over the channel's GEMMs
 * (sum_g lambda_g W_g mod m, order R>C). Device pointers.
 * flag (may be NULL): device int32; the TC engine sets bit 1 if one of its
 * bounded waits ran out (the kernel then stops early and Y is unspecified).
 * The TC engine needs U and V 128-byte aligned.
 */
OZ_API oz_status oz_residue_gemm(oz_plan plan, int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                          const void* U, const void* V, uint8_t* Y, int raw, int32_t* flag, void* stream);

/*
 * oz_reconstruct -- phase 5 (Sec. "Around the GEMMs", Reconstruct): from the
 * CRT digits Y (raw == 0 output of oz_residue_gemm) and the shifts s[m], t[n],
 * C_ij = fl(2^-(s_i + t_j) X_ij), X_ij the integer in [-P/2, P/2) congruent
 * to the digits. C row pitch ldc >= n. Device pointers.
 */
OZ_API oz_status oz_reconstruct(oz_plan plan, int64_t m, int64_t n, const uint8_t* Y, const int32_t* s,
                         const int32_t* t, double* C, int64_t ldc, void* stream);

/* ---- Grouped products: one launch per phase for many products. ---- */

typedef struct oz_group_s* oz_group;

/*
 * oz_grouped_workspace_bytes / oz_group_create / oz_group_run / oz_group_destroy
 * -- count independent products C_i = A_i B_i (row-major, no transposes; the
 * problem of Sec. "Emulation Problem" for each i) whose phases run as one
 * launch per phase over all products whose plans share moduli and bit
 * budget (plans made separately but alike count as one): every A is split in one
 * launch, every B in one, the GEMMs of all products run in one persistent
 * kernel (one CTA per 128 x 256 tile, units of the longest k first), and one
 * reconstruct writes every C. Plans must be INT8 plans of a BF16 engine
 * (OZ_ENGINE_TC or OZ_ENGINE_TC1) with Q <= 16; others give
 * OZ_ERR_UNSUPPORTED.
 *   oz_grouped_workspace_bytes: the device workspace (every product's planes
 *     and residues at once, plus a descriptor table), 0 for invalid arguments.
 *   oz_group_create: checks every problem (as oz_dgemm), lays out the
 *     workspace, and writes the descriptor table into it with a synchronous
 *     copy; the matrix pointers are fixed from then on (new values in the same
 *     buffers need no new group). Arrays are host arrays of length count; the
 *     matrices and the workspace (256-byte aligned, owned by the caller, which
 *     must keep it alive while the group is used) are device memory. The
 *     group also creates two CUDA streams and a few events per set of alike
 *     plans, on the current device.
 *   oz_group_run: enqueues the phases; asynchronous and capturable into a
 *     CUDA graph. The sets of alike plans run side by side, and within a set
 *     the splits of A and of B, on the group's streams, which start after the
 *     work already queued on `stream` and which `stream` waits for at the
 *     end. oz_query_status(workspace, stream) reports non-finite input and
 *     bounded-wait time-outs as for oz_dgemm. Runs of one group must not
 *     overlap (they share the workspace and streams).
 *   oz_group_destroy: frees the handle, its streams and events (NULL is
 *     accepted).
 */
OZ_API size_t oz_grouped_workspace_bytes(int count, const oz_plan* plans, const int64_t* mnk);
OZ_API oz_status oz_group_create(oz_group* out, int count, const oz_plan* plans, const int64_t* mnk,
                                 const double* const* A, const int64_t* lda, const double* const* B,
                                 const int64_t* ldb, double* const* C, const int64_t* ldc, void* workspace,
                                 size_t workspace_bytes);
OZ_API oz_status oz_group_run(oz_group group, void* stream);
OZ_API void oz_group_destroy(oz_group group);

/* ---- Allocation-free variant. ---- */

/* Bytes of the device scratch array built into the library (per GPU). */
#define OZ_STATIC_SCRATCH_BYTES (32ull << 20)

/*
 * oz_dgemm_static -- the product of oz_dgemm for callers that cannot allocate
 * device memory, so cannot pass a workspace. The paper has no counterpart;
 * this exists for callers such as a BLAS-style dgemm front end, whose
 * signature has no workspace argument, or code running under a host program
 * that owns every device allocation through its own pool and forbids
 * cudaMalloc from libraries. Arguments and result are those of oz_dgemm
 * without the workspace pair.
 *   Scratch: a file-scope __device__ array of OZ_STATIC_SCRATCH_BYTES bytes
 *   inside liboz.so. Every GPU that loads the library holds that memory until
 *   the process exits. A product fits when oz_workspace_bytes(plan, m, n, k)
 *   <= OZ_STATIC_SCRATCH_BYTES (square products up to 512^3 on the TC
 *   engine, 768^3 on IMMA, at Q = 16); larger sizes return OZ_ERR_WORKSPACE
 *   before any launch.
 *   Allocation: none. No cudaMalloc, cudaFree or allocating library routine
 *   is called, here or in the phases it runs.
 *   Set-up: every call looks up the array's device address with
 *   cudaGetSymbolAddress in the caller's current device and context (the
 *   address differs between contexts). The first call on a device may load
 *   the library's device code there; make that first call before any stream
 *   capture on that device.
 *   Sharing: every call on a device uses the same array and leaves its
 *   contents behind; each call clears what must start at zero. Two calls that
 *   overlap on the GPU (other streams, other host threads) race on the array
 *   and give undefined results: serialise them.
 *   Status: non-finite input and a bounded device wait that ran out are
 *   recorded in the array's status word, which oz_static_query_status reads;
 *   C is then unspecified.
 */
OZ_API oz_status oz_dgemm_static(oz_plan plan, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k,
                                 const double* A, int64_t lda, const double* B, int64_t ldb,
                                 double* C, int64_t ldc, void* stream);

/*
 * oz_static_query_status -- the status of the last oz_dgemm_static call on
 * the current device, as oz_query_status reports it for a workspace: waits
 * for the stream, then reads the status word of the built-in array (no
 * allocation; a copy from the device symbol) and returns OZ_ERR_NONFINITE for
 * NaN or Inf input, OZ_ERR_CUDA if the stream has a CUDA error or a bounded
 * device wait ran out, else OZ_OK. Meaningful only while no other
 * oz_dgemm_static call on the device has run since the one it reports.
 */
OZ_API oz_status oz_static_query_status(void* stream);

/*
 * oz_selftest_bounded_wait -- exercises the failure path of the GEMM kernels'
 * waits on the device: one thread waits, with the same bounded wait the
 * kernels use, on a shared-memory barrier of its own. arrive != 0: it arrives
 * first and the wait completes (bit 2 of *status is set); arrive == 0: nothing
 * arrives, the wait gives up after about 2 s and sets bit 1, as a kernel's
 * timed-out wait does (oz_query_status then reports OZ_ERR_CUDA when status
 * is a workspace's first word). The kernel returns either way; no fault, no
 * hang. status: device int32, OR-ed into. Asynchronous on the stream.
 */
OZ_API oz_status oz_selftest_bounded_wait(int arrive, int32_t* status, void* stream);

/* Short English description of a status code (static string). */
OZ_API const char* oz_status_str(oz_status status);

#ifdef __cplusplus
}
#endif
#endif /* OZ_H_ */
