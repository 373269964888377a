/*
 * rtcur.h -- C ABI of librtcur.so, the GB300 (sm_103a) hot path of RTCUR (Robust Tensor CUR),
 * the alternating-projection robust tensor PCA method of Cai, Chao, Huang and Needell
 * ("Fast Robust Tensor Principal Component Analysis via Fiber CUR Decomposition").
 *
 * The method (Algorithm 1) splits an observed tensor X = L + S into a low-multilinear-rank L
 * and a sparse S. Each iteration k -> k+1:
 *   zeta^(k+1) = gamma * zeta^(k)                                   (Sec. 3.2, decay)
 *   S^(k+1)    = HT_{zeta^(k+1)}(X - L^(k)) on the sampled entries  (Eq. partial S update;
 *                over the whole tensor too in the FULL scope, Eq. S=HT(X-L))
 *   R = (X - S)(I_1..I_n),  C_i = (X - S)_(i)(:, J_i),  U_i = SVD_{r_i}(C_i(I_i, :))
 *   L^(k+1)    = R x_1 (C_1 U_1^+) x_2 ... x_n (C_n U_n^+)           (Eq. L=CUR)
 *   e^(k+1)    = sampled relative error                             (Eq. rel_err)
 * until e^(k) <= tol or k = max_iter.
 *
 * Conventions for every entry point:
 *   - Tensors are dense, row-major (C order, last mode contiguous), FP32, in DEVICE memory,
 *     owned by the caller. The library never frees caller memory.
 *   - Index sets are 0-based int64 in HOST memory, each strictly increasing. Per set: I_1..I_n
 *     (|I_i| = nI[i] entries in [0, d_i)) then J_1..J_n (|J_i| = nJ[i] entries in
 *     [0, prod_{j != i} d_j)). J_i indexes the columns of the mode-i unfolding X_(i) in row-major
 *     order of the remaining modes (last mode fastest).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is stream-ordered; calls
 *     that return results on the host synchronise `stream` once before returning.
 *   - No call throws. Every call returns an rtcur_status. Invalid arguments return
 *     RTCUR_EINVAL before any GPU work; the message is kept per plan (rtcur_last_error).
 *   - A plan owns all device workspace, sized at rtcur_create; rtcur_solve, rtcur_begin /
 *     rtcur_iterate / rtcur_finish, rtcur_backward and the export calls allocate nothing. The one
 *     exception is rtcur_solve_batched: the first call for a new list of plans builds and caches
 *     a batch graph, which allocates a small device array (one pointer per plan) and the graph's
 *     own resources; later calls with the same list allocate nothing. A plan is not thread-safe;
 *     distinct plans are independent.
 */
#ifndef RTCUR_H
#define RTCUR_H

#include <stdint.h>

#if defined(__GNUC__)
#define RTCUR_API __attribute__((visibility("default")))
#else
#define RTCUR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rtcur_plan rtcur_plan; /* opaque */

typedef enum {
  RTCUR_OK = 0,
  RTCUR_NOT_CONVERGED = 1, /* status, not an error: stopped at max_iter with e > tol */
  RTCUR_EINVAL = -1,       /* invalid argument (message in rtcur_last_error) */
  RTCUR_ENOMEM = -2,       /* device allocation failed at create */
  RTCUR_ECUDA = -3,        /* a CUDA runtime call failed */
  RTCUR_ENONFINITE = -4,   /* NaN or Inf met in X on the sampled entries */
  RTCUR_ETIMEOUT = -5,     /* a bounded device-side wait gave up */
  RTCUR_EDEVICE = -6       /* a device-side consistency check failed */
} rtcur_status;

enum { RTCUR_VARIANT_F = 0, RTCUR_VARIANT_R = 1 };      /* Sec. 3.4: fixed / resampled indices */
enum { RTCUR_SCOPE_SAMPLED = 0, RTCUR_SCOPE_FULL = 1 }; /* Eq. partial S update / Eq. S=HT(X-L) */
/* Dense-pass forms (FULL scope): how L^(k) is evaluated when S^(k+1) is formed over the whole
 * tensor. FP32: the factored last-mode product in FP32 FMA, fused with the threshold (default).
 * FP32_PLAIN: the literal chain of Eq. (L=CUR) materialised in FP32, then a separate HT pass.
 * BF16 / TF32: the factored product on tcgen05 tensor cores with FP32 accumulation. */
enum { RTCUR_FORM_FP32 = 0, RTCUR_FORM_FP32_PLAIN = 1, RTCUR_FORM_BF16 = 2, RTCUR_FORM_TF32 = 3 };

/* Output format of S^(k) in the FULL scope (the tensor the dense pass writes every iteration).
 * DENSE: prod d_i floats (default). COMPRESSED: the support as a bitmask plus the nonzero values
 * (rtcur_s_compressed); the method is unchanged, only the bytes written drop (at 30% density from
 * 4 to 1.33 bytes per element). Needs dense_form FP32, d_n % 4 == 0, d_n <= 4096, r_n <= 8. */
enum { RTCUR_S_DENSE = 0, RTCUR_S_COMPRESSED = 1 };

/* Where the sampled step (Step (I) on the sample, Eq. partial S update, and the gathers of R and
 * C_i) reads X from. FP32: the caller's tensor (default). BF16: a copy of X rounded to BF16
 * (round to nearest even), made by rtcur_begin in plan memory (prod d_i x 2 bytes, allocated at
 * create): the iterates are then those of the method applied to the BF16-rounded tensor (each
 * sampled value carries up to 2^-9 relative rounding), while the FULL scope's dense pass and the
 * outputs keep reading the FP32 X. FP32 values beyond BF16's range round to infinity and are
 * reported as RTCUR_ENONFINITE. */
enum { RTCUR_SAMPLE_X_FP32 = 0, RTCUR_SAMPLE_X_BF16 = 1 };

/* Bits of rtcur_result.flags */
enum {
  RTCUR_FLAG_RANK_DEFICIENT = 1, /* some SVD_{r_i} kept fewer than r_i singular values */
  RTCUR_FLAG_TIE = 2             /* some sigma_{r_i} and sigma_{r_i + 1} were not separable */
};

typedef struct rtcur_options {
  int32_t scope;             /* RTCUR_SCOPE_*; default SAMPLED */
  int32_t dense_form;        /* RTCUR_FORM_*; default FP32 (used by the FULL scope only) */
  int32_t refine_steps;      /* FP64 refinement steps of the truncated pinv; default 2 */
  int32_t jacobi_max_sweeps; /* cap on FP32 Jacobi sweeps of the pinv; default 30 */
  double inband_rel;         /* half-width of the reported threshold band, relative to zeta; 1e-6 */
  int32_t eig_method;        /* FP32 eigenbasis of the pinv: 0 tridiagonal + inverse iteration
                                (used when every |I_i| <= 128, default), 1 cyclic Jacobi */
  int32_t checkpoint;        /* record the first `checkpoint` iterations for rtcur_backward
                                (their sampled values X - S and HT masks, 5 B per sampled entry
                                per iteration); 0 = off (default). Requires n_modes == 3 and
                                checkpoint <= max_iter. */
  int32_t refine_cluster;    /* CTAs per mode in the FP64 pinv refinement (a thread-block
                                cluster): 0 = auto (16, else 8), or 2, 4, 8, 16; smaller clusters
                                suit many concurrent problems (the batched form) */
  int32_t s_format;          /* RTCUR_S_*: format of S in the FULL scope; default DENSE */
  int32_t sample_x;          /* RTCUR_SAMPLE_X_*: what the sampled step reads X from; default FP32 */
  int32_t dense_ctas;        /* persistent CTAs of the FULL scope's dense pass, one per SM; 0 = auto
                                (148 of the 152 SMs for the FP32 pass, 144 for the tensor-core
                                forms, leaving room for the concurrent sampled chain), else 1..1024 */
  int32_t reserved[2];       /* must be zero */
} rtcur_options;

/* Compressed S^(k) (s_format COMPRESSED), in device memory owned by the plan and overwritten by
 * the next dense pass. The tensor is viewed as `rows` = prod_{i<n} d_i rows of `cols` = d_n
 * elements (row-major, the last mode fastest: element e is row e / d_n, column e % d_n).
 *   mask   rows * words_per_row words; bit b of mask[r * words_per_row + w] is set iff
 *          S(r, 32 w + b) != 0 (bits at columns >= d_n are zero)
 *   vals   for each block of block_cols = 128 columns of a row (the last one may be shorter):
 *          its nonzero values, in column order, from the block's first element index on, i.e.
 *          the j-th nonzero of block k of row r is vals[r * cols + 128 k + j]; the rest of the
 *          block's range is not written
 * rtcur_compact_s packs all nonzeros into one array in element order (CSR-like). */
typedef struct rtcur_s_compressed {
  const uint32_t* mask;
  const float* vals;
  int64_t nnz;           /* nonzeros of S^(k) */
  int64_t rows;
  int64_t cols;
  int64_t words_per_row; /* ceil(d_n / 32) */
  int64_t block_cols;    /* 128 */
} rtcur_s_compressed;

typedef struct rtcur_result {
  int32_t iters;        /* k at exit */
  int32_t status;       /* RTCUR_OK or RTCUR_NOT_CONVERGED */
  int32_t flags;        /* RTCUR_FLAG_* seen in any iteration */
  int32_t jacobi_sweeps; /* FP32 Jacobi sweeps in the last iteration (max over modes) */
  double e;             /* e^(k) */
  double zeta;          /* zeta^(k) */
  int64_t nnz_sample;   /* nonzeros of S^(k) on the sampled entries (R and fiber segments) */
  int64_t inband_sample;/* sampled entries with ||X - L^(k-1)| - zeta^(k)| <= inband_rel*zeta^(k) */
  int64_t nnz_full;     /* FULL scope: nonzeros of S^(k) over the whole tensor; else -1 */
  int64_t inband_full;  /* FULL scope: the band count over the whole tensor; else -1 */
  double resid_full;    /* FULL scope: ||X - L^(k-1) - S^(k)||_F^2 over the whole tensor; else -1 */
  int64_t warm_hits;    /* (iteration, mode) pairs whose truncated SVD came from the certified
                           warm-started subspace iteration instead of the full eigensolver */
  /* Optional per-iteration histories: caller arrays of max_iter entries, or NULL. */
  double* e_hist;
  double* zeta_hist;
  int64_t* nnz_hist;
} rtcur_result;

/* rtcur_create -- validate the problem geometry and allocate a plan with all its workspace.
 *   out       receives the plan (set to NULL on failure)
 *   n_modes   n, 2 <= n <= 4
 *   dims      n mode sizes d_i >= 1, prod d_i < 2^40
 *   ranks     n target multilinear ranks r_i, 1 <= r_i <= 16 (Algorithm 1 input)
 *   nI, nJ    |I_i| in [r_i, min(d_i, 192)], |J_i| in [r_i, min(prod_{j!=i} d_j, 4096)]
 *             (Sec. 2.2 sample sizes; Sec. 4 uses ceil(v r_i ln d_i) and ceil(v r_i ln prod))
 *   zeta0     initial threshold; <= 0 means max|X| computed on the device at each solve
 *   gamma     decay factor, 0 < gamma < 1 (Sec. 3.2)
 *   tol       target e^(k) (Eq. rel_err); the loop runs while e > tol
 *   max_iter  1 <= max_iter <= 100000
 *   variant   RTCUR_VARIANT_F or RTCUR_VARIANT_R (Sec. 3.4)
 *   opt       NULL for defaults
 * Errors: RTCUR_EINVAL (bad argument), RTCUR_ENOMEM, RTCUR_ECUDA. */
RTCUR_API rtcur_status rtcur_create(rtcur_plan** out, int32_t n_modes, const int64_t* dims,
                          const int32_t* ranks, const int32_t* nI, const int32_t* nJ,
                          double zeta0, double gamma, double tol, int32_t max_iter,
                          int32_t variant, const rtcur_options* opt);

/* rtcur_solve -- run Algorithm 1 to completion on one tensor.
 *   X      device, prod d_i floats, caller-owned, read only
 *   idx    host index sets (layout above): 1 set for variant F, max_iter sets for variant R
 *          (iteration k uses set k)
 *   L_out  device, prod d_i floats or NULL: receives L^(k) = R x_i (C_i U_i^+) (Eq. L=CUR)
 *   S_out  device, prod d_i floats or NULL: receives S^(k) = HT_{zeta^(k)}(X - L^(k-1)) over
 *          the whole tensor (in the FULL scope with s_format DENSE it is also the buffer
 *          written every iteration; with COMPRESSED it is filled once, by expanding the
 *          compressed S^(k), see rtcur_get_s_compressed)
 *   res    host, filled on return (may be NULL)
 * The loop runs on the device as one CUDA graph with a conditional WHILE node; the host
 * synchronises once at the end. Returns RTCUR_OK or RTCUR_NOT_CONVERGED on success. */
RTCUR_API rtcur_status rtcur_solve(rtcur_plan* plan, const float* X, const int64_t* idx, float* L_out,
                         float* S_out, rtcur_result* res, void* stream);

/* Step-wise form of rtcur_solve (same arguments, same semantics):
 * rtcur_begin uploads the index sets and resets the state to L^(0) = 0, zeta^(0) (no host sync);
 * rtcur_iterate runs exactly n_iter iterations regardless of tol (no host sync; variant R uses
 * set (k mod max_iter)); rtcur_finish materialises L_out / S_out, fills res and synchronises. */
RTCUR_API rtcur_status rtcur_begin(rtcur_plan* plan, const float* X, const int64_t* idx, float* S_work,
                         void* stream);
RTCUR_API rtcur_status rtcur_iterate(rtcur_plan* plan, int32_t n_iter, void* stream);
RTCUR_API rtcur_status rtcur_finish(rtcur_plan* plan, float* L_out, float* S_out, rtcur_result* res,
                          void* stream);

/* rtcur_threshold_dense -- Step (I) of Algorithm 1 over the whole tensor for the current state:
 * S_work = HT_{gamma zeta^(k)}(X - L^(k)) (Eq. S=HT(X-L)) with the plan's dense form, n_launch
 * times (identical launches; for timing the fused pass alone). Needs a FULL-scope plan after
 * rtcur_begin; writes the S_work buffer given to rtcur_begin (with s_format COMPRESSED the
 * plan's compressed S instead; S_work is then unused) and the dense counters that
 * rtcur_finish reports. Does not advance k. No host sync. */
RTCUR_API rtcur_status rtcur_threshold_dense(rtcur_plan* plan, int32_t n_launch, void* stream);

/* rtcur_threshold_dense_noalloc -- the dense fused threshold pass, S = HT_zeta(X - L) with
 * L = G x_1 B_1 ... x_n B_n, for callers that cannot allocate device memory. The paper has no
 * counterpart: it is an allocation-free form of rtcur_threshold_dense for callers such as a
 * serving process whose device memory belongs to a pre-reserved pool with a hard budget, or a
 * latency-critical caller that cannot afford cudaMalloc's possible implicit synchronisation.
 *   n_modes, dims, ranks   geometry as in rtcur_create
 *   G      device, prod r_i floats (row-major core);  B  device, sum d_i r_i floats (B_i is d_i x r_i
 *          row-major, packed mode after mode) -- the layout rtcur_get_factors returns
 *   X      device, prod d_i floats, 16-byte aligned;  S  device output, prod d_i floats, 16-byte aligned
 *   zeta   threshold used as given (HT keeps |x - L| > zeta, compared in FP32)
 *   counts host double[3] or NULL: {||X - L - S||_F^2, nnz(S), band count}; when given, the call
 *          synchronises `stream` and returns a device-side error of the pass (RTCUR_ETIMEOUT when a
 *          bounded wait gave up and S may be incomplete); with NULL the call does not synchronise
 *          and such an error is not reported
 * Scratch: one fixed 32 MiB device array inside the library (held by every GPU that loads it
 * until the process exits); problems needing more (prod_{i<n} d_i * r_n + 4 floats of table plus
 * ~1.1 MB) return RTCUR_EINVAL. Nothing is allocated: no cudaMalloc, no cudaFree. The first call
 * on each device (with that device current) looks up the array's device address and caches it;
 * make that first call before any stream capture. All calls share the array, so calls that
 * overlap on the GPU race; the parts that must start at zero are cleared at every call. */
RTCUR_API rtcur_status rtcur_threshold_dense_noalloc(int32_t n_modes, const int64_t* dims,
                                                     const int32_t* ranks, const float* G,
                                                     const float* B, const float* X, double zeta,
                                                     float* S, double* counts, void* stream);

/* rtcur_get_s_compressed -- describe the compressed S^(k) = HT_{zeta^(k)}(X - L^(k-1)) of the
 * last dense pass (Sec. 3.2, Eq. S=HT(X-L); the FULL scope's S output) of a plan created with
 * s_format COMPRESSED. Fills `out` with device pointers into the plan (valid until the next
 * dense pass or rtcur_destroy) and the layout above. Synchronises `stream`.
 * Errors: RTCUR_EINVAL (NULL plan or out, another s_format, no rtcur_begin, or k = 0: no dense
 * pass has run and S^(0) = 0), RTCUR_ECUDA. */
RTCUR_API rtcur_status rtcur_get_s_compressed(rtcur_plan* plan, rtcur_s_compressed* out, void* stream);

/* rtcur_compact_s -- the nonzeros of the compressed S^(k) in element order (CSR-like with the
 * mask: the j-th set bit of the mask, in row-major order, is vals_out[j]).
 *   vals_out  device, >= nnz floats, or NULL
 *   row_off   device, rows + 1 int64, or NULL: row r's first index in vals_out; the last entry
 *             is nnz
 * At least one of the two must be given. Synchronises `stream` once to read k; the copies run
 * on `stream`. Errors: RTCUR_EINVAL (NULL plan or both outputs, another s_format, no
 * rtcur_begin, k = 0), RTCUR_ECUDA. */
RTCUR_API rtcur_status rtcur_compact_s(rtcur_plan* plan, float* vals_out, int64_t* row_off, void* stream);

/* rtcur_decode_s -- expand the compressed S^(k) into a dense tensor.
 *   S_out  device, prod d_i floats (any 4-byte alignment); receives zeros when k = 0
 * rtcur_finish (and rtcur_solve) do the same when given S_out. Synchronises `stream` once to
 * read k. Errors: RTCUR_EINVAL (NULL arguments, another s_format, no rtcur_begin), RTCUR_ECUDA. */
RTCUR_API rtcur_status rtcur_decode_s(rtcur_plan* plan, float* S_out, void* stream);

/* rtcur_get_factors -- copy the current L^(k) in Tucker form L = G x_1 B_1 ... x_n B_n to host
 * arrays (FP32): G has prod r_i entries (row-major), B_i is d_i x r_i row-major, packed mode
 * after mode in B (sum d_i r_i entries). This is the same tensor as R x_i (C_i U_i^+) of
 * Eq. (L=CUR) (B_i = C_i V_r Sigma_r^-1, G = R x_i Q_{r,i}^T with U_i = Q_r Sigma_r V_r^T).
 * Also returns k (iterations done) and zeta^(k). Synchronises `stream`. */
RTCUR_API rtcur_status rtcur_get_factors(rtcur_plan* plan, float* G, float* B, int32_t* k, double* zeta,
                               void* stream);

/* rtcur_get_cur -- copy Algorithm 1's output of the current iterate, the Fiber CUR pieces
 * (R, C_i, U_i^+) with L^(k) = R x_1 (C_1 U_1^+) x_2 ... x_n (C_n U_n^+) (Eq. (L=CUR), Eq. (R, C_i,
 * U_i) of Sec. 3.1), to host arrays. They are the pieces of the last iteration k: formed from
 * X - S^(k) on that iteration's index sets (set 0 for variant F, set (k - 1) mod max_iter for
 * variant R), in the order of those sets.
 *   R      host, prod |I_i| floats or NULL: R = (X - S^(k))(I_1, ..., I_n), row-major
 *   C      host, sum_i d_i |J_i| floats or NULL: C_i = (X - S^(k))_(i)(:, J_i), d_i x |J_i|
 *          row-major, packed mode after mode
 *   Upinv  host, sum_i |J_i| |I_i| doubles or NULL: U_i^+ = (SVD_{r_i}(C_i(I_i, :)))^+ in FP64,
 *          |J_i| x |I_i| row-major, packed mode after mode (rank r_i, or fewer where the SVD_r
 *          cutoff dropped singular values: RTCUR_FLAG_RANK_DEFICIENT)
 *   k      host or NULL: receives the iteration count k
 * The staging buffers are plan workspace (no allocation). Synchronises `stream`.
 * Errors: RTCUR_EINVAL (NULL plan, no rtcur_begin, or k = 0: L^(0) = 0 has no CUR pieces),
 * RTCUR_ECUDA. */
RTCUR_API rtcur_status rtcur_get_cur(rtcur_plan* plan, float* R, float* C, double* Upinv, int32_t* k,
                                     void* stream);

/* Batched form: `count` independent problems (each with its own plan, so dims, ranks, sample
 * sizes, variant and tolerance may all differ) solved together by ONE graph launch. The graph is
 * a device-side WHILE loop whose body holds, per problem, a conditional IF node around that
 * problem's Algorithm 1 iteration; a problem whose stopping test (Algorithm 1's loop condition)
 * fails drops out, and the loop ends when none continues. No host synchronisation happens between
 * iterations. X[i], idx[i], L_out[i], S_out[i] and res[i] are as for rtcur_solve on plans[i]
 * (L_out, S_out, res may be NULL arrays; their entries may be NULL). Every plan must have
 * tol < 1 and appear once. The graph is built on the first call for a given list of plans and
 * cached with plans[0] (rebuilt when the list changes; destroying any listed plan invalidates
 * it). Returns the first failing status of a problem, else RTCUR_OK (RTCUR_NOT_CONVERGED is
 * reported per problem in res[i].status). */
RTCUR_API rtcur_status rtcur_solve_batched(rtcur_plan* const* plans, int32_t count,
                                           const float* const* X, const int64_t* const* idx,
                                           float* const* L_out, float* const* S_out,
                                           rtcur_result* res, void* stream);

/* Adjoint of the last solve (Algorithm 1 unrolled over its K iterations, K = the iteration count
 * of the last rtcur_solve / rtcur_finish): dX = (dL^(K)/dX)^T dL, the vector-Jacobian product of
 * X -> L^(K) = R x_i (C_i U_i^+) (Eq. (L=CUR)) with dL (device, FP32, dims, row-major).
 * Hard thresholding (Eq. (HT)) is differentiated almost everywhere, with each iteration's support
 * masks on the sampled entries frozen at their forward values: an unmasked sampled entry passes
 * its adjoint to X, a masked one to the previous L^(k). The truncated pseudoinverse U_i^+ is
 * differentiated where sigma_{r_i} > sigma_{r_i+1} > ... (a.e.), through the eigenpairs of
 * U_i U_i^T (FP64 Jacobi, Daleckii-Krein divided differences). Only L^(K) depends on X through
 * the sampled entries, so dX is zero off the sample.
 * dX: device, FP32, dims, overwritten (16-byte aligned). dL may alias nothing the plan owns.
 * Requires a plan created with options.checkpoint >= K (and n_modes == 3); otherwise
 * RTCUR_EINVAL. Synchronises the stream once (to read K). Uses plan-owned workspace sized at
 * create; allocates nothing. */
RTCUR_API rtcur_status rtcur_backward(rtcur_plan* plan, const float* dL, float* dX, void* stream);

/* rtcur_set_wait_limit -- bound on the device-side waits of the plan's FP32 dense threshold pass
 * (the FULL scope's per-iteration pass over the whole tensor, Eq. S=HT(X-L)). Each tile of that
 * pass waits for its asynchronous copy on a shared-memory barrier; a wait that does not complete
 * within its bound gives up, the pass waits (with the default bound) for its own copies still in
 * flight, records RTCUR_ETIMEOUT and returns, the solve stops after the iteration and
 * rtcur_finish / rtcur_solve return RTCUR_ETIMEOUT. The context stays usable and the next
 * rtcur_begin clears the error.
 *   polls  0: the default bound (2^26 polls, seconds); n > 0: n non-blocking polls per wait, from
 *          the next launch on (a short bound reports a stalled pass sooner; 1 makes the first
 *          wait of every launch give up, which is how the failure path is tested)
 * The paper has no counterpart (failure detection of the pass). Synchronises `stream`.
 * Errors: RTCUR_EINVAL (NULL plan, polls < 0), RTCUR_ECUDA. */
RTCUR_API rtcur_status rtcur_set_wait_limit(rtcur_plan* plan, int64_t polls, void* stream);

/* Number of sampled entries per iteration: prod |I_i| + sum_i d_i |J_i| (the subtensor R and the
 * n fiber sets C_i of Sec. 3.3). 0 for a NULL plan. */
RTCUR_API int64_t rtcur_sample_count(const rtcur_plan* plan);

/* Last error message of a plan (NULL plan: the last create failure); never NULL. */
RTCUR_API const char* rtcur_last_error(const rtcur_plan* plan);

/* Free a plan and its workspace; NULL is allowed. Synchronises the device first. */
RTCUR_API void rtcur_destroy(rtcur_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* RTCUR_H */
