/*
 * lrq.h -- C ABI of liblrq, the GB300 (sm_103a) library for batched
 * candidate scoring in low-rank discrete quadratic maximisation
 * (arXiv 2602.20376, "Exploiting Low-Rank Objective Structure in Discrete
 * Quadratic Optimization").
 *
 * Problem (Sec. 1, Eq. 1-2): maximise z^H Q z over z in A_K^n, where
 * A_K = { exp(2 pi i k / K) : k = 0..K-1 } and Q ~= V V^H, V in C^{n x r}.
 * With Q = V V^H the objective is ||V^H z||^2 (Sec. 2.2, Eq. 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an lrq_status (0 = LRQ_OK).  No C++ exception
 *   crosses the ABI.  On failure lrq_last_error() returns a message for the
 *   calling thread.
 * - Argument errors (sizes, null pointers, unsupported K or r) are detected
 *   on the host before any launch and return LRQ_EINVAL or
 *   LRQ_EUNSUPPORTED; nothing is launched in that case.
 * - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *   means the legacy default stream).  Errors found on the device (non-finite
 *   input, a bounded wait that ran out) are written as an lrq_status into
 *   `*dev_status` (a device int32 the caller zeroes and reads after
 *   synchronising); the first error wins.  dev_status may not be NULL where a
 *   signature has it.
 * - The caller owns every buffer.  All array arguments are DEVICE pointers
 *   unless a comment says "host".  The library allocates no device memory:
 *   scratch space is the caller's `ws` of `ws_bytes` bytes, sized by the
 *   matching *_workspace_size query; ws must be 256-byte aligned.
 * - Complex arrays are interleaved (re, im): complex64 = 2 x float,
 *   complex128 = 2 x double (the layout of torch.complex64 / complex128).
 *   Matrices are row-major and contiguous: V is n x r (row i = V_{i,:}),
 *   C is S x r (row s = candidate direction c_s).
 * - Assignments z are returned as codes k_i in [0, K), z_i = exp(2 pi i k_i/K),
 *   one uint8 per coordinate.
 * - The decision rule (Sec. 3, Eq. 9) maps w = V_i c to the nearest K-th root
 *   of unity in angle.  Exactly on a boundary several roots are equally
 *   near; the library then picks one of them (which one is unspecified).
 */
#ifndef LRQ_H
#define LRQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRQ_OK = 0,
  LRQ_EINVAL = 1,        /* invalid argument, or non-finite input found on the device */
  LRQ_EUNSUPPORTED = 2,  /* valid but unsupported (K, r, size or mode)                */
  LRQ_ECUDA = 3,         /* a CUDA runtime call failed                                 */
  LRQ_ETIMEOUT = 4,      /* a bounded device-side wait ran out                         */
  LRQ_ENOCONV = 5,       /* an iterative solver did not converge                       */
  LRQ_EWORKSPACE = 6     /* ws is NULL, misaligned or smaller than required            */
} lrq_status;

/* Scoring modes of lrq_sample_score.
 *
 * LRQ_MODE_FP32: CUDA-core FP32 scoring; f within 1e-5 relative of the FP64
 *   value of the same candidate (blocked FP32 sums added in FP64).
 * LRQ_MODE_TC: tcgen05 tensor-core scoring.  Operand and accumulator types:
 *   GEMM1 (boundary projections, whose signs give the rounding): F16 x F16
 *   with an F16 accumulator, every coordinate row and every direction scaled
 *   by a power of two (signs unchanged); GEMM2 (per-class sums): FP8 E4M3 x
 *   E4M3 with FP32 accumulation, the class operand split as hi + lo E4M3 and
 *   scaled per coordinate by a power of two; FP32 accumulation periods of at
 *   most 2048 coordinates added error-free (two-sum) and written in FP64.
 *   Error bound: a projection is off by at most 2^-6.8 sum_j |V_ij|_1 |c_j|_1,
 *   so a code can differ from the FP64 decision only where |w_i| sin(margin)
 *   is below that; each such coordinate moves ||V^H z|| by at most
 *   2 sin(pi/K) |V_i|, and the E4M3 class operand adds at most
 *   2^-8 sqrt(2) max|beta| |V_i| + sqrt(2) 2^-15 max|V component| per
 *   coordinate.  The winners are re-scored in FP64 (lrq_rescore).
 * LRQ_MODE_BF16_TC: deprecated alias of LRQ_MODE_TC (its first version used
 *   BF16 operands for both contractions); kept so that old callers compile. */
typedef enum {
  LRQ_MODE_FP32 = 0,
  LRQ_MODE_TC = 1,
  LRQ_MODE_BF16_TC = 1
} lrq_mode;

/* Human-readable name of a status code (static string, never NULL). */
const char* lrq_status_string(int status);

/* Message describing the most recent failure on the calling thread
 * (static per-thread buffer; empty string if none). */
const char* lrq_last_error(void);

/* ABI version of this header (incremented on any signature change). */
int lrq_abi_version(void);

/* --------------------------------------------------------------------------
 * lrq_sample_directions -- uniform directions on the unit sphere of C^r.
 *
 * Sec. 4.2 (sampling candidates) and App. E (Lemma "innerIsBeta"):
 * c = Z / ||Z|| with Z ~ CN(0, I_r) is uniform on the complex sphere.
 * Z is drawn with the counter-based generator Philox4x32-10 (Salmon et al.,
 * SC'11): component j of candidate s uses counter (lo32(s), hi32(s), j, 0)
 * and key (lo32(seed), hi32(seed)); output words (0,1) and (2,3) give two
 * 53-bit uniforms u1, u2 = (top 53 bits + 0.5) / 2^53, and
 * Z_j = sqrt(-ln u1) * exp(2 pi i u2) (Box-Muller, Re and Im ~ N(0, 1/2)).
 * The normalisation runs in FP64; the result is rounded once to complex64.
 *
 *   C_out : S x r complex64 (device), written.
 *   1 <= r <= 64, S >= 0 (S = 0 launches nothing).
 * ------------------------------------------------------------------------ */
int lrq_sample_directions(uint64_t seed, int64_t S, int r, void* C_out, void* stream);

/* --------------------------------------------------------------------------
 * lrq_sample_null_directions -- the null-vector sampler (Sec. 5, "The
 * analyzed sampler matches the one used in practice"): the randomised form
 * of Algorithm 2, the alternative to lrq_sample_directions.
 *
 * Each candidate is the null vector of 2r - 1 rows of the augmented real
 * matrix (Eq. 6), drawn uniformly without replacement from its N = n B_K
 * rows h_(i,m) = [Im(rho_m V_i), Re(rho_m V_i)], rho_m = exp(-i pi(2m+1)/K),
 * numbered R = i B_K + m (B_K = K/2 for even K, K for odd K).  Rows that are
 * linearly dependent (FP64 elimination with full pivoting: largest
 * remaining pivot <= 1e-10 max|H|) give no unique direction: the draw is
 * rejected and the slot draws again, up to 64 times.
 *
 * Draws: Philox4x32-10, key (lo32 seed, hi32 seed); row j of attempt a of
 * slot s, try t, uses counter (lo32 s, hi32 s, (a << 8) | (j << 4) | t,
 * 0x4E56) and row R = high 64 bits of ((w0 << 32) | w1) * N; a row already
 * in the attempt is drawn again with the next t (up to 16).  The null vector
 * is scaled to unit norm with its largest-magnitude entry positive (first
 * on ties), negated when bit 0 of w2 of the attempt's first draw is set;
 * c = c~[0:r] + i c~[r:2r], rounded to complex64.
 *
 *   V         : n x r complex64 (device), the scoring input.
 *   C_out     : S x r complex64 (device), unit-norm rows; feed it to
 *               lrq_sample_score with generate_C = 0.
 *   draws_out : 1 int64 (device): subsets drawn in total (S / draws is the
 *               acceptance rate).
 * Limits: 1 <= r <= 8, 2 <= K <= 64, 1 <= S < 2^31, n B_K >= 2r - 1.  A
 * slot with no accepted draw in 64 gets a zero row and *dev_status =
 * LRQ_EUNSUPPORTED (e.g. V of rank below r).
 * ------------------------------------------------------------------------ */
int lrq_sample_null_directions(const void* V, int64_t n, int r, int K, uint64_t seed, int64_t S, void* C_out,
                               int64_t* draws_out, int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * lrq_sample_score -- score S candidate directions and select the top m.
 *
 * For every direction c_s (Sec. 4.2, Eq. 10):
 *   w_i = V_i c_s                (i = 1..n)
 *   k_i = nearest root in angle  (Sec. 3, Eq. 9)
 *   f_s = || V^H z(c_s) ||^2
 * then the m best (f_s, s) pairs, f descending, ties to the lower s
 * ("returns only the best candidate found", Sec. 5; best-of-S, Sec. 4.2).
 *
 *   V        : n x r complex64 (device).  Must be finite (checked on the
 *              device; a non-finite entry sets *dev_status = LRQ_EINVAL).
 *   n, r, K  : n >= 1; K in [2, 64]; r in [1, 8].
 *   C        : S x r complex64 (device).  If generate_C != 0 the call first
 *              fills C exactly as lrq_sample_directions(seed, S, r, C) would;
 *              otherwise C is read as given (rows need not be unit norm).
 *   S        : number of candidates, S >= 1, S < 2^31.
 *   mode     : LRQ_MODE_FP32 or LRQ_MODE_BF16_TC.  The tensor-core mode
 *              computes the sector signs from w = V c in F16 (operands
 *              and accumulator; every row of V and every direction scaled
 *              by a power of two, which changes no sign), and the
 *              per-class sums of V^H z from a hi + lo pair of FP8 E4M3
 *              numbers per entry, scaled by a power of two per coordinate
 *              (about bfloat16's precision; the class indicators are
 *              exact), accumulated in FP32 and combined in FP64; it
 *              supports K <= 8 and r <= 8.  FP32 mode computes w and V^H z
 *              in FP32 with FP64 partials.
 *   top_m    : 1 <= top_m <= 512 and top_m <= S.
 *   scores_out  : optional S floats (device) receiving f_s; may be NULL.
 *   top_idx_out : top_m int64 (device): candidate indices, best first.
 *   top_f_out   : top_m floats (device): their scores.
 *   ws, ws_bytes: scratch, at least lrq_sample_score_workspace_size(...).
 * ------------------------------------------------------------------------ */
int lrq_sample_score_workspace_size(int64_t n, int r, int K, int64_t S, int mode, int top_m,
                                    size_t* bytes /* host */);
int lrq_sample_score(const void* V, int64_t n, int r, int K, void* C, int generate_C, uint64_t seed,
                     int64_t S, int mode, int top_m, float* scores_out, int64_t* top_idx_out,
                     float* top_f_out, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * Prepared instance -- lrq_sample_score split in two, for many calls on one V.
 *
 * Of the work in lrq_sample_score, the finiteness check of V and (tensor-core
 * mode) the column sums of conj(V) and the packed coordinate operands depend
 * on V only.  lrq_prepare does that part once into a caller-owned device
 * buffer; every lrq_sample_score_prepared call then draws or reads its
 * directions, packs them, scores and selects exactly as lrq_sample_score
 * does (same top_idx_out, top_f_out and scores_out for the same V, C, K,
 * mode, top_m).
 *
 *   lrq_prepared_create(n, r, K, mode, &h)  validates as lrq_sample_score
 *       does (n, r, K, mode); host only, allocates the host object *h.
 *   lrq_prepared_size(h, &bytes)  device bytes of the prepared buffer (0 in
 *       FP32 mode, which reads V itself).
 *   lrq_prepare(h, V, buf, buf_bytes, dev_status, stream)  asynchronous;
 *       buf: at least that many bytes, 256-byte aligned (or NULL when 0);
 *       a non-finite V sets *dev_status = LRQ_EINVAL.  h remembers V and buf:
 *       both must stay allocated and unchanged while h is used (a changed V
 *       needs a new lrq_prepare).  Calls on other streams must be ordered
 *       after this one by the caller.
 *   lrq_sample_score_prepared_workspace_size(h, S, top_m, &bytes)
 *   lrq_sample_score_prepared(h, C, generate_C, seed, S, top_m, scores_out,
 *       top_idx_out, top_f_out, ws, ws_bytes, dev_status, stream)
 *       arguments as in lrq_sample_score; LRQ_EINVAL before lrq_prepare.
 *       Calls on one h may run concurrently with separate workspaces.
 *   lrq_prepared_destroy(h)  frees the host object (not buf, not V).
 * ------------------------------------------------------------------------ */
typedef struct lrq_prepared_v lrq_prepared_v;
int lrq_prepared_create(int64_t n, int r, int K, int mode, lrq_prepared_v** out);
void lrq_prepared_destroy(lrq_prepared_v* h);
int lrq_prepared_size(const lrq_prepared_v* h, size_t* bytes /* host */);
int lrq_prepare(lrq_prepared_v* h, const void* V, void* buf, size_t buf_bytes, int32_t* dev_status, void* stream);
int lrq_sample_score_prepared_workspace_size(const lrq_prepared_v* h, int64_t S, int top_m, size_t* bytes /* host */);
int lrq_sample_score_prepared(const lrq_prepared_v* h, void* C, int generate_C, uint64_t seed, int64_t S, int top_m,
                              float* scores_out, int64_t* top_idx_out, float* top_f_out, void* ws, size_t ws_bytes,
                              int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * lrq_rescore -- FP64 re-scoring of selected candidates.
 *
 * For each of the m candidates idx[t] (rows of C), recompute w = V c, the
 * decision rule (Eq. 9) and f = || V^H z ||^2 (Eq. 10) to FP64 accuracy from
 * the complex64 V and C upcast exactly; the decisions are exact FP64
 * decisions.  Also returns the best of the m (largest f, ties to the earlier
 * position t), i.e. the winner of the "top-m candidates are re-scored"
 * step.
 *
 *   idx      : m int64 (device), each in [0, S) (checked on the device).
 *   f_out    : m doubles (device).
 *   z_out    : optional m x n uint8 codes (device); may be NULL.
 *   best_out : 1 int64 (device): idx[t*] of the best candidate.
 *   best_f_out : 1 double (device): its f.
 *   1 <= m <= 4096; K in [2, 64]; r in [1, 8].
 *   ws       : lrq_rescore_workspace_size(n, r, m) bytes of device memory,
 *              owned by the caller: the per-chunk partial sums, m x chunks x
 *              16 doubles, chunks = the larger of about four blocks of 16
 *              candidates per SM and ceil(n / 65536), at most 65535.
 * ------------------------------------------------------------------------ */
int lrq_rescore_workspace_size(int64_t n, int r, int m, size_t* bytes /* host */);
int lrq_rescore(const void* V, int64_t n, int r, int K, const void* C, int64_t S, const int64_t* idx,
                int m, double* f_out, uint8_t* z_out, int64_t* best_out, double* best_f_out, void* ws,
                size_t ws_bytes, int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * lrq_rescore_no_alloc -- lrq_rescore without a workspace argument.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (a plugin whose host framework owns all
 * device allocations, a latency-critical path where cudaMalloc / cudaFree may
 * synchronise the device, a service that forbids allocation after start-up).
 * It computes exactly what lrq_rescore computes, with the same arguments
 * minus ws / ws_bytes, and allocates nothing.
 *
 * Scratch: a fixed 4 MiB array inside the library (each GPU that loads the
 * library holds it until the process exits).  Sizes whose scratch need,
 * lrq_rescore_workspace_size(n, r, m), exceeds 4194304 bytes are rejected
 * with LRQ_EUNSUPPORTED (e.g. m = 64 works up to n = 2^25).  The array's
 * device address belongs to a CUDA context: the first call in each context
 * (the device's primary context, a caller's own driver-API context, a new
 * primary context after a device reset) looks it up and caches it for that
 * context; make that first call before any stream capture.  All calls in a
 * context share the array: calls that overlap on the GPU (e.g. on two
 * streams) race and must be serialised by the caller.
 * ------------------------------------------------------------------------ */
int lrq_rescore_no_alloc(const void* V, int64_t n, int r, int K, const void* C, int64_t S,
                         const int64_t* idx, int m, double* f_out, uint8_t* z_out, int64_t* best_out,
                         double* best_f_out, int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * Batched scoring: many independent instances in one persistent launch.
 *
 * Each problem p is the sampling method of Sec. 4.2 on its own V_p (n_p x r_p
 * complex64) and alphabet K_p: S_p directions (the caller's, or drawn on the
 * device as in lrq_sample_directions with seed_p + call index), FP32
 * scoring, then the top_m candidates by FP32 score are re-scored in FP64
 * (decisions and sums in FP64) and the best is returned.  All problems'
 * (problem, candidate tile) work items run in one persistent kernel, longest
 * first; the candidate tile per (r, K, floor(log2 n)) class comes from the
 * library's autotuner (lrq_batched_autotune) or its cache, else 128.
 *
 * Life cycle (all host calls; plan is a HOST object):
 *   lrq_batched_plan_create(problems, P, top_m, &plan)  validates, no launch
 *   lrq_batched_workspace_size(plan, &bytes)
 *   lrq_batched_prepare(plan, ws, ws_bytes, stream)      uploads descriptors
 *       into ws and resets the call index; synchronous
 *   lrq_batched_autotune(plan, ws, ws_bytes, dev_status, stream)  optional,
 *       synchronous: times tiles 64/128/256 per class on the plan's own
 *       problems, keeps the fastest in the plan and a process-wide cache
 *   lrq_sample_score_batched(plan, ws, ...)              asynchronous; only
 *       kernel launches and a memset, so it can be captured in a CUDA graph
 *   lrq_batched_graph_create(...) captures exactly that into a graph
 *       (stream must not be the legacy default stream); replay with
 *       lrq_graph_launch, free with lrq_graph_destroy.  Replays advance the
 *       call index, so drawn directions differ between replays.
 *   lrq_batched_plan_destroy(plan)
 *
 *   problems : P problem descriptors (HOST array; V and C device pointers,
 *              which must stay valid while the plan is used).
 *   best_f_out : P doubles (device), FP64 objective of each problem's winner.
 *   best_idx_out : P int64 (device), the winner's candidate index (-1 for
 *              an exact problem).
 * Exact sub-batch: a problem with S = 0 (and C = NULL) is solved exactly in
 * the same persistent launch by vertex enumeration (Sec. 3, Algorithm 2;
 * the candidates and FP64 arithmetic of lrq_enumerate, on V converted to
 * FP64): best_f_out is max over A_K^n of ||V^H z||^2 and best_idx_out is
 * -1.  Allowed when r <= 4, K <= 8, n <= 512 and r n^(2r+1) <= 1e10 (for
 * r = 2: n <= 87); otherwise plan creation fails with
 * LRQ_EUNSUPPORTED.  A vertex at which too many coordinates touch a
 * boundary to be branched exactly reports LRQ_EUNSUPPORTED in *dev_status,
 * as does a V whose first column is zero (no index set of full rank).
 * Limits: 1 <= r_p <= 8, 2 <= K_p <= 64, 0 <= S_p <= 8192, 1 <= n_p < 2^31,
 * 1 <= top_m <= 16 and top_m <= S_p for every sampled problem, P <= 65535.
 * Non-finite V or C -> LRQ_EINVAL in *dev_status.
 * ------------------------------------------------------------------------ */
typedef struct {
  const void* V;   /* n x r complex64 (device) */
  int64_t n;
  int r;
  int K;
  const void* C;   /* S x r complex64 (device), or NULL: drawn on the device */
  int64_t S;
  uint64_t seed;
} lrq_problem;

typedef struct lrq_batched_plan lrq_batched_plan;

int lrq_batched_plan_create(const lrq_problem* problems, int P, int top_m, lrq_batched_plan** plan_out);
void lrq_batched_plan_destroy(lrq_batched_plan* plan);
int lrq_batched_workspace_size(const lrq_batched_plan* plan, size_t* bytes);
int lrq_batched_prepare(lrq_batched_plan* plan, void* ws, size_t ws_bytes, void* stream);
int lrq_batched_autotune(lrq_batched_plan* plan, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream);
int lrq_batched_tile(const lrq_batched_plan* plan, int p); /* the candidate tile of problem p, or -1 */
int lrq_sample_score_batched(const lrq_batched_plan* plan, void* ws, size_t ws_bytes, double* best_f_out,
                             int64_t* best_idx_out, int32_t* dev_status, void* stream);
int lrq_batched_graph_create(const lrq_batched_plan* plan, void* ws, size_t ws_bytes, double* best_f_out,
                             int64_t* best_idx_out, int32_t* dev_status, void* stream, void** graph_exec_out);
int lrq_graph_launch(void* graph_exec, void* stream);
int lrq_graph_destroy(void* graph_exec);

/* --------------------------------------------------------------------------
 * lrq_truncate -- spectral truncation Q ~= V V^H (Sec. 4.1, Algorithm 3).
 *
 * Computes the r largest (algebraic) eigenvalues lambda_1 >= ... >= lambda_r
 * of a Hermitian operator and their eigenvectors u_j, and returns
 * V = [sqrt(lambda_1) u_1, ..., sqrt(lambda_r) u_r] with the columns of
 * non-positive eigenvalues set to zero (a maximisation of z^H Q z gains
 * nothing from them).  FP64 Lanczos with full reorthogonalisation on the GPU;
 * converged pairs are locked and further runs from fresh random starts
 * recover every copy of a repeated eigenvalue among the r largest.
 *
 * Operators (lrq_matrix, a HOST struct whose array members are device
 * pointers):
 *   LRQ_MATRIX_DENSE_C128   values: n x ld complex128, row-major; the caller
 *                           guarantees Q = Q^H (only y = Q x is used).
 *   LRQ_MATRIX_CSR_LAPLACIAN  L = D - A of an undirected graph: rowptr (n+1
 *                           int32), colidx (nnz int32), weights (nnz double,
 *                           or NULL for unit weights); each edge stored in
 *                           both rows; self loops ignored.  This is the Q of
 *                           Max-K-Cut (Sec. 1).
 *
 *   r        : 1 <= r <= min(8, n).
 *   tol      : residual tolerance ||Q y - theta y|| <= tol ||T|| for every
 *              wanted Ritz pair (<= 0 selects 1e-10).
 *   max_iter : Krylov dimension cap per run (0 selects min(500, n); at most
 *              4096).  Workspace grows as n * (max_iter + 2r + 9) scalars.
 *   seed     : start vectors are Philox4x32-10 Gaussians keyed by seed.
 *   V_out    : n x r complex128 (device) or NULL.
 *   V32_out  : n x r complex64 (device, V rounded to nearest) or NULL; the
 *              input layout of lrq_sample_score.
 *   lambda_out : r doubles (device), descending.
 *   iters_out  : HOST int64, total Lanczos steps over all runs, or NULL.
 * Errors: invalid CSR (rowptr not monotone, rowptr[0] != 0,
 * rowptr[n] != nnz, colidx out of range) or non-finite values -> LRQ_EINVAL
 * (found on the device and returned by this call); no convergence within
 * max_iter -> LRQ_ENOCONV.
 * Unlike the other entry points this call is synchronous: it waits on
 * `stream` at every convergence check (every 2 to 8 Lanczos steps) and
 * returns after the outputs are written.
 * ------------------------------------------------------------------------ */
typedef enum {
  LRQ_MATRIX_DENSE_C128 = 0,
  LRQ_MATRIX_CSR_LAPLACIAN = 1
} lrq_matrix_kind;

typedef struct {
  int kind;               /* lrq_matrix_kind */
  int64_t n;
  const void* values;     /* dense: n x ld complex128 (device) */
  int64_t ld;
  const int32_t* rowptr;  /* CSR: n + 1 (device) */
  const int32_t* colidx;  /* CSR: nnz (device) */
  const double* weights;  /* CSR: nnz (device) or NULL = unit weights */
  int64_t nnz;
} lrq_matrix;

int lrq_truncate_workspace_size(const lrq_matrix* Q, int r, int max_iter, size_t* bytes);
int lrq_truncate(const lrq_matrix* Q, int r, double tol, int max_iter, uint64_t seed, void* V_out, void* V32_out,
                 double* lambda_out, int64_t* iters_out, void* ws, size_t ws_bytes, int32_t* dev_status,
                 void* stream);

/* --------------------------------------------------------------------------
 * lrq_spectral_energy -- the spectral energy ratio rho_r (Sec. 5, "When does
 * low-rank work?"): the share of Q's spectral energy that its top r
 * eigenvalues leave out, a cheap test of whether a rank-r truncation (and so
 * this library's solvers) suits the instance.
 *
 *   rho_r = 1 - sum_{j<=r} max(lambda_j, 0) / trace(Q).
 *
 * For the PSD Q of the paper's problem (Sec. 1) trace(Q) is the sum of all
 * eigenvalues, so only the top r (from lrq_truncate) are needed; for an
 * indefinite Q the denominator is still trace(Q) and rho_r is then not a
 * share of the positive spectrum.
 *
 *   Q        : as for lrq_truncate (dense: sum of Re Q_ii; Laplacian: sum of
 *              the edge weights over both rows, self loops ignored).
 *   lambda   : r doubles (device), the top eigenvalues, e.g. lambda_out of
 *              lrq_truncate; r >= 0.
 *   trace_out, rho_out : 1 double each (device), written.  trace(Q) = 0
 *              (Q = 0) gives rho_r = 0.
 * Errors: a negative or non-finite trace, non-finite lambda, or a malformed
 * CSR (as for lrq_truncate) -> LRQ_EINVAL in *dev_status.  The trace is an
 * FP64 sum in a nondeterministic order (exact for unit weights).
 * ------------------------------------------------------------------------ */
int lrq_spectral_energy(const lrq_matrix* Q, const double* lambda, int r, double* trace_out, double* rho_out,
                        int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * lrq_rank1_sweep -- exact maximiser for rank 1 by an angular sweep
 * (Sec. 2.5, Algorithm 1), optionally scored on a graph's exact cut.
 *
 * For Q = q q^H and c = exp(i phi), every code of z(c) advances once as phi
 * runs over one period 2 pi / K; the optimum of |q^H z|^2 is one of the
 * n + 1 states met on the way.  Convention: t_i = K arg(q_i) / (2 pi); state
 * 0 has codes floor(t_i) mod K; coordinate i advances at
 * phi_i = (2 pi / K)(1/2 + floor(t_i) - t_i); state s has advanced the s
 * coordinates first in the order (phi_i, i).  All states are evaluated in
 * FP64 (sort, prefix sums); ties go to the earliest state.
 *
 *   q        : n complex128 (device), e.g. sqrt(lambda_1) u_1 from
 *              lrq_truncate with r = 1.
 *   z_out    : n uint8 codes of the best state (device), f_out: 1 double,
 *              its |q^H z|^2 (device).
 *   rowptr, colidx, nnz : optional undirected graph, symmetric CSR int32
 *              (each edge in both rows, self loops ignored); NULL to skip.
 *              Then cut_out (1 int64) and zcut_out (n uint8) receive the
 *              state with the largest exact cut #{edges with k_i != k_j}
 *              and its codes: the sweep path of the rank-1 relaxation scored
 *              on the true Max-K-Cut objective (Sec. 1), all n + 1 states at
 *              once through a per-edge difference array.
 *   ws       : lrq_rank1_workspace_size(n) bytes.
 * Limits: 1 <= n < 2^31, 2 <= K <= 64.  Non-finite q -> LRQ_EINVAL in
 * *dev_status.  CSR reads are bounds-guarded by nnz.
 * ------------------------------------------------------------------------ */
int lrq_rank1_workspace_size(int64_t n, size_t* bytes);
int lrq_rank1_sweep(const void* q, int64_t n, int K, uint8_t* z_out, double* f_out, const int32_t* rowptr,
                    const int32_t* colidx, int64_t nnz, int64_t* cut_out, uint8_t* zcut_out, void* ws,
                    size_t ws_bytes, int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * lrq_two_eigvec_q -- the rank-1 input of two-eigenvector complex rounding
 * (App. "Two-Eigenvector Complex Rounding", Eq. 12).
 *
 * A real symmetric Q (a graph Laplacian) has real eigenvectors, whose phases
 * are 0 or pi: a rank-1 sweep on one of them reaches only two of the K = 3
 * sectors.  The fix combines the top two, q_i = u_1(i) + i u_2(i), so that
 * arg(q_i) covers the whole circle.
 *
 *   V      : n x r complex128, row-major (device), r >= 2: the V of
 *            lrq_truncate, columns sqrt(lambda_j) u_j with u_j real (the
 *            CSR Laplacian path computes in real arithmetic); only the real
 *            parts of columns 0 and 1 are read.
 *   lambda : r doubles (device), the eigenvalues lrq_truncate returned;
 *            u_j = V_j / sqrt(lambda_j), and a column with lambda_j <= 0
 *            contributes 0.
 *   q_out  : n complex128 (device), written; the q of lrq_rank1_sweep.
 * ------------------------------------------------------------------------ */
int lrq_two_eigvec_q(const void* V, int64_t n, int r, const double* lambda, void* q_out, void* stream);

/* --------------------------------------------------------------------------
 * lrq_enumerate -- exact maximiser for rank r by vertex enumeration.
 *
 * Sec. 3, Algorithm 2 (with Theorem 3.2: for Q = V V^H of rank r the
 * enumeration finds a global maximiser of z^H Q z over A_K^n).  Runs the
 * levels d = r, r-1, ..., 1 on the leading columns V[:, :d].  At each level
 * the augmented rows (Eq. 6) h_(i,m) = [Im(rho_m V_i), Re(rho_m V_i)],
 * rho_m = exp(-i pi (2m+1)/K), m < B_K, are the normals of the decision
 * boundaries in R^{2d}.  Every index set I of 2d-1 rows with at most two rows
 * per coordinate is solved in FP64 for the null vector of its rows (sets of
 * lower rank are skipped); both signs of that direction are expanded into
 * every assignment of the cells touching the vertex (all K codes for a
 * coordinate with two rows in I, the two codes across a boundary that passes
 * within 1e-9 rad of w_i, the decision-rule code of Eq. 9 elsewhere), and
 * each is scored as ||V^H z||^2 on the full V in FP64.  This candidate set
 * contains the paper's (Algorithm 4 resolves the same ambiguity with one
 * fixed-angle solve per vertex).
 *
 *   V        : n x r complex128 (device), row-major.
 *   budget   : refuse with LRQ_EUNSUPPORTED when r * n^(2r+1) > budget
 *              (<= 0 selects 1e12).
 *   z_out    : n uint8 codes of the best assignment (device), written.
 *   f_out    : 1 double, ||V^H z||^2 of z_out (device), written.
 *   n_sets_out : 1 int64, number of full-rank index sets over all levels
 *              (device, written), or NULL.
 *   ws       : lrq_enumerate_workspace_size bytes.
 * Limits: 1 <= n <= 512, 1 <= r <= 4, 2 <= K <= 8.  A vertex touching more
 * than 12 boundaries at once or giving more than 65536 assignments (a
 * degenerate V, e.g. many identical rows) makes the call report
 * LRQ_EUNSUPPORTED in *dev_status instead of an uncertified answer.
 * Non-finite V -> LRQ_EINVAL in *dev_status.  Zero rows of V get code 0.
 * Ties between equal objectives go to the first vertex in the order
 * (level descending, index sets in colexicographic order, + before -).
 * ------------------------------------------------------------------------ */
int lrq_enumerate_workspace_size(int64_t n, int r, int K, size_t* bytes);
int lrq_enumerate(const void* V, int64_t n, int r, int K, double budget, uint8_t* z_out, double* f_out,
                  int64_t* n_sets_out, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * Learned proposal (the paper has no counterpart: it samples directions
 * uniformly, Sec. 4.2).  A small network maps spectral features of V to a
 * mixture of 16 von Mises-Fisher densities on the unit sphere S^7 of
 * C^4 = R^8 (r = 4), from which directions are drawn instead.  Directions c
 * and omega^k c score the same (Sec. 2.3), so targets are kept in the
 * window arg c_1 in (-pi/K, pi/K] and samples get a random omega^k.
 *
 * lrq_proposal_features: for B instances (V: B x n x r complex64, lambda:
 *   B x r doubles, both device), writes the gauge-fixed V (each column times
 *   |a| / a, a its entry of largest modulus, lowest row on ties) to Vg_out
 *   (B x n x r complex64) and F = 5 r + 4 features per instance to feat_out
 *   (B x F floats): lambda_j / sum lambda, then mean, variance, skewness and
 *   excess kurtosis of ||V_i||^2 n / sum lambda and of |V_ij|^2 n / lambda_j
 *   for each column j (FP64 inside).  sum lambda <= 0 -> LRQ_EINVAL on the
 *   device.
 * lrq_mlp_forward / lrq_mlp_backward: the network F -> 256 -> 256 -> 160,
 *   ReLU after the hidden layers.  params (lrq_proposal_num_params(F)
 *   floats): W1 (F x 256), b1, W2 (256 x 256), b2, W3 (256 x 160), b3, each W
 *   row-major (in x out).  X: B x F; H1, H2: B x 256 (written by forward,
 *   read by backward); O: B x 160.  backward: dO (B x 160) -> grads (same
 *   layout as params), scratch: 2 B x 256 floats.  bf16 != 0 rounds every
 *   GEMM operand to bfloat16 and runs the GEMMs on the tensor cores
 *   (tcgen05, BF16 x BF16 -> FP32 in tensor memory); a bounded device wait
 *   in that path that runs out (never observed) writes NaN into its output
 *   tile.  bf16 == 0 computes in FP32 on the CUDA cores.  1 <= B <= 2097120
 *   (LRQ_EUNSUPPORTED above).
 * lrq_vmf_nll: O (B x 160): per component m, outputs 10m..10m+7 give
 *   mu_m = u / ||u||, 10m+8 gives kappa_m = softplus, 10m+9 the mixture
 *   logit.  targets: B x T x 8 unit vectors.  loss_out (1 double, device):
 *   mean over the B T targets of -log sum_m pi_m C_8(kappa_m)
 *   exp(kappa_m mu_m . x), C_8(kappa) = kappa^3 / ((2 pi)^4 I_3(kappa));
 *   dO (B x 160 floats): its gradient.  FP64 inside.
 * lrq_vmf_sample: S draws per instance from the mixture of O (component by
 *   weight, Wood's rejection method for the cosine to mu, a uniform
 *   direction orthogonal to mu), each multiplied by omega^k with k uniform
 *   in [0, K); C_out: B x S x 4 complex64.  Philox4x32-10 keyed by seed with
 *   counter (s, b, draw, 0x564D46).  A rejection loop that failed 1000 times
 *   (never observed) reports LRQ_ETIMEOUT.
 * lrq_vmf_modes: the 16 component means mu_m of the mixture of O (u / ||u||;
 *   e_1 when u = 0) as directions of C^4, ordered by mixture weight (largest
 *   logit first, lower component index on ties): C_out B x 16 x 4 complex64
 *   (device).  These are the proposal's most probable directions; a stream
 *   that starts with them and continues with lrq_vmf_sample draws is the
 *   learned stream of the evaluation.  B in [1, 65535].
 * lrq_adam_step: Adam with bias correction for step t >= 1 on count floats.
 * lrq_proposal_targets: training targets.  For each of the m indices idx[t]
 *   (device int64, in [0, S); the scoring's top-m selection, e.g. the top 1%
 *   of S uniform directions) the direction c = C[idx[t]] (C: S x r
 *   complex64, device) is moved to the canonical window -- c omega^-k with
 *   k = ceil(K arg(c_1) / (2 pi) - 1/2), so that arg c_1 lies in
 *   (-pi/K, pi/K] (Sec. 2.3: c and omega^k c score the same) -- and written
 *   as 2r floats (Re c_1, Im c_1, Re c_2, ...) to targets_out (m x 2r,
 *   device).  FP64 inside.  An index outside [0, S) reports LRQ_EINVAL in
 *   dev_status and writes zeros.
 * lrq_standardize_fit: per feature f of feat (B x F floats, device) the mean
 *   over the B rows and the sample standard deviation (ddof 1, at least
 *   1e-6; 1 when B = 1), FP64 sums, to mean_out and std_out (F floats each).
 * lrq_standardize: X_out[b][f] = (feat[b][f] - mean[f]) / std_dev[f] (B x F
 *   floats, device): the network's input.
 * ------------------------------------------------------------------------ */
int lrq_proposal_num_features(int r);
int64_t lrq_proposal_num_params(int F);
int lrq_proposal_features(const void* V, int B, int64_t n, int r, const double* lambda, void* Vg_out,
                          float* feat_out, int32_t* dev_status, void* stream);
int lrq_mlp_forward(const float* params, int F, int B, const float* X, float* H1, float* H2, float* O, int bf16,
                    void* stream);
int lrq_mlp_backward(const float* params, int F, int B, const float* X, const float* H1, const float* H2,
                     const float* dO, float* grads, float* scratch, int bf16, void* stream);
int lrq_vmf_nll(const float* O, int B, const float* targets, int T, double* loss_out, float* dO, void* stream);
int lrq_vmf_sample(const float* O, int B, int S, int K, uint64_t seed, void* C_out, int32_t* dev_status,
                   void* stream);
int lrq_vmf_modes(const float* O, int B, void* C_out, void* stream);
int lrq_adam_step(float* params, const float* grads, float* m, float* v, int64_t count, int t, float lr,
                  float beta1, float beta2, float eps, void* stream);
int lrq_proposal_targets(const void* C, int64_t S, int r, int K, const int64_t* idx, int64_t m, float* targets_out,
                         int32_t* dev_status, void* stream);
int lrq_standardize_fit(const float* feat, int B, int F, float* mean_out, float* std_out, void* stream);
int lrq_standardize(const float* feat, int B, int F, const float* mean, const float* std_dev, float* X_out,
                    void* stream);

/* --------------------------------------------------------------------------
 * lrq_cut_count -- exact Max-K-Cut value of an assignment on a graph.
 *
 * Sec. 1: for K = 3 and Q the graph Laplacian the problem is Max-3-Cut.
 * cut(z) = #{ undirected edges {i, j} : k_i != k_j }, counted exactly in
 * int64 from a symmetric CSR adjacency (each edge stored in both rows; self
 * loops never count).  With unit weights and K = 3, z^H L z = 3 cut(z),
 * since |z_i - z_j|^2 is 3 for different labels and 0 otherwise.
 *
 *   rowptr : n+1 int32 (device), colidx : rowptr[n] int32 (device),
 *   z      : n uint8 codes (device), cut_out : 1 int64 (device), written.
 * ------------------------------------------------------------------------ */
int lrq_cut_count(const int32_t* rowptr, const int32_t* colidx, int64_t n, const uint8_t* z,
                  int64_t* cut_out, void* stream);

/* --------------------------------------------------------------------------
 * lrq_greedy_cut -- greedy local search for Max-K-Cut, in place (the
 * refinement step of the hybrid solver, App. "Hybrid Warm-Start": greedy
 * hill-climbing started from the rank-1 partition, e.g. zcut_out of
 * lrq_rank1_sweep).
 *
 * Vertex i with neighbour counts n_i(c) = #{j in N(i), j != i : k_j = c}
 * gains g_i = n_i(k_i) - min_{c != k_i} n_i(c) by moving to that label (ties
 * to the smallest label).  Every round moves, simultaneously, each vertex
 * with g_i > 0 that no neighbour with positive gain outranks in the order
 * (larger gain, then smaller index).  The moved vertices are pairwise
 * non-adjacent, so the cut rises by exactly the sum of their gains, and the
 * steepest single move is always among them.  Rounds repeat until one moves
 * nothing (a state no single move improves) or max_rounds have run.  The
 * result is deterministic.
 *
 *   rowptr, colidx, nnz : undirected graph, symmetric CSR int32 (device),
 *              each edge in both rows, self loops ignored, parallel edges
 *              counted with their multiplicity.
 *   z        : n uint8 labels in [0, K) (device), read and overwritten.
 *   max_rounds : >= 0.
 *   cut_out  : 1 int64 (device) receives the final cut, or NULL.
 *   rounds_out, moves_out : host int64, rounds that moved and vertices
 *              moved in total, or NULL.  converged_out : host int32, 1 when
 *              a round found no move, 0 when max_rounds stopped the search
 *              first, or NULL.
 *   ws       : lrq_greedy_workspace_size(n) bytes.
 * Limits: 1 <= n < 2^31, 2 <= K <= 8.  Synchronises `stream` once per 8
 * rounds.  A label >= K, a column index outside [0, n) or a row range
 * outside [0, nnz] -> LRQ_EINVAL (returned; *dev_status holds it too).
 * ------------------------------------------------------------------------ */
int lrq_greedy_workspace_size(int64_t n, size_t* bytes);
int lrq_greedy_cut(const int32_t* rowptr, const int32_t* colidx, int64_t n, int64_t nnz, int K, uint8_t* z,
                   int64_t max_rounds, int64_t* cut_out, int64_t* rounds_out, int64_t* moves_out,
                   int32_t* converged_out, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream);

/* --------------------------------------------------------------------------
 * Measurement hooks (no counterpart in the paper).
 *
 * lrq_set_timing_events: for the calling thread, makes every later scoring
 * call (lrq_sample_score) record `start_event` just before and `stop_event`
 * just after its main scoring kernel, on the call's stream.  Both are
 * cudaEvent_t handles passed as void*, created by the caller; NULL, NULL
 * turns the hook off.  Lets a benchmark time the dominant kernel alone.
 *
 * lrq_kernel_launches: number of CUDA kernels this library has launched in
 * the process so far (all threads).
 * ------------------------------------------------------------------------ */
int lrq_set_timing_events(void* start_event, void* stop_event);
uint64_t lrq_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* LRQ_H */
