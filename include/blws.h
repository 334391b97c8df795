/* blws.h -- C ABI of the GB300 (sm_103a) block-Lanczos-with-warm-start library.
 *
 * Method: Lin & Wei, "A Block Lanczos with Warm Start Technique for
 * Accelerating Nuclear Norm Minimization Algorithms".  Every nuclear-norm
 * solver evaluates, once per iteration, the singular value thresholding
 *     A = T_eps(W) = U Theta_eps(S) V^T,  Theta_eps(x) = sgn(x) max(|x|-eps, 0)
 * (Section 1, Eq. (3)-(4)).  BLWS computes the needed partial SVD by block
 * Lanczos on the augmented matrix [[0, W], [W^T, 0]] (Theorem 1, Eq. (7)),
 * restarted from the previous iteration's singular subspaces (Section 4,
 * "BLWS"; mixed start of Section 4.1) for a few blocks only (Section 4.1),
 * with the number of output pairs following the predicted rank (Section 4.2).
 *
 * Conventions for every entry point:
 *   - Matrices are column-major (LAPACK order) with an explicit leading
 *     dimension; all array arguments are DEVICE pointers owned by the caller
 *     unless the comment says "host".  The library never frees them.
 *   - Scalars are FP64.  Sparse indices are 0-based int32 (CSR).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  All device work of a call is enqueued on it.  The
 *     solvers and blws_svt synchronise `stream` before returning, because
 *     they return host-side results (counts, iteration info).
 *   - The library owns its workspace (grown on demand, freed by
 *     blws_destroy).  A context is not thread-safe: use one context per host
 *     thread / stream.
 *   - No exception crosses the ABI.  A negative return is an error; the
 *     message of the last error is available from blws_last_error().
 */
#ifndef BLWS_H
#define BLWS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int blws_status;
#define BLWS_OK 0
#define BLWS_EINVAL (-1)      /* bad argument (size, pointer, parameter) */
#define BLWS_ENOMEM (-2)      /* device allocation failed */
#define BLWS_ECUDA (-3)       /* a CUDA call or kernel launch failed */
#define BLWS_ENOCONV (-4)     /* a solver hit max_iter before its tolerance */
#define BLWS_ENONFINITE (-5)  /* NaN/Inf met in an input or an iterate */
#define BLWS_ETIMEOUT (-6)    /* a bounded device wait gave up */
#define BLWS_ENOTSUP (-7)     /* requested mode not built for this device */

/* Arithmetic of the block products (a2, a9).  The small steps (Cholesky of
 * the Gram matrix, the eigenproblem of T_k, the count of values above eps)
 * are FP64 in every mode. */
#define BLWS_PREC_FP64 0      /* all arithmetic FP64 */
/* Mixed: products with a dense W on the tensor cores from split TF32
 * operands (hi + lo, three products, FP32 accumulation over at most 256
 * terms, FP64 sums beyond); the other block products (Gram matrices, block
 * coefficients, residuals, Ritz lift) and the RPCA reconstruction in FP32
 * arithmetic with FP64 sums.  Products that need FP64 accuracy (the eigen
 * stage's refinement, block widths above 256, and every block product of
 * the refinement tail: rpca_solve returns to FP64-level products once its
 * residual falls below rpca_params.mixed_tol) run as in BLWS_PREC_FP64_TC:
 * BF16 digit-plane products from 8e6 multiply-adds, FP64 below.  Sparse
 * operators keep FP64 products. */
#define BLWS_PREC_MIXED 1
/* FP64-equivalent products on the tensor cores (dense W only): every row of W
 * and every column of X is written as 7 balanced base-128 digits under one
 * power-of-two scale (exact in BF16); the 28 digit products with the leading
 * weights are formed by tensor cores with exact FP32 sums (256 terms at a
 * time) and combined in double-FP32 / FP64.  Error ~2^-47 of the leading
 * term per product term, against the DFMA GEMM's ~2^-53.  Everything else
 * is FP64, as in BLWS_PREC_FP64. */
#define BLWS_PREC_FP64_TC 2

typedef struct blws_ctx blws_ctx;

typedef struct {
  int k;          /* Lanczos blocks per warm-started call (paper's k, Section
                     4.1; the paper typically uses 2).  Default 3. */
  int k_cold;     /* blocks for a cold start (no previous subspace), run with
                     full reorthogonalisation.  Default 4. */
  int precision;  /* BLWS_PREC_* ; default BLWS_PREC_FP64 */
  uint64_t seed;  /* seed of the counter-based generator (Philox4x32-10) that
                     draws extra start columns.  Default 0x5eed. */
  int device;     /* CUDA device ordinal the context binds to.  Default 0. */
  int start;      /* warm-start block of blws_svt, rpca_solve and mc_solve
                     (Section 4.1; blws_evd has a single subspace and ignores it):
                     0 (default) the mixed start [U; V]/sqrt(2), 1 the
                     standard start [U; 0] the paper compares it with. */
  int warm;       /* 1 (default): every outer iteration of rpca_solve /
                     mc_solve restarts from the previous iteration's singular
                     subspaces (BLWS); 0: every call is a cold start (k_cold
                     blocks from a seeded Gaussian block, full
                     reorthogonalisation), the random-start block Lanczos the
                     paper compares against.  Variants for ablations. */
  int grid_sms;   /* SMs the context sizes its grids and K splits for: 0
                     (default) all of the device's SMs.  A smaller share lets
                     solves on concurrent streams run side by side instead of
                     each filling the GPU in turn (the server's workers). */
  int graphs;     /* 1 (default): rpca_solve captures the two phases of an
                     outer iteration (the block steps up to the eigen-solver's
                     device stage; the Ritz lift and fused epilogue) in CUDA
                     graphs and replays them with one launch each while their
                     launches repeat (once the predicted rank settles); 0:
                     every kernel is launched directly.  The same kernels run
                     with the same arguments either way: results are
                     bit-identical.  The environment variable BLWS_GRAPH=0 at
                     context creation turns it off. */
  int tune;       /* 0 (default): FP64 / FP32 CUDA-core products take their
                     tile shape and K split from a fixed rule (least padding,
                     about 8 CTAs per SM).  1: from a timed autotuner -- the
                     first product of each size bucket (every dimension rounded
                     up to a quarter octave) times every (tile, split) pair
                     and keeps the fastest unless the rule is within 5%.
                     Choices are process-wide; with the environment variable
                     BLWS_TUNE_FILE set they are read from and appended to
                     that file.  Products differ from the rule's in rounding
                     only (the split-K sums are grouped differently). */
  double guard;   /* Ritz-residual guard of rpca_solve and mc_solve: 0
                     (default) off.  > 0: every BLWS call also forms the
                     residual of its last block, whose Gram matrix gives each
                     Ritz pair's residual ||W~ y - theta y|| (the block Lanczos
                     relation); when a pair above the threshold has a residual
                     above guard x the largest Ritz value, the call is run
                     again from the same start with one more block, at most
                     twice per outer iteration (rpca_info / mc_info .restarts
                     counts them).  A guard against inaccurate partial SVDs
                     in rank-growth transients; it costs one residual product
                     and one Gram matrix per call. */
} blws_config;

/* Fill *cfg with the defaults above.  Never fails for a non-NULL cfg. */
blws_status blws_config_default(blws_config* cfg);

/* Create a context bound to cfg->device (cfg NULL: defaults).  *ctx receives
 * the handle; release it with blws_destroy. */
blws_status blws_create(blws_ctx** ctx, const blws_config* cfg);
blws_status blws_destroy(blws_ctx* ctx);

/* Number of kernels this context has launched so far (host counter, exact). */
uint64_t blws_launch_count(const blws_ctx* ctx);

/* CUDA graphs of this context so far (blws_config.graphs): phases captured
 * and phase replays (each replay launched the captured kernels with one graph
 * launch; blws_launch_count counts those kernels too).  Either pointer may be
 * NULL.  Never fails for a non-NULL ctx. */
blws_status blws_graph_stats(const blws_ctx* ctx, uint64_t* captures, uint64_t* replays);

/* Size buckets the product autotuner (blws_config.tune) holds in this
 * process, read from BLWS_TUNE_FILE or measured.  Never fails. */
size_t blws_tune_count(void);

/* Text of a status code (static string). */
const char* blws_status_str(blws_status s);
/* Message of the last error recorded on ctx (static per ctx; "" if none). */
const char* blws_last_error(const blws_ctx* ctx);

/* The operator W (m x n) of one SVT evaluation.
 *   dense:  W != NULL, column-major with leading dimension ldw >= m.
 *   sparse: W == NULL, CSR (rowptr[m+1], colidx[nnz], val[nnz]) plus an
 *           optional low-rank term Ul diag(sl) Vl^T (rl columns, Ul m x rl
 *           with ld m, Vl n x rl with ld n; rl = 0 means none).  This is the
 *           "sparse residual plus low-rank" input of matrix completion.
 *           W^T X needs the pattern by columns: colptr/rowidx/perm may give
 *           a mirror built by blws_csc_mirror for this pattern (reused across
 *           calls); NULL (default) builds one in the context at each call. */
typedef struct {
  int m, n;
  const double* W;
  int ldw;
  int nnz;
  const int* rowptr;
  const int* colidx;
  const double* val;
  int rl;
  const double* Ul;
  const double* sl;
  const double* Vl;
  const int* colptr;   /* optional CSC mirror: n + 1 column pointers */
  const int* rowidx;   /* nnz row indices, rows increasing within a column */
  const int* perm;     /* nnz: CSC entry e is CSR entry perm[e] */
} blws_op;

/* The column-major mirror of a CSR pattern (m x n, nnz entries): colptr
 * (n + 1), rowidx (nnz) and perm (nnz), caller-owned device arrays, written
 * on `stream`; within each column the rows increase (deterministic).  For
 * callers that apply the same sparse operator many times (blws_op.colptr).
 * Does not synchronise. */
blws_status blws_csc_mirror(blws_ctx* ctx, int m, int n, int nnz, const int* rowptr,
                            const int* colidx, int* colptr, int* rowidx, int* perm,
                            void* stream);

/* One SVT evaluation T_eps(W) by BLWS (Sections 4, 4.1, 4.2; Eq. (4)).
 *
 *   eps     threshold (> 0).
 *   r       Ritz pairs to output (the predicted rank), 1 <= r <= min(m, n).
 *   U0, V0  warm start: the previous principal subspaces, m x w and n x w
 *           (ld m and n); w = 0 means cold start (U0, V0 ignored).
 *   G, g    optional extra start columns ((m+n) x g, ld m+n) appended after
 *           the warm block; when G == NULL and r > w the library draws
 *           b - w = r - w (cold start: r) columns itself with its seeded
 *           generator.  The block width is b = max(r, w + g).
 *   U, V    out: the r leading Ritz vectors as left/right singular vectors,
 *           m x r and n x r (ld m and n), the sqrt(2)-scaled halves of the
 *           Ritz vectors of the augmented matrix (Theorem 1).
 *   sigma   out: the r leading Ritz values, decreasing.
 *   count   out (host): #{sigma_t > eps}; A = U[:, :c] diag(sigma - eps) V^T.
 *   Requires 1 <= r <= b and k*b <= m + n (k the context's block count, or
 *   k_cold on a cold start).  The call synchronises `stream`. */
blws_status blws_svt(blws_ctx* ctx, const blws_op* W, double eps, int r,
                     const double* U0, const double* V0, int w,
                     const double* G, int g,
                     double* U, double* V, double* sigma, int* count,
                     void* stream);

/* Partial EVD of a symmetric W by block Lanczos with warm start: the BLWS
 * definition of Section 4, (U_i, Lambda_i) = BL_EVD(W_i, U_{i-1}, k), i.e.
 * Algorithms 2 and 3 run on W itself rather than on the augmented matrix.
 *   W       m x m symmetric, dense FP64 column-major, ld ldw >= m (device);
 *           the products read all of W (P = W X), so both triangles must
 *           hold the matrix.
 *   eps     finite; count = #{lambda_t > eps} (the eigenvalues an
 *           eigenvalue thresholding at eps keeps).
 *   r       Ritz pairs to output, 1 <= r <= m: the r largest (algebraic).
 *   U0, w   warm start: the previous principal eigen-subspace, m x w (ld m);
 *           w = 0 means cold start (k_cold blocks, full reorthogonalisation).
 *   G, g    optional extra start columns, m x g (ld m), after the warm ones;
 *           when G == NULL and r > w the library draws them.  The block
 *           width is b = max(r, w + g).
 *   U       out: m x r (ld m) Ritz vectors, orthonormal columns.
 *   lam     out: the r leading Ritz values, decreasing.
 *   count   out (host).
 *   Requires k*b <= m.  The context's precision applies as for blws_svt
 *   (digit-plane tensor-core products for large ones in the FP64-equivalent
 *   mode; FP32 tall products in the mixed mode).  The call synchronises
 *   `stream`.  Errors: BLWS_EINVAL for bad sizes or missing pointers (nothing
 *   launched), BLWS_ECUDA for a failed launch or copy. */
blws_status blws_evd(blws_ctx* ctx, const double* W, int m, int ldw, double eps, int r,
                     const double* U0, int w, const double* G, int g,
                     double* U, double* lam, int* count, void* stream);

/* Step a2 alone: P = W~ X for the augmented matrix without forming it
 * (Section 4, end): P[0:m] = W X[m:m+n], P[m:m+n] = W^T X[0:m].
 *   X   (m+n) x b, leading dimension ldx >= m+n (device, FP64)
 *   P   (m+n) x b, leading dimension ldp >= m+n (device, FP64, output)
 * The building block every BLWS step repeats k times; exported so callers
 * (and benchmarks) can run and time it on its own.  Does not synchronise, so
 * a bounded tensor-core wait that gives up inside it (BLWS_ETIMEOUT from the
 * calls that synchronise) is not reported by this call. */
blws_status blws_apply(blws_ctx* ctx, const blws_op* W, const double* X, int ldx, int b,
                       double* P, int ldp, void* stream);

/* blws_apply for a dense W, without allocating anything.  (The paper has no
 * counterpart: this is a deployment variant of step a2.)
 *
 * For callers that cannot call cudaMalloc: code running inside another
 * framework's memory pool or a plugin host that forbids its own device
 * allocations, code that must not trigger the implicit device
 * synchronisation an allocation or free can cause, or code that may not
 * create a blws_ctx (creating one allocates its workspace).
 *
 * Computes P[0:m] = W X[m:m+n] and P[m:m+n] = W^T X[0:m] with the same
 * kernels as blws_apply for a dense operator; it splits the inner dimension
 * less finely (for about two CTAs per SM), so the two agree to rounding.  W is m x n (ld ldw >= m), X and P are (m+n) x b (ld ldx,
 * ldp >= m+n), all device FP64 owned by the caller.  No context is needed.
 *
 * Scratch: the split-K partial sums live in one 16 MiB array
 * (2,097,152 doubles) that the library declares statically; every GPU that
 * loads the library holds it until the process exits.  A product of r rows
 * needs s * r * b doubles of it, where s is the split-K factor the library
 * picks to fill the GPU (s = 1, i.e. no scratch, once the product has at
 * least two tiles per SM).  If either product would need more than the
 * array holds, the call returns BLWS_EINVAL before launching anything.
 * Every element the call reads from the array was written by the same call,
 * so nothing needs clearing between calls.
 *
 * Every call looks up the array's device address in the calling thread's
 * current context (a lookup, no allocation or synchronisation), so the
 * address is never stale after cudaDeviceReset and is right for a caller
 * that runs in its own driver-API context.  The first call on a device also
 * loads the library's device code and reads the SM count; make that first
 * call before any stream capture.  All calls share the one array: calls that
 * can overlap on the GPU (different streams, or different host threads) race
 * on it and must be serialised by the caller.
 *
 * Returns BLWS_OK, BLWS_EINVAL (bad pointer or size, or scratch need above
 * the maximum), BLWS_ECUDA (a launch or the set-up failed) or BLWS_ENOTSUP
 * (device ordinal >= 64).  Does not synchronise. */
blws_status blws_apply_noalloc(const double* W, int m, int n, int ldw, const double* X, int ldx,
                               int b, double* P, int ldp, void* stream);

/* The dense block product every step of Algorithms 2 and 3 is built from
 * (P = W~ X, M_l = X_l^T P_l, R_l = P_l - X_l M_l - X_{l-1} B_{l-1}^T, the
 * CholeskyQR2 Gram matrices, the Ritz lift Q_k Z of Algorithm 3, and the
 * refinement products of the T_k eigen-solver), exported with the
 * arithmetic the context's precision gives it inside the procedure:
 *   C = alpha op(A) op(B) + beta C,  op(X) = X^T when ta / tb is nonzero;
 *   C is M x N, the inner size is K; A, B, C device FP64 column-major with
 *   lda >= (ta ? K : M), ldb >= (tb ? N : K), ldc >= M.  beta == 0 never
 *   reads C.
 *   sym != 0: the product is known to be symmetric (A^T A, or X^T (T X) with
 *   T symmetric); one triangle of tiles is computed and mirrored, so C is
 *   exactly symmetric.  Needs M == N and beta == 0.
 * In a BLWS_PREC_FP64_TC context products of at least 8e6 multiply-adds run
 * as BF16 digit-plane products on the tensor cores (FP64-equivalent), the
 * rest on the FP64 pipe; BLWS_PREC_MIXED uses FP32 arithmetic with FP64
 * sums; BLWS_PREC_FP64 is FP64 throughout.  Synchronises `stream`.  Returns
 * BLWS_EINVAL for bad sizes (nothing launched), BLWS_ETIMEOUT if a bounded
 * tensor-core wait gave up, BLWS_ECUDA for a failed launch. */
blws_status blws_gemm(blws_ctx* ctx, int ta, int tb, int M, int N, int K, double alpha,
                      const double* A, int lda, const double* B, int ldb, double beta, double* C,
                      int ldc, int sym, void* stream);

/* Device timing of step a2 (Section 4, end: the product P = W~ X with the
 * zero blocks skipped), the dominant step of the procedure.  After
 * blws_timing_start, every product with a dense W that this context runs
 * (inside blws_svt, blws_evd, blws_apply, rpca_solve) is bracketed by a pair
 * of CUDA events on its stream, around the product's kernel (the digit-plane
 * kernel in BLWS_PREC_FP64_TC, the TF32x3 kernel in BLWS_PREC_MIXED, both FP64
 * GEMMs and their split-K reduction in BLWS_PREC_FP64).  blws_timing_stop
 * waits for the last event and returns the summed device time (*ms), the
 * number of products (*launches) and their multiply-adds (*work = sum of
 * 2 m n b: both halves of each product).  Recording costs two event records
 * per product; timing is off by default. */
blws_status blws_timing_start(blws_ctx* ctx);
blws_status blws_timing_stop(blws_ctx* ctx, double* ms, uint64_t* launches, double* work);
/* The per-product records of the last blws_timing_stop: ms[i] (device
 * time), work[i] (2 m n b) and kind[i] (the kernel that computed it: 0 FP64
 * DFMA GEMMs, 1 split-TF32 tensor-core products, 2 BF16 digit-plane
 * tensor-core products) for i < min(cap, count), host arrays (any may be
 * NULL); products launched directly come first, in launch order, then those
 * timed inside replayed CUDA graphs.  Returns the count. */
size_t blws_timing_records(const blws_ctx* ctx, size_t cap, double* ms, double* work, int* kind);

/* Self-test of the bounded waits (no counterpart in the paper).  Every wait
 * of the tensor-core kernels (a TMA copy or an MMA that should complete) is
 * capped; when a cap is reached the kernel raises an error word and returns,
 * and the calls that synchronise report BLWS_ETIMEOUT.  This call launches
 * one small kernel that waits, through the same bounded wait, on a barrier
 * nothing arrives at, with a cap of `polls` polls (1 .. 65536, well under a
 * millisecond); it returns BLWS_ETIMEOUT, which shows the path from a wait
 * that gives up to the status a caller sees.  No copy, MMA or tensor memory
 * is involved.  Synchronises `stream`. */
blws_status blws_wait_probe(blws_ctx* ctx, unsigned polls, void* stream);

/* Robust PCA (Section 5, Table 1): min ||A||_* + lambda ||E||_1 s.t. D = A+E
 * by inexact ALM with every SVT evaluated by BLWS. */
typedef struct {
  double lambda;   /* <= 0: 1/sqrt(max(m, n)) */
  double tol;      /* stop when ||D - A - E||_F / ||D||_F < tol.  Default 1e-7 */
  int max_iter;    /* default 1000 */
  double rho;      /* mu growth factor, default 1.5 */
  double mu0;      /* <= 0: 1.25 / ||D||_2 */
  double mu_bar_ratio; /* mu cap = ratio * mu0, default 1e7 */
  int sv0;         /* initial predicted rank, default 10 */
  double* trace;   /* optional HOST array of 3 * trace_len doubles: per outer
                      iteration i < trace_len, (residual, count above eps,
                      predicted rank used).  NULL (default): no trace. */
  int trace_len;
  double mixed_tol; /* BLWS_PREC_MIXED contexts: iterations run with mixed
                      products while the residual is >= mixed_tol, FP64
                      after (0: never switch).  Default 1e-5. */
} rpca_params;

typedef struct {
  int iters;        /* outer iterations run */
  int rank;         /* #{sigma > 1/mu} at the last iteration = rank(A) */
  int64_t nnzE;     /* nonzeros of E */
  double residual;  /* ||D - A - E||_F / ||D||_F at exit */
  double norm_two;  /* the estimate of ||D||_2 used for mu0 and Y0 */
  int status;       /* BLWS_OK or BLWS_ENOCONV */
  int mixed_iters;  /* iterations that ran with mixed products */
  int restarts;     /* BLWS calls repeated with one more block (blws_config.guard) */
} rpca_info;

blws_status rpca_params_default(rpca_params* p);

/* D, A, E: m x n, column-major, common leading dimension ld >= m, FP64.
 * A and E are outputs (overwritten).  Returns BLWS_ENOCONV (with A, E the
 * last iterate and info filled) if max_iter is reached. */
blws_status rpca_solve(blws_ctx* ctx, const double* D, int m, int n, int ld,
                       const rpca_params* p, double* A, double* E,
                       rpca_info* info, void* stream);

/* Matrix completion (Section 5, Table 2) from the observed entries of M on
 * Omega (CSR, sorted column indices within a row, no duplicates).
 *   variant 0: SVT of [Cai08] (the paper's host): Y^0 = k0 delta P_Omega(M),
 *              X^k = T_tau(Y^{k-1}), Y^k = Y^{k-1} + delta P_Omega(M - X^k).
 *   variant 1: proximal / FPC form: W_k = X_k + delta P_Omega(M - X_k)
 *              (low-rank + sparse operator), X_{k+1} = T_tau(W_k) with tau
 *              continuation. */
typedef struct {
  int variant;      /* 0 SVT, 1 PROX */
  double tau;       /* <= 0: 5 sqrt(m n) (SVT); ignored by PROX */
  double delta;     /* <= 0: 1.2 m n / nnz (SVT); 1 (PROX) */
  double tol;       /* stop on ||P_Omega(X - M)||_F / ||P_Omega M||_F <= tol; default 1e-4 */
  int max_iter;     /* default 500 (SVT), 1000 (PROX) */
  int incr;         /* SVT rank increment l of [Cai08], default 5 */
  double eta;       /* PROX continuation factor, default 0.25 */
  double tau_min_rel; /* PROX floor tau_min = tau_min_rel * ||P_Omega M||_2, default 1e-4 */
  double xtol;      /* PROX: lower tau when ||dX||_F / max(1, ||X||_F) < xtol; default 1e-3 */
} mc_params;

typedef struct {
  int iters;
  int rank;         /* columns of the returned factors */
  double residual;  /* observed relative residual at exit */
  double norm_two;  /* the estimate of ||P_Omega M||_2 */
  int status;
  int restarts;     /* BLWS calls repeated with one more block (blws_config.guard) */
} mc_info;

blws_status mc_params_default(mc_params* p);

/* Output: X = U diag(theta) V^T with rank <= max_rank columns: U m x
 * max_rank (ld m), V n x max_rank (ld n), theta max_rank entries; columns
 * past info->rank are zero.  Returns BLWS_EINVAL if the rank would exceed
 * max_rank, BLWS_ENOCONV at max_iter. */
blws_status mc_solve(blws_ctx* ctx, int m, int n, int nnz, const int* rowptr,
                     const int* colidx, const double* vals,
                     const mc_params* p, int max_rank,
                     double* U, double* theta, double* V,
                     mc_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Serving and batching (no counterpart in the paper: a runtime around the
 * solvers).  A server owns `workers` host threads, each with its own context
 * (workspace, generator) and its own CUDA stream, on one device.  Requests
 * (Robust PCA or matrix completion, device buffers owned by the caller)
 * queue in arrival order; the head of the queue is admitted when a worker is
 * free and its estimated device memory (blws_request_bytes) fits in what the
 * admitted requests leave of the budget (a request larger than the whole
 * budget runs alone).  Admitted solves run concurrently on their streams, so
 * requests that arrive while others run overlap with them on the GPU.  Each
 * solve is the same computation as a direct rpca_solve / mc_solve call with
 * the server's configuration (fixed reduction orders: the result does not
 * depend on what else runs).  The caller must keep a request's buffers
 * alive and untouched until blws_server_wait has returned its result.
 * ---------------------------------------------------------------------- */
#define BLWS_REQ_RPCA 0
#define BLWS_REQ_MC 1

typedef struct blws_server blws_server;

typedef struct {
  int workers;          /* concurrent solves (host threads / streams), default 8 */
  size_t hbm_budget;    /* device bytes the admitted solves may hold; 0 (default):
                           70% of the free device memory at creation */
  blws_config cfg;      /* configuration of every worker context */
} blws_server_config;

typedef struct {
  int kind;             /* BLWS_REQ_RPCA or BLWS_REQ_MC */
  /* BLWS_REQ_RPCA: rpca_solve arguments */
  const double* D;
  int m, n, ld;
  rpca_params rpca;
  double* A;
  double* E;
  /* BLWS_REQ_MC: mc_solve arguments (m, n above) */
  int nnz;
  const int* rowptr;
  const int* colidx;
  const double* vals;
  mc_params mc;
  int max_rank;
  double* U;
  double* theta;
  double* V;
} blws_request;

typedef struct {
  int status;           /* the solver's status (BLWS_OK, BLWS_ENOCONV, ...) */
  double queue_ms;      /* submit -> admitted */
  double run_ms;        /* admitted -> finished (device work complete) */
  rpca_info rpca;       /* filled for BLWS_REQ_RPCA */
  mc_info mc;           /* filled for BLWS_REQ_MC */
} blws_result;

typedef struct {
  uint64_t submitted, completed;
  size_t budget, in_use, peak_in_use;  /* admission accounting, bytes */
  int peak_running;                     /* most solves admitted at once */
} blws_server_stats;

blws_status blws_server_config_default(blws_server_config* cfg);
/* Start the workers (each creates its context on cfg->cfg.device). */
blws_status blws_server_create(blws_server** srv, const blws_server_config* cfg);
/* Estimated device bytes of a request's solve (its admission weight). */
size_t blws_request_bytes(const blws_request* req, int precision);
/* Queue a request (copied); *ticket identifies it.  Never blocks on the GPU. */
blws_status blws_server_submit(blws_server* srv, const blws_request* req, uint64_t* ticket);
/* Block until the ticket's solve has finished; fills *out.  Each ticket can
 * be waited for once.  BLWS_EINVAL for an unknown ticket. */
blws_status blws_server_wait(blws_server* srv, uint64_t ticket, blws_result* out);
blws_status blws_server_stats_get(blws_server* srv, blws_server_stats* out);
/* Finish every queued request, stop the workers, free the contexts. */
blws_status blws_server_destroy(blws_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* BLWS_H */
