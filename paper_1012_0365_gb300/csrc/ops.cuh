// Internal operations of the BLWS library (host launchers of the kernels).
// All matrices are column-major FP64 unless a name says otherwise.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace blws {

// C = alpha op(A) op(B) + beta C, op = transpose when ta / tb.  M x N result,
// inner size K.  beta == 0 never reads C.  Split-K partial sums are reduced
// in a fixed order (deterministic).  fp32: products and in-CTA sums in FP32
// (at most 256 terms each), FP64 in and out (mixed-precision mode).
// In a BLWS_PREC_FP64_TC context the FP64 products of at least kOzGemmMin
// multiply-adds go to oz_gemm (FP64-equivalent digit products on the tensor
// cores); smaller ones stay on the FP64 pipe.
blws_status gemm(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int M, int N, int K,
                 double alpha, const double* A, int lda, const double* B, int ldb,
                 double beta, double* C, int ldc, bool fp32 = false);
// C = alpha op(A) op(B) (n x n) for a product known to be symmetric, such as
// X^T (T X) with T symmetric: the tiles of one triangle are computed and
// mirrored, so C is exactly symmetric.  (gemm does the same by itself for
// A^T A.)
blws_status gemm_sym(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int n, int K, double alpha,
                     const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                     bool fp32 = false);
// sym: the product is known to be symmetric (M = N, beta = 0): the result is
// made exactly symmetric (each element below the diagonal from its mirror)
blws_status oz_gemm(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                    const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                    bool sym = false);
constexpr double kOzGemmMin = 8.0e6;

// sum of squares of an M x N matrix (ld) into *out (device), deterministic
blws_status sumsq(Ctx* ctx, cudaStream_t s, int M, int N, const double* A, int ld, double* out);

// out[j] = ||A(:, j)||_2 for j < N; and *colmax = max_j out[j] (device)
blws_status col_norms(Ctx* ctx, cudaStream_t s, int M, int N, const double* A, int ld,
                      double* out, double* colmax);

// Symmetric eigen-decomposition of the n x n FP64 matrix T (ld n):
// lam (n, decreasing) and Z (n x n, ld n, columns in the same order).
// Eigenvalue clusters that reach above eps - 3 d (d the first level's
// resolution) are re-solved on their own (see eig.cu).  Synchronises s once.
blws_status sym_eig(Ctx* ctx, cudaStream_t s, int n, const double* T, double* lam, double* Z,
                    double eps);
// sym_eig in two stages around the synchronisation: the device stage (no
// host wait; it ends with copies of what the host stage reads into pinned
// host memory), then, once s has been synchronised, the host stage (the
// fallback and the cluster re-solve, which launch and synchronise only when
// they apply).  sym_eig = sym_eig_start, synchronise, sym_eig_finish.
blws_status sym_eig_start(Ctx* ctx, cudaStream_t s, int n, const double* T, double* lam, double* Z);
// one double after the host copies of sym_eig_start (n): for a caller's own
// value copied back with them
double* sym_eig_host_extra(Ctx* ctx, int n);
blws_status sym_eig_finish(Ctx* ctx, cudaStream_t s, int n, const double* T, double* lam, double* Z,
                           double eps);

// FP32 eigenvectors of T (n x n FP64, symmetric) by the tridiagonal route
// (tri_eig.cu): X (n x n FP64, ld n) receives them, columns in increasing
// order of eigenvalue, with FP32 accuracy.  Eigenvalues closer than
// kTriGroupTol ||T|| to a neighbour form a group whose columns are an
// orthonormal basis of the group's joint eigenspace, not eigenvectors one by
// one: grp[j] (device, n ints) is the group's first column, or -1 for a
// column alone, and gtop[j] (device, n floats) the group's largest
// eigenvalue as the FP32 stage found it (within ~1e-6 ||T||).  *fail
// (device int) is set when a group could not be orthonormalised or a solve
// normalised (X is then not to be used).  n <= kTriMaxN: up to
// kTriOneCtaMaxN the packed lower triangle fits one CTA's shared memory;
// larger matrices are reduced on a thread-block cluster of 4 or 8 CTAs
// (tri_fits tells whether this GPU's shared memory holds a cluster's share).
constexpr int kTriOneCtaMaxN = 336;
constexpr int kTriMaxN = 736;
bool tri_fits(Ctx* ctx, int n);
constexpr float kTriGroupTol = 1e-4f;
blws_status tri_stage(Ctx* ctx, cudaStream_t s, int n, const double* T, double* X, int* grp, float* gtop,
                      int* fail);

// CholeskyQR2 with column equilibration and deflation: on return X (N x b,
// ld) holds an orthonormal basis of span(R) with dead columns zeroed and
// B (b x b upper, ld b) satisfies R = X B (dead rows zero).  R is destroyed.
// `scale` (device scalar) and `tol`: a column dies when its diagonal of B is
// <= tol * scale.  `tmp` is an N x b scratch array (ld).
// fp32: the four tall products (Gram matrices, X = R S) in FP32 arithmetic;
// the b x b factorisation stays FP64.  one_pass: R's columns are known to be
// orthonormal to rounding already (a warm start made of the previous call's
// Ritz vectors), so a first pass -- whose Gram matrix is then I + E with E at
// the rounding level, factored exactly by the near-identity rule -- already
// leaves X as orthonormal as a second one would; the second is skipped.
blws_status chol_qr2(Ctx* ctx, cudaStream_t s, int N, int b, double* R, int ld,
                     double* X, double* tmp, double* B, const double* scale, double tol,
                     bool fp32 = false, bool one_pass = false);

// ------------------------------------------- tensor-core products (tc_gemm)
// A matrix as two TF32 planes (hi + lo) in FP32 containers, K-major:
// element (r, k) at r * ld + k, ld = tc_ld(inner) (a multiple of 32).
struct TcPlanes {
  float* hi;
  float* lo;
  int rows, inner, ld;
};
int tc_ld(int inner);
// padded accumulator width for b columns (0 when b > 256)
int tc_npad(int b);
// planes of the column-major rows x inner slab: plane(r, k) = A[row0 + k + r lda]
blws_status tc_planes_from_cols(Ctx* ctx, cudaStream_t s, const double* A, int lda, int row0, int inner,
                                int rows, const TcPlanes& out);
// transposed planes of the m x n column-major A: plane(i, j) = A[i + j lda]
blws_status tc_planes_from_rows(Ctx* ctx, cudaStream_t s, const double* A, int lda, int m, int n,
                                const TcPlanes& out);
// C = alpha op(A) op(B) + beta C from split TF32 operands on the tensor cores
// (mixed-precision block products; any N, 256 columns per launch); sym: the
// product is known to be symmetric and C is made exactly so (N <= 256)
blws_status tc_gemm(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                    const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                    bool sym = false);
constexpr double kTcGemmMin = 4.0e6;
// P = [W X_v; W^T X_u] (FP64 out) from W's row-major planes Wr (m rows) and
// column-major planes Wc (n rows); X is (m+n) x b FP64, b <= 256.
blws_status tc_dual_apply(Ctx* ctx, cudaStream_t s, const TcPlanes& Wr, const TcPlanes& Wc, int m,
                          int n, const double* X, int ldx, int b, double* P, int ldp);

// ---------------------------------- FP64-equivalent tensor-core products (tc_ozaki)
// A matrix as S BF16 planes of balanced base-128 digits with one power-of-two
// scale per row: plane t, element (r, k) at d[t rows ld + r ld + k]; e[r] the
// scale exponent of row r.  ld = oz_ld(inner) (a multiple of 64).
struct OzPlanes {
  __nv_bfloat16* d;
  int* e;
  int rows, inner, ld;
};
int oz_ld(int inner);
int oz_digits();
// digit planes of an m x n W in both orientations, in the context's workspace
blws_status oz_alloc(Ctx* ctx, int m, int n, OzPlanes* Or, OzPlanes* Oc);
// transposed digit planes of the m x n column-major A (rows of A, scale per row)
blws_status oz_planes_from_rows(Ctx* ctx, cudaStream_t s, const double* A, int lda, int m, int n,
                                const OzPlanes& out);
// digit planes of the column-major slab (row r of the planes = column r of A,
// K along A's rows row0 .. row0 + inner; scale per column)
blws_status oz_planes_from_cols(Ctx* ctx, cudaStream_t s, const double* A, int lda, int row0, int inner,
                                int rows, const OzPlanes& out);
// P = [W X_v; W^T X_u] (FP64 out, errors at the FP64 level) from W's digit
// planes in both orientations (Wr: m rows, Wc: n rows).
blws_status oz_dual_apply(Ctx* ctx, cudaStream_t s, const OzPlanes& Wr, const OzPlanes& Wc, int m, int n,
                          const double* X, int ldx, int b, double* P, int ldp);

// Bounded-wait self-test: one CTA waits on an mbarrier nothing arrives at,
// through the tensor-core kernels' bounded wait with `polls` polls, and sets
// SLOT_TCERR when the wait gives up (the path a stalled copy or MMA takes).
blws_status wait_probe(Ctx* ctx, cudaStream_t s, unsigned polls);

}  // namespace blws
