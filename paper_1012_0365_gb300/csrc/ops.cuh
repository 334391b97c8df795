// Internal operations of the BLWS library (host launchers of the kernels).
// All matrices are column-major FP64 unless a name says otherwise.
#pragma once
#include "common.cuh"

namespace blws {

// C = alpha op(A) op(B) + beta C, op = transpose when ta / tb.  M x N result,
// inner size K.  beta == 0 never reads C.  Split-K partial sums are reduced
// in a fixed order (deterministic).
blws_status gemm(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int M, int N, int K,
                 double alpha, const double* A, int lda, const double* B, int ldb,
                 double beta, double* C, int ldc);

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

// CholeskyQR2 with column equilibration and deflation: on return X (N x b,
// ld) holds an orthonormal basis of span(R) with dead columns zeroed and
// B (b x b upper, ld b) satisfies R = X B (dead rows zero).  R is destroyed.
// `scale` (device scalar) and `tol`: a column dies when its diagonal of B is
// <= tol * scale.  `tmp` is an N x b scratch array (ld).
blws_status chol_qr2(Ctx* ctx, cudaStream_t s, int N, int b, double* R, int ld,
                     double* X, double* tmp, double* B, const double* scale, double tol);

}  // namespace blws
