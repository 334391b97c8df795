// Matrix-completion building blocks shared by the sparse operator and mc_solve.
#pragma once
#include "blws_core.cuh"

namespace blws {

// CSC mirror (colptr[n+1], rowidx[nnz], perm[nnz]) of a CSR pattern, on the
// device, deterministic (segments sorted by row).
blws_status build_csc(Ctx* ctx, cudaStream_t s, int m, int n, int nnz, const int* rowptr,
                      const int* colidx, int** colptr, int** rowidx, int** perm);

// For every (i, j) in Omega: x = sum_{t<c} U_it th_t V_jt, r = mval - x;
// mode 0: y += delta r; mode 1: y = delta r.  *sumsq_out = sum r^2.
// Ut (m x c) and Vt (n x c) are scratch for row-major copies of U and V.
blws_status sddmm(Ctx* ctx, cudaStream_t s, int m, int n, int c, const int* rowptr,
                  const int* colidx, const double* mval, const double* U, int ldu,
                  const double* th, const double* V, int ldv, double delta, int mode, double* y,
                  double* sumsq_out, double* Ut, double* Vt);

}  // namespace blws
