/* One-sided (Hestenes) Jacobi SVD in plain C, FP64.
 *
 * TEST INFRASTRUCTURE ONLY: an independent brute-force check of the oracle's
 * full-SVD singular value thresholding (paper Eq. (3)-(4)) on tiny matrices,
 * sharing nothing with LAPACK.  Never linked into the product library.
 *
 * Method (textbook one-sided Jacobi): orthogonalise the columns of a working
 * copy G of A (m x n, m >= n) by plane rotations applied on the right,
 * accumulating them in V, until every pair of columns is orthogonal to
 * relative precision tol.  Then sigma_j = ||g_j||, u_j = g_j / sigma_j, and
 * A = U diag(sigma) V^T.  Columns are sorted by decreasing sigma.
 *
 * Layout: column-major, A is m x n with leading dimension m; U is m x n,
 * V is n x n, s has n entries.  Requires m >= n (transpose the input
 * otherwise).  Returns the number of sweeps, or -1 on bad arguments, or -2
 * if it did not converge within max_sweeps.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

int jacobi_svd(int m, int n, const double* A, double* s, double* U, double* V,
               double tol, int max_sweeps) {
  if (m < n || n < 1 || !A || !s || !U || !V) return -1;
  double* G = (double*)malloc(sizeof(double) * (size_t)m * n);
  if (!G) return -1;
  memcpy(G, A, sizeof(double) * (size_t)m * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) V[i + (size_t)j * n] = (i == j) ? 1.0 : 0.0;

  int sweep = 0, converged = 0;
  while (!converged && sweep < max_sweeps) {
    converged = 1;
    ++sweep;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        double* gp = G + (size_t)p * m;
        double* gq = G + (size_t)q * m;
        for (int i = 0; i < m; ++i) {
          alpha += gp[i] * gp[i];
          beta += gq[i] * gq[i];
          gamma += gp[i] * gq[i];
        }
        if (fabs(gamma) <= tol * sqrt(alpha * beta) || gamma == 0.0) continue;
        converged = 0;
        /* rotation that zeroes the (p,q) entry of G^T G */
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double sn = c * t;
        for (int i = 0; i < m; ++i) {
          double x = gp[i], y = gq[i];
          gp[i] = c * x - sn * y;
          gq[i] = sn * x + c * y;
        }
        double* vp = V + (size_t)p * n;
        double* vq = V + (size_t)q * n;
        for (int i = 0; i < n; ++i) {
          double x = vp[i], y = vq[i];
          vp[i] = c * x - sn * y;
          vq[i] = sn * x + c * y;
        }
      }
    }
  }
  /* singular values and left vectors */
  for (int j = 0; j < n; ++j) {
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += G[i + (size_t)j * m] * G[i + (size_t)j * m];
    nrm = sqrt(nrm);
    s[j] = nrm;
    for (int i = 0; i < m; ++i) U[i + (size_t)j * m] = nrm > 0 ? G[i + (size_t)j * m] / nrm : 0.0;
  }
  /* selection sort by decreasing sigma, permuting U and V columns */
  for (int j = 0; j < n - 1; ++j) {
    int best = j;
    for (int l = j + 1; l < n; ++l)
      if (s[l] > s[best]) best = l;
    if (best != j) {
      double tmp = s[j]; s[j] = s[best]; s[best] = tmp;
      for (int i = 0; i < m; ++i) {
        double x = U[i + (size_t)j * m]; U[i + (size_t)j * m] = U[i + (size_t)best * m]; U[i + (size_t)best * m] = x;
      }
      for (int i = 0; i < n; ++i) {
        double x = V[i + (size_t)j * n]; V[i + (size_t)j * n] = V[i + (size_t)best * n]; V[i + (size_t)best * n] = x;
      }
    }
  }
  free(G);
  return converged ? sweep : -2;
}
