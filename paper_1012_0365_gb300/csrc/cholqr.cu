// Block orthogonalisation (the "qr" of Algorithm 2) by CholeskyQR2 with
// column equilibration and deflation.
//
//   pass 1: G = R^T R;  d_j = sqrt(G_jj);  G^ = D^-1 G D^-1 = L L^T (FP64
//           Cholesky);  X1 = R D^-1 L^-T;  B1 = L^T D   (so R = X1 B1)
//   pass 2: the same on X1 (G ~ I), X = X1 S2, B = B2 B1.
// A column dies when its R-factor diagonal d_j sqrt(pivot_j) is below
// tol * scale, or when its equilibrated pivot is below kPivMin (it is then
// numerically dependent on earlier columns); a dead column of X is exactly
// zero and its row of B is zero.  This is the deflation that makes the
// procedure exact when a warm start spans an invariant subspace (R_l = 0).
//
// The Gram matrices and the products with the tall block are FP64 GEMMs over
// the whole GPU; the b x b factorisation runs in one CTA.
#include "ops.cuh"

namespace blws {

namespace {

constexpr double kPivMin = 1e-10;

// One CTA: equilibrated Cholesky of G (b x b, ld b) with deflation, then
// S = D^-1 L^-T (upper, X = R S) and B = L^T D (upper, R = X B).
// work: 2 b^2 doubles (shared or global).
__global__ void __launch_bounds__(1024)
chol_equil_kernel(int b, const double* __restrict__ G, const double* __restrict__ scale_ptr,
                  double tol, double* __restrict__ S, double* __restrict__ Bout,
                  double* gwork, int use_smem) {
  extern __shared__ double smem[];
  double* L = use_smem ? smem : gwork;          // b x b, ld b (lower used)
  double* Li = L + (size_t)b * b;               // inverse of L
  __shared__ double d[1024 + 1];                // column scales (b <= 1024)
  __shared__ double dinv[1024 + 1];             // 1 / d, then 1 / L_jj
  __shared__ int dead[1024 + 1];
  __shared__ double piv_sh;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double scale = *scale_ptr;
  const double thr = tol * scale;

  for (int j = tid; j < b; j += nt) {
    const double g = G[j + (size_t)j * b];
    const double dj = g > 0.0 ? sqrt(g) : 0.0;
    const bool dz = !(dj > thr);
    dead[j] = dz ? 1 : 0;
    d[j] = dz ? 1.0 : dj;
    dinv[j] = dz ? 1.0 : 1.0 / dj;
  }
  __syncthreads();
  // equilibrated lower triangle (upper ignored)
  for (int e = tid; e < b * b; e += nt) {
    const int i = e % b, j = e / b;
    double v = 0.0;
    if (i >= j) {
      if (dead[i] || dead[j]) v = (i == j) ? 1.0 : 0.0;
      else v = G[i + (size_t)j * b] * dinv[i] * dinv[j];
    }
    L[e] = v;
  }
  __syncthreads();
  // right-looking Cholesky
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      double p = L[j + (size_t)j * b];
      bool dj = dead[j] != 0;
      if (!dj) {
        const double rdiag = d[j] * sqrt(p > 0.0 ? p : 0.0);
        if (!(p > kPivMin) || !(rdiag > thr)) dj = true;
      }
      dead[j] = dj ? 1 : 0;
      piv_sh = dj ? 1.0 : sqrt(p);
    }
    __syncthreads();
    const double lj = piv_sh;
    const double rlj = 1.0 / lj;  // one FP64 division per column (divisions are slow here)
    const bool dj = dead[j] != 0;
    for (int i = j + 1 + tid; i < b; i += nt) {
      double* lij = &L[i + (size_t)j * b];
      *lij = dj ? 0.0 : *lij * rlj;
    }
    if (tid == 0) L[j + (size_t)j * b] = lj;
    __syncthreads();
    if (!dj) {
      const int rem = b - j - 1;
      for (int e = tid; e < rem * rem; e += nt) {
        const int i = j + 1 + e % rem, kk = j + 1 + e / rem;
        if (i >= kk) L[i + (size_t)kk * b] -= L[i + (size_t)j * b] * L[kk + (size_t)j * b];
      }
    }
    __syncthreads();
  }
  // Li = L^-1 (lower), one thread per column; reciprocals of the diagonal first
  for (int i = tid; i < b; i += nt) dinv[i] = 1.0 / L[i + (size_t)i * b];
  __syncthreads();
  for (int c = tid; c < b; c += nt) {
    for (int i = 0; i < c; ++i) Li[i + (size_t)c * b] = 0.0;
    Li[c + (size_t)c * b] = dinv[c];
    for (int i = c + 1; i < b; ++i) {
      double acc = 0.0;
      for (int k = c; k < i; ++k) acc = fma(L[i + (size_t)k * b], Li[k + (size_t)c * b], acc);
      Li[i + (size_t)c * b] = -acc * dinv[i];
    }
  }
  __syncthreads();
  // scales again (dinv was reused for the diagonal of L)
  for (int j = tid; j < b; j += nt) dinv[j] = 1.0 / d[j];
  __syncthreads();
  // S(k, j) = Li(j, k) / d_k  (upper);  B(k, j) = L(j, k) d_j (upper).
  // A dead column has no X column and no row of B, but keeps its
  // coefficients on the earlier live columns (its column of B above the
  // diagonal), as Gram-Schmidt with deflation does: R(:, j) = X B(:, j).
  for (int e = tid; e < b * b; e += nt) {
    const int k = e % b, j = e / b;
    double sv = 0.0, bv = 0.0;
    if (k <= j && !dead[k]) {
      if (!dead[j]) sv = Li[j + (size_t)k * b] * dinv[k];
      if (!dead[j] || k < j) bv = L[j + (size_t)k * b] * d[j];
    }
    S[e] = sv;
    Bout[e] = bv;
  }
}

blws_status chol_equil(Ctx* ctx, cudaStream_t s, int b, const double* G, const double* scale,
                       double tol, double* S, double* B, double* gwork) {
  if (b > 1024) return ctx->fail(BLWS_EINVAL, "block width %d exceeds 1024", b);
  const size_t need = 2ull * b * b * sizeof(double);
  const int use_smem = need <= 200 * 1024 ? 1 : 0;
  if (use_smem) {
    BLWS_TRY_CUDA(ctx, cudaFuncSetAttribute(chol_equil_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
  }
  chol_equil_kernel<<<1, 1024, use_smem ? need : 0, s>>>(b, G, scale, tol, S, B, gwork, use_smem);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

}  // namespace

blws_status chol_qr2(Ctx* ctx, cudaStream_t s, int N, int b, double* R, int ld, double* X,
                     double* tmp, double* B, const double* scale, double tol) {
  // small scratch: G, S, B1, B2, work (2 b^2)
  double* sm = nullptr;
  BLWS_TRY(ctx->get(BUF_SMALL, 6ull * b * b, &sm));
  double* G = sm;
  double* S = G + (size_t)b * b;
  double* B1 = S + (size_t)b * b;
  double* B2 = B1 + (size_t)b * b;
  double* work = B2 + (size_t)b * b;
  // pass 1
  BLWS_TRY(gemm(ctx, s, true, false, b, b, N, 1.0, R, ld, R, ld, 0.0, G, b));
  BLWS_TRY(chol_equil(ctx, s, b, G, scale, tol, S, B1, work));
  BLWS_TRY(gemm(ctx, s, false, false, N, b, b, 1.0, R, ld, S, b, 0.0, tmp, ld));
  // pass 2 (columns are now unit or zero: same deflation rule against 1)
  BLWS_TRY(gemm(ctx, s, true, false, b, b, N, 1.0, tmp, ld, tmp, ld, 0.0, G, b));
  double* one = nullptr;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &one));
  BLWS_TRY(chol_equil(ctx, s, b, G, one + SLOT_ONE, 0.5, S, B2, work));
  BLWS_TRY(gemm(ctx, s, false, false, N, b, b, 1.0, tmp, ld, S, b, 0.0, X, ld));
  // B = B2 B1
  BLWS_TRY(gemm(ctx, s, false, false, b, b, b, 1.0, B2, b, B1, b, 0.0, B, b));
  return BLWS_OK;
}

}  // namespace blws
