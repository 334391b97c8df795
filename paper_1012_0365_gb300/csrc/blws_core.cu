// Block Lanczos with warm start on the augmented matrix W~ = [[0, W], [W^T, 0]].
//
//   * start block (Section 4.1, mixed start): X~_1 = [U_{i-1}; V_{i-1}] / sqrt 2,
//     padded with extra columns when the predicted rank exceeds the warm
//     width (Section 4.2), orthonormalised by CholeskyQR2;
//   * Algorithm 2 with W~ applied by skipping its zero blocks (Section 4, end):
//     P_l = [W X_{l,v}; W^T X_{l,u}],  M_l = sym(X_l^T P_l),
//     R_l = P_l - X_l M_l - X_{l-1} B_{l-1}^T,  (X_{l+1}, B_l) = qr(R_l);
//     R_l is projected once more against X_l, X_{l-1} before its QR (with a
//     warm start R_l is small and its computed direction carries rounding
//     error along X_l), or against every block on a cold start;
//   * T_k assembled as in Eq. (11), its EVD in decreasing order (Algorithm 3);
//   * Ritz lift U = sqrt2 Q_u Z(:, 1:r), V = sqrt2 Q_v Z(:, 1:r) (Theorem 1).
// For a symmetric W (Operator::sym) the same procedure runs on W itself: the
// start block is [U_{i-1} | extra columns], P_l = W X_l, and the Ritz vectors
// are Q Z(:, 1:r) -- BL_EVD(W_i, U_{i-1}, k) of Section 4 (Algorithm 3).
#include <math.h>

#include <algorithm>

#include "blws_core.cuh"

namespace blws {

namespace {

constexpr double kDeflTol = 1e-12;
constexpr double kDeflTolMixed = 1e-6;  // FP32 products resolve columns down to ~1e-6

// standard != 0: the warm columns are [U0; 0] (the one-sided start Section
// 4.1 compares the mixed start with) instead of [U0; V0] / sqrt(2)
__global__ void build_start(int m, int n, int w, const double* __restrict__ U0, int ldu0,
                            const double* __restrict__ V0, int ldv0, const double* __restrict__ G,
                            int ldg, int g, int b, uint64_t seed, uint32_t stream_id, int standard,
                            double* X, int ldx) {
  const int N = m + n;
  const double r2 = 0.70710678118654752440;
  const size_t total = (size_t)N * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), j = (int)(e / N);
    double v;
    if (j < w) {
      v = i < m ? U0[i + (size_t)j * ldu0] * r2 : (standard ? 0.0 : V0[(i - m) + (size_t)j * ldv0] * r2);
    } else if (j - w < g) {
      v = G[i + (size_t)(j - w) * ldg];
    } else {
      v = philox_normal(seed, (uint32_t)i, (uint32_t)j, stream_id);
    }
    X[i + (size_t)j * ldx] = v;
  }
}

// T(l*b + i, l*b + j) = (M_ij + M_ji) / 2
__global__ void put_sym_block(int b, const double* __restrict__ M, double* T, int ldt, int off) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < b * b; e += gridDim.x * blockDim.x) {
    const int i = e % b, j = e / b;
    T[(off + i) + (size_t)(off + j) * ldt] = 0.5 * (M[i + (size_t)j * b] + M[j + (size_t)i * b]);
  }
}

// T((l+1) b + i, l b + j) = B_ij and its transpose (Eq. 11)
__global__ void put_offdiag_block(int b, const double* __restrict__ B, double* T, int ldt, int row0,
                                  int col0) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < b * b; e += gridDim.x * blockDim.x) {
    const int i = e % b, j = e / b;
    const double v = B[i + (size_t)j * b];
    T[(row0 + i) + (size_t)(col0 + j) * ldt] = v;
    T[(col0 + j) + (size_t)(row0 + i) * ldt] = v;
  }
}

// sigma[0:r] = lam[0:r]; count = #{sigma_t > eps}; eps from device memory
// when eps_dev is set (a replayed graph's per-iteration threshold)
__global__ void ritz_values(int r, const double* __restrict__ lam, double eps,
                            const double* __restrict__ eps_dev, double* sigma, int* count) {
  __shared__ int cnt;
  if (eps_dev) eps = *eps_dev;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int t = threadIdx.x; t < r; t += blockDim.x) {
    sigma[t] = lam[t];
    c += lam[t] > eps ? 1 : 0;
  }
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) *count = cnt;
}

// The guard's measure.  Y = G Z_last (G = R_k^T R_k, b x b; Z_last the last
// block's rows of the first r eigenvectors of T_k): rho_j^2 = Z_last(:, j) .
// Y(:, j) is ||R_k Z_last(:, j)||^2, the squared residual ||W~ y_j -
// theta_j y_j|| of Ritz pair j (block Lanczos relation W~ Q_k = Q_k T_k +
// R_k E_k^T).  *out = max over the pairs with theta_j > eps of rho_j /
// |theta_1| (0 when there is none).  One CTA, a warp per pair.
__global__ void ritz_residual(int b, int r, const double* __restrict__ Zl, int ldz,
                              const double* __restrict__ Y, int ldy, const double* __restrict__ lam,
                              double eps, const double* __restrict__ eps_dev, double* out) {
  __shared__ double red[32];
  if (eps_dev) eps = *eps_dev;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const double top = fabs(lam[0]);
  double worst = 0.0;
  for (int j = warp; j < r; j += nw) {
    double acc = 0.0;
    for (int i = lane; i < b; i += 32) acc = fma(Zl[i + (size_t)j * ldz], Y[i + (size_t)j * ldy], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lam[j] > eps && top > 0.0) worst = fmax(worst, sqrt(fmax(acc, 0.0)) / top);
  }
  if (lane == 0) red[warp] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    double w = 0.0;
    for (int q = 0; q < nw; ++q) w = fmax(w, red[q]);
    *out = w;
  }
}

}  // namespace

blws_status apply_op(Ctx* ctx, cudaStream_t s, const Operator& op, const double* X, int ldx, int b,
                     double* P, int ldp) {
  const int m = op.m, n = op.n;
  if (op.sym) return gemm(ctx, s, false, false, m, b, m, 1.0, op.W, op.ldw, X, ldx, 0.0, P, ldp);
  if (op.W && op.Or && op.Oc) return oz_dual_apply(ctx, s, *op.Or, *op.Oc, m, n, X, ldx, b, P, ldp);
  if (op.W && op.Wr && op.Wc && tc_npad(b) > 0)
    return tc_dual_apply(ctx, s, *op.Wr, *op.Wc, m, n, X, ldx, b, P, ldp);
  if (op.W) {
    BLWS_TRY(ctx->time_begin(s));
    BLWS_TRY(gemm(ctx, s, false, false, m, b, n, 1.0, op.W, op.ldw, X + m, ldx, 0.0, P, ldp));
    BLWS_TRY(gemm(ctx, s, true, false, n, b, m, 1.0, op.W, op.ldw, X, ldx, 0.0, P + m, ldp));
    return ctx->time_end(s, 2.0 * m * n * b, 0);
  }
  return apply_sparse(ctx, s, op, X, ldx, b, P, ldp);
}

blws_status blws_reserve(Ctx* ctx, int m, int n, int bmax, int kmax) {
  const size_t N = (size_t)m + n;
  const size_t kb = (size_t)kmax * bmax;
  void* p;
  BLWS_TRY(ctx->get(BUF_Q, N * kb * sizeof(double), &p));
  BLWS_TRY(ctx->get(BUF_P, N * bmax * sizeof(double), &p));
  BLWS_TRY(ctx->get(BUF_P2, N * bmax * sizeof(double), &p));
  BLWS_TRY(ctx->get(BUF_T, (3 * kb * kb + 2 * kb + (size_t)bmax * bmax * 2 + 64) * sizeof(double), &p));
  BLWS_TRY(ctx->get(BUF_SMALL, 6 * (size_t)bmax * bmax * sizeof(double), &p));
  // split-K partials: at most 2 * target * BM * BN doubles, target = 8 SMs-worth
  // of CTAs (see gemm_f64.cu)
  BLWS_TRY(ctx->get(BUF_SPLITK, (size_t)16 * ctx->sms * 64 * 64 * sizeof(double), &p));
  // eigen-solver padding: even (one CTA) or a multiple of 32 (block-pair Jacobi)
  const size_t Ne = std::max(kb + (kb & 1), (kb + 31) / 32 * 32);
  BLWS_TRY(ctx->get(BUF_EIG, 3 * Ne * Ne * sizeof(float) + 6 * kb * kb * sizeof(double) +
                                 (4 * kb + 3 * 1024 + 64) * sizeof(double), &p));
  BLWS_TRY(ctx->get(BUF_RED, (size_t)ctx->sms * 8 * sizeof(double), &p));
  return BLWS_OK;
}

blws_status blws_run_a(Ctx* ctx, cudaStream_t s, const Operator& op, const BlwsArgs& a) {
  const int m = op.m, n = op.sym ? 0 : op.n, N = m + n;
  const int w = a.w, g = a.G ? a.g : 0;
  const int b = std::max(a.r, w + g);
  const int k = a.k;
  const int kb = k * b;
  if (a.r < 1 || b < 1 || kb > N || a.r > b)
    return ctx->fail(BLWS_EINVAL, "blws: need 1 <= r <= b and k*b <= m+n (r=%d b=%d k=%d m+n=%d)",
                     a.r, b, k, N);
  BLWS_TRY(blws_reserve(ctx, m, n, b, k));
  double *Q, *P, *P2, *T, *scal;
  BLWS_TRY(ctx->get(BUF_Q, (size_t)N * kb, &Q));
  BLWS_TRY(ctx->get(BUF_P, (size_t)N * b, &P));
  BLWS_TRY(ctx->get(BUF_P2, (size_t)N * b, &P2));
  BLWS_TRY(ctx->get(BUF_T, (size_t)3 * kb * kb + 2 * kb + (size_t)b * b * 2 + 64, &T));
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  double* Z = T + (size_t)kb * kb;
  double* lam = Z + (size_t)kb * kb;
  double* Mtmp = lam + 2 * kb;  // b x b
  double* Bblk = Mtmp + (size_t)b * b;
  // second-projection coefficients, (k b) x b <= kb * kb: the Z area is free until the EVD
  double* C = Z;

  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(T, 0, sizeof(double) * kb * kb, s));
  const int eb = std::min(ceil_div((long long)N * b, 256), ctx->sms * 8);
  build_start<<<eb, 256, 0, s>>>(m, n, w, a.U0, a.ldu0, a.V0, a.ldv0, a.G, a.ldg, g, b,
                                 ctx->cfg.seed, a.draw, a.standard ? 1 : 0, P, N);
  BLWS_CHECK_LAUNCH(ctx);
  // orthonormalise the start block: deflation scale = its largest column norm
  BLWS_TRY(col_norms(ctx, s, N, b, P, N, lam, scal + SLOT_AUX));
  const bool f32 = a.mixed;
  const double defl = f32 ? kDeflTolMixed : kDeflTol;
  // a warm start of the previous call's Ritz vectors alone (mixed start, no
  // drawn or given columns) is orthonormal to the working precision's
  // rounding: one CholeskyQR pass
  const bool one_pass = a.ritz_warm && !a.cold && !a.standard && g == 0 && w == b;
  BLWS_TRY(chol_qr2(ctx, s, N, b, P, N, Q, P2, Bblk, scal + SLOT_AUX, defl, f32, one_pass));

  for (int l = 0; l < k; ++l) {
    double* Xl = Q + (size_t)l * b * N;
    BLWS_TRY(apply_op(ctx, s, op, Xl, N, b, P, N));
    if (l == 0) BLWS_TRY(col_norms(ctx, s, N, b, P, N, lam, scal + SLOT_SCALE));
    BLWS_TRY(gemm(ctx, s, true, false, b, b, N, 1.0, Xl, N, P, N, 0.0, Mtmp, b, f32));
    put_sym_block<<<ceil_div((long long)b * b, 256), 256, 0, s>>>(b, Mtmp, T, kb, l * b);
    BLWS_CHECK_LAUNCH(ctx);
    if (l == k - 1) break;
    // R_l = P_l - X_l M_l - X_{l-1} B_{l-1}^T as one product: [X_{l-1} X_l] are
    // adjacent blocks of Q and [B_{l-1}^T; M_l] adjacent blocks of T's column l
    const int c0r = l > 0 ? l - 1 : l;
    BLWS_TRY(gemm(ctx, s, false, false, N, b, (l + 1 - c0r) * b, -1.0, Q + (size_t)c0r * b * N, N,
                  T + (size_t)c0r * b + (size_t)l * b * kb, kb, 1.0, P, N, f32));
    // second projection against the recurrence's blocks (all blocks when cold)
    const int c0 = a.cold || a.reorth ? 0 : std::max(l - 1, 0);
    const int cols = (l + 1 - c0) * b;
    const double* base = Q + (size_t)c0 * b * N;
    BLWS_TRY(gemm(ctx, s, true, false, cols, b, N, 1.0, base, N, P, N, 0.0, C, cols, f32));
    BLWS_TRY(gemm(ctx, s, false, false, N, b, cols, -1.0, base, N, C, cols, 1.0, P, N, f32));
    BLWS_TRY(chol_qr2(ctx, s, N, b, P, N, Xl + (size_t)b * N, P2, Bblk, scal + SLOT_SCALE, defl, f32));
    put_offdiag_block<<<ceil_div((long long)b * b, 256), 256, 0, s>>>(b, Bblk, T, kb, (l + 1) * b,
                                                                       l * b);
    BLWS_CHECK_LAUNCH(ctx);
  }
  if (a.guard) {
    // the residual of the last block (the recurrence's product with no QR
    // after it) and its Gram matrix
    const int l = k - 1, c0r = l > 0 ? l - 1 : l;
    BLWS_TRY(gemm(ctx, s, false, false, N, b, (l + 1 - c0r) * b, -1.0, Q + (size_t)c0r * b * N, N,
                  T + (size_t)c0r * b + (size_t)l * b * kb, kb, 1.0, P, N, f32));
    double* Gk = nullptr;
    BLWS_TRY(ctx->get(BUF_GUARD, (size_t)b * b + (size_t)b * a.r, &Gk));
    BLWS_TRY(gemm_sym(ctx, s, true, false, b, N, 1.0, P, N, P, N, Gk, b, f32));
  }
  BLWS_TRY(sym_eig_start(ctx, s, kb, T, lam, Z));
  if (a.guard) {
    double* Gk = nullptr;
    BLWS_TRY(ctx->get(BUF_GUARD, (size_t)b * b + (size_t)b * a.r, &Gk));
    double* Yg = Gk + (size_t)b * b;
    const double* Zl = Z + (size_t)(k - 1) * b;  // rows (k-1) b .. k b - 1
    BLWS_TRY(gemm(ctx, s, false, false, b, a.r, b, 1.0, Gk, b, Zl, kb, 0.0, Yg, b));
    ritz_residual<<<1, 256, 0, s>>>(b, a.r, Zl, kb, Yg, b, lam, a.eps, a.eps_dev, scal + SLOT_GUARD);
    BLWS_CHECK_LAUNCH(ctx);
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(sym_eig_host_extra(ctx, kb), scal + SLOT_GUARD, sizeof(double),
                                       cudaMemcpyDeviceToHost, s));
  }
  return BLWS_OK;
}

double blws_guard_ratio(Ctx* ctx, const BlwsArgs& a) {
  const int b = std::max(a.r, a.w + (a.G ? a.g : 0));
  return *sym_eig_host_extra(ctx, a.k * b);
}

namespace {
struct RunDims {
  int b, kb;
  double *Q, *T, *Z, *lam;
};
blws_status run_dims(Ctx* ctx, const Operator& op, const BlwsArgs& a, RunDims* d) {
  const int N = op.m + (op.sym ? 0 : op.n);
  d->b = std::max(a.r, a.w + (a.G ? a.g : 0));
  d->kb = a.k * d->b;
  BLWS_TRY(ctx->get(BUF_Q, (size_t)N * d->kb, &d->Q));
  BLWS_TRY(ctx->get(BUF_T, (size_t)3 * d->kb * d->kb + 2 * d->kb + (size_t)d->b * d->b * 2 + 64, &d->T));
  d->Z = d->T + (size_t)d->kb * d->kb;
  d->lam = d->Z + (size_t)d->kb * d->kb;
  return BLWS_OK;
}
}  // namespace

blws_status blws_run_mid(Ctx* ctx, cudaStream_t s, const Operator& op, const BlwsArgs& a) {
  RunDims d;
  BLWS_TRY(run_dims(ctx, op, a, &d));
  return sym_eig_finish(ctx, s, d.kb, d.T, d.lam, d.Z, a.eps);
}

blws_status blws_run_b(Ctx* ctx, cudaStream_t s, const Operator& op, const BlwsArgs& a, double* U,
                       int ldu, double* V, int ldv, double* sigma, int* count_dev,
                       const double* eps_dev) {
  const int m = op.m, n = op.sym ? 0 : op.n, N = m + n;
  RunDims d;
  BLWS_TRY(run_dims(ctx, op, a, &d));
  const int kb = d.kb;
  double* Q = d.Q;
  double* Z = d.Z;
  double* lam = d.lam;
  const bool f32 = a.mixed;
  if (op.sym) {
    BLWS_TRY(gemm(ctx, s, false, false, m, a.r, kb, 1.0, Q, N, Z, kb, 0.0, U, ldu, f32));
  } else {
    const double r2 = 1.41421356237309504880;
    BLWS_TRY(gemm(ctx, s, false, false, m, a.r, kb, r2, Q, N, Z, kb, 0.0, U, ldu, f32));
    BLWS_TRY(gemm(ctx, s, false, false, n, a.r, kb, r2, Q + m, N, Z, kb, 0.0, V, ldv, f32));
  }
  ritz_values<<<1, 256, 0, s>>>(a.r, lam, a.eps, eps_dev, sigma, count_dev);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

blws_status blws_run(Ctx* ctx, cudaStream_t s, const Operator& op, const BlwsArgs& a,
                     double* U, int ldu, double* V, int ldv, double* sigma, int* count_dev) {
  BLWS_TRY(blws_run_a(ctx, s, op, a));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  BLWS_TRY(blws_run_mid(ctx, s, op, a));
  return blws_run_b(ctx, s, op, a, U, ldu, V, ldv, sigma, count_dev, nullptr);
}

}  // namespace blws
