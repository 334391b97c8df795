// Matrix completion hosts (Section 5, Table 2) with every SVT by BLWS.
//
// SVT of [Cai08] (variant 0), the paper's host:
//   k0 = ceil(tau / (delta ||P_Omega M||_2));  Y^0 = k0 delta P_Omega(M)
//   X^k = T_tau(Y^{k-1});  stop when ||P_Omega(X^k - M)|| / ||P_Omega M|| <= tol
//   Y^k = Y^{k-1} + delta P_Omega(M - X^k)
// with [Cai08]'s rank prediction: s_k = r_{k-1} + 1, raised by l while the
// s_k-th value still exceeds tau.  Y lives on Omega (values in CSR order), so
// the SVT operator is the CSR matrix alone.
//
// Proximal / FPC form (variant 1): W_k = X_k + delta P_Omega(M - X_k), an
// operator made of the low-rank X_k = U diag(theta) V^T plus the sparse
// residual; X_{k+1} = T_tau(W_k) with tau lowered by eta (down to tau_min)
// whenever ||X_{k+1} - X_k||_F / max(1, ||X_k||_F) < xtol.
//
// The sampled product and the update of Y (or of the sparse residual) are one
// fused SDDMM pass over Omega.
#include <math.h>

#include <algorithm>
#include <vector>

#include "graph.cuh"
#include "mc_kernels.cuh"
#include "solver.cuh"

namespace blws {

namespace {

__global__ void scale_copy(int nnz, double a, const double* __restrict__ x, double* y) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x)
    y[e] = a * x[e];
}

__global__ void thresholds_mc(int r, const double* __restrict__ sigma, double tau,
                              const double* __restrict__ tau_dev, double* th) {
  if (tau_dev) tau = *tau_dev;
  for (int t = threadIdx.x; t < r; t += blockDim.x) th[t] = fmax(sigma[t] - tau, 0.0);
}

// the threshold a replayed graph reads (tau changes in the proximal form)
__global__ void set_tau(double* slot, double tau) { *slot = tau; }

__global__ void check_finite(int nnz, const double* __restrict__ v, int* flag) {
  int bad = 0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x)
    if (!isfinite(v[e])) bad = 1;
  if (bad) atomicOr(flag, 1);
}

}  // namespace

blws_status mc_run(Ctx* ctx, cudaStream_t s, int m, int n, int nnz, const int* rowptr,
                   const int* colidx, const double* vals, const mc_params& p, int max_rank,
                   double* Uout, double* thout, double* Vout, mc_info* info) {
  const int N = m + n, pmin = std::min(m, n);
  const bool prox = p.variant == 1;
  double* scal;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  double* red;
  BLWS_TRY(ctx->get(BUF_RED, (size_t)std::max(ceil_div((long long)m * 32, 256), ctx->sms * 8) + 4096, &red));
  (void)red;
  info->iters = 0;
  info->rank = 0;
  info->residual = 0.0;
  info->norm_two = 0.0;
  info->status = BLWS_OK;
  info->restarts = 0;
  BLWS_TRY_CUDA(ctx, cudaMemset2DAsync(Uout, sizeof(double) * m, 0, sizeof(double) * m, max_rank, s));
  BLWS_TRY_CUDA(ctx, cudaMemset2DAsync(Vout, sizeof(double) * n, 0, sizeof(double) * n, max_rank, s));
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(thout, 0, sizeof(double) * max_rank, s));
  if (nnz == 0) {  // nothing observed: X = 0 (vals may be a null pointer here)
    BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    return BLWS_OK;
  }
  int* flag = reinterpret_cast<int*>(scal + SLOT_FLAG);
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), s));
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(scal + SLOT_TCERR, 0, sizeof(double), s));
  check_finite<<<std::min(ceil_div(nnz, 256), ctx->sms * 8), 256, 0, s>>>(nnz, vals, flag);
  BLWS_CHECK_LAUNCH(ctx);
  BLWS_TRY(sumsq(ctx, s, nnz, 1, vals, nnz, scal + SLOT_NORM));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * SLOT_MAX,
                                     cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  if (*reinterpret_cast<int*>(ctx->host_pinned + SLOT_FLAG))
    return ctx->fail(BLWS_ENONFINITE, "mc_solve: observed values have NaN/Inf");
  const double norm_pm = sqrt(ctx->host_pinned[SLOT_NORM]);
  if (norm_pm == 0.0) {
    BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    return BLWS_OK;
  }

  int *colptr, *rowidx, *perm;
  BLWS_TRY(build_csc(ctx, s, m, n, nnz, rowptr, colidx, &colptr, &rowidx, &perm));
  Operator Mop;
  Mop.m = m;
  Mop.n = n;
  Mop.nnz = nnz;
  Mop.rowptr = rowptr;
  Mop.colidx = colidx;
  Mop.val = vals;
  Mop.colptr = colptr;
  Mop.rowidx = rowidx;
  Mop.perm = perm;
  double norm2 = 0.0;
  BLWS_TRY(spectral_norm(ctx, s, Mop, &norm2));
  info->norm_two = norm2;

  const double delta = p.delta > 0 ? p.delta : (prox ? 1.0 : 1.2 * (double)m * n / nnz);
  const int k = ctx->cfg.k, k_cold = ctx->cfg.k_cold;
  const int bcap = std::max(1, std::min(pmin, N / std::max(k, k_cold)));
  const int incr = std::max(p.incr, 1);

  // iterate storage: sparse values y (CSR order), factors of the current X
  // (U, V, sigma, theta) and of the previous X (PROX), row-major scratch
  double *y, *Uw, *Vw, *sig, *Xf;
  BLWS_TRY(ctx->get(BUF_MC_Y, (size_t)nnz, &y));
  BLWS_TRY(ctx->get(BUF_WARM_U, (size_t)m * bcap, &Uw));
  BLWS_TRY(ctx->get(BUF_WARM_V, (size_t)n * bcap, &Vw));
  BLWS_TRY(ctx->get(BUF_SIG, (size_t)4 * bcap, &sig));
  double* th = sig + bcap;
  double* th_prev = th + bcap;
  // previous factors (PROX low-rank term) + row-major scratch for the SDDMM
  BLWS_TRY(ctx->get(BUF_Y, (size_t)(m + n) * bcap * 2, &Xf));
  double* Up = Xf;
  double* Vp = Up + (size_t)m * bcap;
  double* Ut = Vp + (size_t)n * bcap;
  double* Vt = Ut + (size_t)m * bcap;
  int* count_dev = reinterpret_cast<int*>(scal + SLOT_COUNT);

  double tau;
  if (!prox) {
    tau = p.tau > 0 ? p.tau : 5.0 * sqrt((double)m * n);
    const double k0 = ceil(tau / (delta * norm2));
    scale_copy<<<std::min(ceil_div(nnz, 256), ctx->sms * 8), 256, 0, s>>>(nnz, k0 * delta, vals, y);
  } else {
    tau = p.eta * norm2;
    scale_copy<<<std::min(ceil_div(nnz, 256), ctx->sms * 8), 256, 0, s>>>(nnz, delta, vals, y);
  }
  BLWS_CHECK_LAUNCH(ctx);
  const double tau_min = p.tau_min_rel * norm2;

  Operator Wop = Mop;
  Wop.val = y;
  int w = 0, r_prev = 0, c = 0, rp = 0;
  double res = 1.0, xnorm_prev = 0.0;
  bool converged = false;
  int it = 0;
  for (it = 1; it <= p.max_iter; ++it) {
    if (prox && rp > 0) {  // low-rank part of W_k = X_k
      Wop.rl = rp;
      Wop.Ul = Up;
      Wop.sl = th_prev;
      Wop.Vl = Vp;
    }
    int sk = std::min(std::max(r_prev + 1, 1), bcap);
    for (;;) {
      BlwsArgs a;
      a.eps = tau;
      a.r = sk;
      a.mixed = ctx->cfg.precision == BLWS_PREC_MIXED;
      a.draw = (uint32_t)(it * 64 + (sk - r_prev));
      a.standard = ctx->cfg.start == 1;
      if (w == 0 || !ctx->cfg.warm) {
        a.cold = true;
        a.k = std::max(1, std::min(k_cold, N / sk));
      } else {
        a.U0 = Uw;
        a.ldu0 = m;
        a.V0 = Vw;
        a.ldv0 = n;
        a.w = w;
        a.ritz_warm = true;
        a.k = std::max(1, std::min(k, N / std::max(sk, w)));
      }
      // the warm block is read before U, V are overwritten, so in place is safe.
      // Two graph phases around the eigen-solver's host stage (graph.cuh): the
      // block steps, then the Ritz lift and count with the count copied back
      const int bw = std::max(a.r, a.w);
      set_tau<<<1, 1, 0, s>>>(scal + SLOT_EPS, tau);
      BLWS_CHECK_LAUNCH(ctx);
      a.guard = ctx->cfg.guard > 0.0;
      a.eps_dev = scal + SLOT_EPS;
      // with the Ritz-residual guard, an inaccurate call runs again from the
      // same start with one more block (at most twice)
      for (int extra = 0;; ++extra) {
        GraphKey ka;
        ka.u(0x4D43u).u(1).u(m).u(n).u(nnz).p(rowptr).p(colidx).p(Wop.val).p(colptr).p(rowidx).p(perm);
        ka.u(Wop.rl).p(Wop.Ul).p(Wop.sl).p(Wop.Vl).u(a.r).u(a.k).u(a.w).u(a.cold).u(a.standard).u(a.mixed);
        ka.p(Uw).p(Vw).u(ctx->cfg.seed).u(a.guard).u(a.reorth).u(a.cold || bw > a.w ? a.draw : 0u);
        BLWS_TRY(graph_phase(ctx, s, ka, [&](cudaStream_t q) { return blws_run_a(ctx, q, Wop, a); }));
        BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        BLWS_TRY(graph_harvest(ctx));
        if (!a.guard || extra == 2 || (a.k + 1) * bw > N || !(blws_guard_ratio(ctx, a) > ctx->cfg.guard)) break;
        ++a.k;
        a.reorth = true;
        ++info->restarts;
      }
      BLWS_TRY(blws_run_mid(ctx, s, Wop, a));
      GraphKey kb;
      kb.u(0x4D43u).u(2).u(m).u(n).u(a.r).u(a.k).u(a.w).u(a.mixed).p(Uw).p(Vw).p(sig);
      BLWS_TRY(graph_phase(ctx, s, kb, [&](cudaStream_t q) -> blws_status {
        BLWS_TRY(blws_run_b(ctx, q, Wop, a, Uw, m, Vw, n, sig, count_dev, scal + SLOT_EPS));
        BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * SLOT_MAX,
                                           cudaMemcpyDeviceToHost, q));
        return BLWS_OK;
      }));
      BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
      c = *reinterpret_cast<int*>(ctx->host_pinned + SLOT_COUNT);
      if (*reinterpret_cast<int*>(ctx->host_pinned + SLOT_TCERR))
        return ctx->fail(BLWS_ETIMEOUT, "mc_solve: a tensor-core wait ran out");
      w = sk;
      // [Cai08]: if the last computed value is still above tau, widen by l
      if (c < sk || sk >= bcap) break;
      sk = std::min(sk + incr, bcap);
    }
    if (c > max_rank)
      return ctx->fail(BLWS_EINVAL, "mc_solve: rank %d exceeds max_rank %d", c, max_rank);
    // thresholds and the SDDMM on Omega (residual and update of the sparse
    // values): a third graph phase
    GraphKey kc;
    kc.u(0x4D43u).u(3).u(m).u(n).u(nnz).u(c).u(w).p(rowptr).p(colidx).p(vals).p(Uw).p(Vw).p(sig);
    kc.p(y).p(Ut).p(Vt).d(delta).u(prox);
    BLWS_TRY(graph_phase(ctx, s, kc, [&](cudaStream_t q) -> blws_status {
      thresholds_mc<<<1, 256, 0, q>>>(w, sig, tau, scal + SLOT_EPS, th);
      BLWS_CHECK_LAUNCH(ctx);
      return sddmm(ctx, q, m, n, c, rowptr, colidx, vals, Uw, m, th, Vw, n, delta, prox ? 1 : 0, y,
                   scal + SLOT_NORM, Ut, Vt);
    }));
    double dx = 0.0, xnorm = 0.0;
    if (prox) {
      // ||X_{k+1} - X_k||_F^2 = sum th^2 + sum th_prev^2 - 2 tr(th U^T Up th_prev Vp^T V)
      double* G1 = Ut;  // c x rp, reuse scratch after the SDDMM
      double* G2 = G1 + (size_t)std::max(c, 1) * std::max(rp, 1);
      std::vector<double> h_th(c), h_thp(rp), h_g1((size_t)c * rp), h_g2((size_t)c * rp);
      if (c > 0 && rp > 0) {
        BLWS_TRY(gemm(ctx, s, true, false, c, rp, m, 1.0, Uw, m, Up, m, 0.0, G1, c));
        BLWS_TRY(gemm(ctx, s, true, false, c, rp, n, 1.0, Vw, n, Vp, n, 0.0, G2, c));
        BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(h_g1.data(), G1, sizeof(double) * c * rp, cudaMemcpyDeviceToHost, s));
        BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(h_g2.data(), G2, sizeof(double) * c * rp, cudaMemcpyDeviceToHost, s));
      }
      if (c > 0) BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(h_th.data(), th, sizeof(double) * c, cudaMemcpyDeviceToHost, s));
      if (rp > 0) BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(h_thp.data(), th_prev, sizeof(double) * rp, cudaMemcpyDeviceToHost, s));
      BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
      double a2 = 0.0, b2 = 0.0, cross = 0.0;
      for (int i = 0; i < c; ++i) a2 += h_th[i] * h_th[i];
      for (int j = 0; j < rp; ++j) b2 += h_thp[j] * h_thp[j];
      for (int i = 0; i < c; ++i)
        for (int j = 0; j < rp; ++j) cross += h_th[i] * h_g1[i + (size_t)j * c] * h_thp[j] * h_g2[i + (size_t)j * c];
      dx = sqrt(std::max(a2 + b2 - 2.0 * cross, 0.0));
      xnorm = sqrt(a2);
    }
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * SLOT_MAX,
                                       cudaMemcpyDeviceToHost, s));
    BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    const double r2 = ctx->host_pinned[SLOT_NORM];
    if (!isfinite(r2)) return ctx->fail(BLWS_ENONFINITE, "mc_solve: iterate became non-finite");
    if (*reinterpret_cast<int*>(ctx->host_pinned + SLOT_TCERR))
      return ctx->fail(BLWS_ETIMEOUT, "mc_solve: a tensor-core wait ran out");
    res = sqrt(r2) / norm_pm;
    r_prev = c;
    if (res <= p.tol) {
      converged = true;
      break;
    }
    if (prox) {
      // keep X_{k+1} as the low-rank term of the next operator
      if (c > 0) {
        BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(Up, Uw, sizeof(double) * m * c, cudaMemcpyDeviceToDevice, s));
        BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(Vp, Vw, sizeof(double) * n * c, cudaMemcpyDeviceToDevice, s));
        BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(th_prev, th, sizeof(double) * c, cudaMemcpyDeviceToDevice, s));
      }
      rp = c;
      if (dx / std::max(1.0, xnorm_prev) < p.xtol && tau > tau_min) tau = std::max(p.eta * tau, tau_min);
      xnorm_prev = xnorm;
    }
  }
  if (!converged) it = p.max_iter;
  if (c > 0) {
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(Uout, Uw, sizeof(double) * m * c, cudaMemcpyDeviceToDevice, s));
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(Vout, Vw, sizeof(double) * n * c, cudaMemcpyDeviceToDevice, s));
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(thout, th, sizeof(double) * c, cudaMemcpyDeviceToDevice, s));
  }
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  info->iters = it;
  info->rank = c;
  info->residual = res;
  info->status = converged ? BLWS_OK : BLWS_ENOCONV;
  return converged ? BLWS_OK : BLWS_ENOCONV;
}

}  // namespace blws
