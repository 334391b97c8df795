// Robust PCA host (Section 5, Table 1): inexact ALM whose SVT (Eq. 3-4) is
// evaluated by BLWS each iteration.  The paper takes the host from its
// references; its step rules, written out:
//   Y_0 = D / J(D), J(D) = max(||D||_2, ||D||_inf / lambda);  mu_0 = 1.25/||D||_2
//   E  = Theta_{lambda/mu}(D - A + Y/mu);  A = T_{1/mu}(D - E + Y/mu)
//   Z  = D - A - E;  Y += mu Z;  mu = min(rho mu, 1e7 mu_0);  stop ||Z||/||D|| < tol
// and the rank prediction: sv = svp + 1 if svp < sv else svp + round(0.05 n).
//
// One fused pass over HBM per iteration (rpca_epilogue): with A kept
// factored as U diag(theta) V^T it rebuilds each a_ij in registers (rank-c
// tile product), forms Z, updates Y, shrinks the next E and writes the next
// SVT input W.  Reads D, E, Y; writes E', Y, W.  In the FP64-equivalent mode
// the rank-c product is an FP64 ALU bound of its own (2c flops per element),
// so there A = (U diag(theta)) V^T is formed first as a digit-plane
// tensor-core product and the pass reads it (EP_PRE); the mixed mode forms it
// the same way from split TF32 operands on the tensor cores.
#include <math.h>

#include <algorithm>

#include "blws_core.cuh"
#include "graph.cuh"
#include "solver.cuh"

namespace blws {

namespace {

constexpr int kEpBM = 64, kEpBN = 64, kEpBK = 16;

__device__ inline double shrink(double x, double t) {
  // Theta_t(x) = sgn(x) max(|x| - t, 0)  (Eq. 4)
  const double ax = fabs(x) - t;
  return ax > 0.0 ? copysign(ax, x) : 0.0;
}

enum EpMode { EP_ITER = 0, EP_FINAL = 1, EP_PRE = 2 };  // EP_PRE: as EP_ITER, A read from Aout

// Rank-c tile reconstruction a = U[i,:] diag(th) V[j,:]^T plus the host update.
// CT: arithmetic of the rank-c reconstruction (double, or float in the
// mixed-precision mode); the host update itself is FP64.
template <int MODE, typename CT>
__global__ void __launch_bounds__(256)
rpca_epilogue(int m, int n, int ld, const double* __restrict__ U, int ldu,
              const double* __restrict__ th, const double* __restrict__ V, int ldv,
              const int* __restrict__ count_ptr, const double* __restrict__ D,
              const double* __restrict__ Ein, double* __restrict__ Eout, double* __restrict__ Y,
              double* __restrict__ Wout, double* __restrict__ Aout, double mu, double mu_next,
              double lam, double* __restrict__ part, const double* __restrict__ dyn) {
  __shared__ CT Us[kEpBK][kEpBM + 1];
  if (dyn) {  // this iteration's mu and next mu from device memory (replayed graphs)
    mu = dyn[1];
    mu_next = dyn[2];
  }
  __shared__ CT Vs[kEpBK][kEpBN + 1];
  __shared__ double red[256];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.x * kEpBM, j0 = blockIdx.y * kEpBN;
  const int c = *count_ptr;
  CT a[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) a[p][q] = CT(0);
  for (int t0 = 0; MODE != EP_PRE && t0 < c; t0 += kEpBK) {
    for (int e = threadIdx.x; e < kEpBM * kEpBK; e += 256) {
      const int i = e % kEpBM, t = e / kEpBM;
      const int gi = i0 + i, gt = t0 + t;
      Us[t][i] = (CT)((gi < m && gt < c) ? U[gi + (size_t)gt * ldu] * th[gt] : 0.0);
    }
    for (int e = threadIdx.x; e < kEpBN * kEpBK; e += 256) {
      const int j = e % kEpBN, t = e / kEpBN;
      const int gj = j0 + j, gt = t0 + t;
      Vs[t][j] = (CT)((gj < n && gt < c) ? V[gj + (size_t)gt * ldv] : 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kEpBK; ++t) {
      CT u[4], v[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) u[p] = Us[t][tx + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = Vs[t][ty + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) a[p][q] = fma(u[p], v[q], a[p][q]);
    }
    __syncthreads();
  }
  double z2 = 0.0;
  const double inv_mu_next = 1.0 / mu_next;
  const double thr = lam * inv_mu_next;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = j0 + ty + 16 * q;
    if (gj >= n) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int gi = i0 + tx + 16 * p;
      if (gi >= m) continue;
      const size_t o = gi + (size_t)gj * ld;
      const double av = MODE == EP_PRE ? Aout[o] : (double)a[p][q];
      if (MODE == EP_FINAL) {
        Aout[o] = av;
      } else {
        const double d = D[o];
        const double z = d - av - Ein[o];
        const double y = fma(mu, z, Y[o]);
        z2 = fma(z, z, z2);
        const double e = shrink(fma(y, inv_mu_next, d - av), thr);
        Y[o] = y;
        Eout[o] = e;
        Wout[o] = fma(y, inv_mu_next, d - e);
      }
    }
  }
  if (MODE != EP_FINAL) {
    red[threadIdx.x] = z2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x + (size_t)blockIdx.y * gridDim.x] = red[0];
  }
}

// First iteration (A = 0): Y = D / J, E = Theta_{lam/mu}(D + Y/mu), W = D - E + Y/mu.
__global__ void rpca_start(int m, int n, int ld, const double* __restrict__ D, double invJ, double mu,
                           double lam, double* E, double* Y, double* W) {
  const size_t total = (size_t)m * n;
  const double inv_mu = 1.0 / mu;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t o = (e % m) + (e / m) * (size_t)ld;
    const double d = D[o];
    const double y = d * invJ;
    const double ev = shrink(fma(y, inv_mu, d), lam * inv_mu);
    Y[o] = y;
    E[o] = ev;
    W[o] = fma(y, inv_mu, d - ev);
  }
}

__global__ void maxabs_partial(int m, int n, int ld, const double* __restrict__ D, double* part,
                               int* nonfinite) {
  __shared__ double red[256];
  double acc = 0.0;
  int bad = 0;
  const size_t total = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double v = D[(e % m) + (e / m) * (size_t)ld];
    if (!isfinite(v)) bad = 1;
    acc = fmax(acc, fabs(v));
  }
  if (bad) atomicOr(nonfinite, 1);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void reduce_max(int n, const double* __restrict__ part, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fmax(acc, part[i]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void reduce_sum(int n, const double* __restrict__ part, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void count_nonzero(int m, int n, int ld, const double* __restrict__ E,
                              unsigned long long* out) {
  __shared__ unsigned long long red[256];
  unsigned long long c = 0;
  const size_t total = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    c += E[(e % m) + (e / m) * (size_t)ld] != 0.0 ? 1 : 0;
  red[threadIdx.x] = c;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);  // integer sum: order-independent
}

// Us(:, t) = U(:, t) th_t, m x r
__global__ void scale_columns(int m, int r, const double* __restrict__ U, const double* __restrict__ th,
                              double* __restrict__ Us) {
  const size_t total = (size_t)m * r;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    Us[e] = U[e] * th[e / m];
}

__global__ void thresholds(int r, const double* __restrict__ sigma, double eps,
                           const double* __restrict__ eps_dev, double* th) {
  if (eps_dev) eps = *eps_dev;
  for (int t = threadIdx.x; t < r; t += blockDim.x) th[t] = fmax(sigma[t] - eps, 0.0);
}

// the per-iteration scalars a replayed graph reads: eps, mu, next mu
__global__ void set_scalars(double* slot, double eps, double mu, double mu_next) {
  slot[0] = eps;
  slot[1] = mu;
  slot[2] = mu_next;
}

}  // namespace

// everything of an operator the launches of a BLWS call depend on (graph keys)
void key_operator(GraphKey& k, const Operator& op) {
  k.u(op.m).u(op.n).u(op.sym).p(op.W).u(op.ldw).u(op.nnz).p(op.rowptr).p(op.colidx).p(op.val);
  k.p(op.colptr).p(op.rowidx).p(op.perm).u(op.rl).p(op.Ul).p(op.sl).p(op.Vl);
  for (const OzPlanes* o : {op.Or, op.Oc}) {
    k.p(o);
    if (o) k.p(o->d).p(o->e).u(o->rows).u(o->inner).u(o->ld);
  }
  for (const TcPlanes* t : {op.Wr, op.Wc}) {
    k.p(t);
    if (t) k.p(t->hi).p(t->lo).u(t->rows).u(t->inner).u(t->ld);
  }
}

blws_status spectral_norm(Ctx* ctx, cudaStream_t s, const Operator& op, double* out_host, double stable) {
  // block Lanczos from a seeded block, restarted from its own Ritz vectors
  // (warm start) until the leading Ritz value stops moving
  const int p = std::min(op.m, op.n), N = op.m + op.n;
  const int r = std::min(8, p);
  double *U, *V, *sig, *scal;
  BLWS_TRY(ctx->get(BUF_WARM_U, (size_t)op.m * r, &U));
  BLWS_TRY(ctx->get(BUF_WARM_V, (size_t)op.n * r, &V));
  BLWS_TRY(ctx->get(BUF_SIG, (size_t)2 * r, &sig));
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  double prev = -1.0, cur = 0.0;
  for (int pass = 0; pass < 40; ++pass) {
    BlwsArgs a;
    a.eps = 0.0;
    a.r = r;
    a.k = std::max(1, std::min(8, N / r));
    a.draw = 0xC01Du;
    if (pass == 0) {
      a.cold = true;
    } else {
      a.U0 = U;
      a.ldu0 = op.m;
      a.V0 = V;
      a.ldv0 = op.n;
      a.w = r;
      a.ritz_warm = true;
    }
    // the passes after the first repeat the same launches: graph phases as in
    // the solvers' outer iterations (graph.cuh)
    GraphKey ka;
    ka.u(0x4E524Du).u(1).u(a.r).u(a.k).u(a.w).u(a.cold).p(U).p(V).p(sig).u(ctx->cfg.seed).u(a.draw);
    key_operator(ka, op);
    GraphKey kb = ka;
    kb.v[1] = 2;
    BLWS_TRY(graph_phase(ctx, s, ka, [&](cudaStream_t q) { return blws_run_a(ctx, q, op, a); }));
    BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    BLWS_TRY(graph_harvest(ctx));
    BLWS_TRY(blws_run_mid(ctx, s, op, a));
    BLWS_TRY(graph_phase(ctx, s, kb, [&](cudaStream_t q) -> blws_status {
      BLWS_TRY(blws_run_b(ctx, q, op, a, U, op.m, V, op.n, sig, reinterpret_cast<int*>(scal + SLOT_COUNT),
                          nullptr));
      BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, sig, sizeof(double), cudaMemcpyDeviceToHost, q));
      return BLWS_OK;
    }));
    BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    cur = ctx->host_pinned[0];
    if (fabs(cur - prev) <= stable * fabs(cur)) break;
    prev = cur;
  }
  *out_host = cur;
  return BLWS_OK;
}

blws_status rpca_run(Ctx* ctx, cudaStream_t s, const double* D, int m, int n, int ld,
                     const rpca_params& p, double* A, double* E, rpca_info* info) {
  const int N = m + n;
  const int pmin = std::min(m, n);
  const double lam = p.lambda > 0 ? p.lambda : 1.0 / sqrt((double)std::max(m, n));
  double *Y, *W, *E2, *scal, *red;
  BLWS_TRY(ctx->get(BUF_Y, (size_t)ld * n, &Y));
  BLWS_TRY(ctx->get(BUF_W, (size_t)ld * n, &W));
  BLWS_TRY(ctx->get(BUF_E2, (size_t)ld * n, &E2));
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  const int gb = ctx->sms * 4;
  const dim3 egrid(ceil_div(m, kEpBM), ceil_div(n, kEpBN));
  const int nparts = egrid.x * egrid.y;
  // the reduction buffer is taken once, at its largest size, before any
  // other request can grow it
  BLWS_TRY(ctx->get(BUF_RED, (size_t)std::max(nparts, ctx->sms * 8) + 4096, &red));
  double* zpart = red;
  // norms of D: Frobenius, max-abs (and finiteness)
  int* nonfinite = reinterpret_cast<int*>(scal + SLOT_FLAG);
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(nonfinite, 0, sizeof(int), s));
  // a bounded tensor-core wait that gave up in an earlier call is not this solve's
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(scal + SLOT_TCERR, 0, sizeof(double), s));
  BLWS_TRY(sumsq(ctx, s, m, n, D, ld, scal + SLOT_NORM));
  maxabs_partial<<<gb, 256, 0, s>>>(m, n, ld, D, red, nonfinite);
  BLWS_CHECK_LAUNCH(ctx);
  reduce_max<<<1, 256, 0, s>>>(gb, red, scal + SLOT_AUX);
  BLWS_CHECK_LAUNCH(ctx);
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * SLOT_MAX,
                                     cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  const double d_norm = sqrt(ctx->host_pinned[SLOT_NORM]);
  const double d_inf = ctx->host_pinned[SLOT_AUX];
  if (*reinterpret_cast<int*>(ctx->host_pinned + SLOT_FLAG))
    return ctx->fail(BLWS_ENONFINITE, "rpca_solve: D has NaN/Inf entries");
  info->iters = 0;
  info->rank = 0;
  info->nnzE = 0;
  info->residual = 0.0;
  info->status = BLWS_OK;
  info->mixed_iters = 0;
  info->restarts = 0;
  if (d_norm == 0.0) {  // D = 0: A = E = 0
    BLWS_TRY_CUDA(ctx, cudaMemset2DAsync(A, sizeof(double) * ld, 0, sizeof(double) * m, n, s));
    BLWS_TRY_CUDA(ctx, cudaMemset2DAsync(E, sizeof(double) * ld, 0, sizeof(double) * m, n, s));
    BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    return BLWS_OK;
  }
  Operator Dop;
  Dop.m = m;
  Dop.n = n;
  Dop.W = D;
  Dop.ldw = ld;
  double norm_two = 0.0;
  // ||D||_2 with FP64-equivalent products where the context has them (and in
  // the mixed mode, whose TF32 products could not resolve it to 1e-10): the
  // digit planes of D are built once for all its passes
  const bool norm_oz = ctx->cfg.precision == BLWS_PREC_FP64_TC || ctx->cfg.precision == BLWS_PREC_MIXED;
  OzPlanes Dr{}, Dc{};
  if (norm_oz) {
    BLWS_TRY(oz_alloc(ctx, m, n, &Dr, &Dc));
    BLWS_TRY(oz_planes_from_rows(ctx, s, D, ld, m, n, Dr));
    BLWS_TRY(oz_planes_from_cols(ctx, s, D, ld, 0, m, n, Dc));
    Dop.Or = &Dr;
    Dop.Oc = &Dc;
    ctx->oz_tail = true;  // the block products of the norm estimate too (reset below)
  }
  const blws_status nst = spectral_norm(ctx, s, Dop, &norm_two);
  ctx->oz_tail = false;
  BLWS_TRY(nst);
  info->norm_two = norm_two;
  const double J = std::max(norm_two, d_inf / lam);
  double mu = p.mu0 > 0 ? p.mu0 : 1.25 / norm_two;
  const double mu_bar = mu * p.mu_bar_ratio;

  // warm-start storage sized for the widest block this solve can use
  const int k = ctx->cfg.k, k_cold = ctx->cfg.k_cold;
  const int bcap = std::max(1, std::min(pmin, N / std::max(k, k_cold)));
  double *Uw, *Vw, *sig;
  BLWS_TRY(ctx->get(BUF_WARM_U, (size_t)m * bcap, &Uw));
  BLWS_TRY(ctx->get(BUF_WARM_V, (size_t)n * bcap, &Vw));
  BLWS_TRY(ctx->get(BUF_SIG, (size_t)2 * bcap, &sig));
  double* th = sig + bcap;
  int* count_dev = reinterpret_cast<int*>(scal + SLOT_COUNT);

  const size_t total = (size_t)m * n;
  const int eb = (int)std::min<size_t>((total + 255) / 256, (size_t)ctx->sms * 8);
  double* Ecur = E;
  double* Enext = E2;
  rpca_start<<<eb, 256, 0, s>>>(m, n, ld, D, 1.0 / J, mu, lam, Ecur, Y, W);
  BLWS_CHECK_LAUNCH(ctx);

  Operator Wop;
  Wop.m = m;
  Wop.n = n;
  Wop.W = W;
  Wop.ldw = ld;
  // mixed precision: TF32 planes of W in both orientations, rebuilt from W
  // each iteration until the residual reaches p.mixed_tol
  bool mixed = ctx->cfg.precision == BLWS_PREC_MIXED;
  // FP64-equivalent digit-plane products: the whole solve in a FP64_TC
  // context, and the refinement tail of a mixed one (switched on below)
  bool fp64tc = ctx->cfg.precision == BLWS_PREC_FP64_TC;
  struct TailReset {  // the context's tail switch never outlives this solve
    Ctx* c;
    ~TailReset() { c->oz_tail = false; }
  } tail_reset{ctx};
  int mixed_iters = 0;
  TcPlanes Wr{}, Wc{};
  OzPlanes Or{}, Oc{};
  double* Apre = nullptr;
  // (a mixed solve takes both plane sets from one workspace buffer, the digit
  // planes first, at their larger size: the TF32 planes of the mixed phase
  // and the digit planes of its tail are never in use at the same time)
  if (fp64tc || mixed) BLWS_TRY(oz_alloc(ctx, m, n, &Or, &Oc));
  if (fp64tc || mixed) BLWS_TRY(ctx->get(BUF_RPCA_A, (size_t)ld * n, &Apre));
  if (mixed) {
    const int ldr = tc_ld(n), ldc = tc_ld(m);
    float* wp = nullptr;
    BLWS_TRY(ctx->get(BUF_TC_W, (size_t)2 * m * ldr + (size_t)2 * n * ldc, &wp));
    Wr = TcPlanes{wp, wp + (size_t)m * ldr, m, n, ldr};
    Wc = TcPlanes{wp + (size_t)2 * m * ldr, wp + (size_t)2 * m * ldr + (size_t)n * ldc, n, m, ldc};
  }
  int sv = std::min(std::max(p.sv0, 1), bcap);
  int w = 0;
  int svp = 0;
  double res = 1.0;
  int it = 0;
  bool converged = false;
  for (it = 1; it <= p.max_iter; ++it) {
    if (it > 1) std::swap(Ecur, Enext);  // the E shrunk by the last epilogue
    const double eps = 1.0 / mu;
    BlwsArgs a;
    a.eps = eps;
    a.r = sv;
    a.draw = (uint32_t)it;  // extra columns depend on the iteration only
    a.standard = ctx->cfg.start == 1;
    if (w == 0 || !ctx->cfg.warm) {
      a.cold = true;
      a.k = std::max(1, std::min(k_cold, N / sv));
    } else {
      a.U0 = Uw;
      a.ldu0 = m;
      a.V0 = Vw;
      a.ldv0 = n;
      a.w = w;
      a.ritz_warm = true;
      a.k = std::max(1, std::min(k, N / std::max(sv, w)));
    }
    if (mixed) {
      Wop.Wr = &Wr;
      Wop.Wc = &Wc;
      a.mixed = true;
      ++mixed_iters;
    } else {
      Wop.Wr = Wop.Wc = nullptr;
    }
    if (fp64tc) {
      Wop.Or = &Or;
      Wop.Oc = &Oc;
    }
    const int bw = std::max(a.r, a.w);
    const double mu_next = std::min(mu * p.rho, mu_bar);
    set_scalars<<<1, 1, 0, s>>>(scal + SLOT_EPS, eps, mu, mu_next);
    BLWS_CHECK_LAUNCH(ctx);
    const double* dyn = scal + SLOT_EPS;
    a.guard = ctx->cfg.guard > 0.0;
    a.eps_dev = dyn;
    // phase 1: this iteration's planes of W, the start block, the k block
    // steps and the device stage of the EVD of T_k.  With the Ritz-residual
    // guard, a call whose pairs above eps are not yet accurate is run again
    // from the same start with one more block (at most twice)
    for (int extra = 0;; ++extra) {
      GraphKey ka;
      ka.u(0x52504341u).u(1).u(m).u(n).u(ld).p(W).u(mixed).u(fp64tc).u(a.r).u(a.k).u(a.w);
      ka.u(a.cold).u(a.standard).p(Uw).p(Vw).u(ctx->cfg.seed).u(a.guard).u(a.reorth);
      ka.u(a.cold || bw > a.w ? a.draw : 0u);  // the generator stream matters only for drawn columns
      BLWS_TRY(graph_phase(ctx, s, ka, [&](cudaStream_t q) -> blws_status {
        if (mixed) {
          BLWS_TRY(tc_planes_from_rows(ctx, q, W, ld, m, n, Wr));
          BLWS_TRY(tc_planes_from_cols(ctx, q, W, ld, 0, m, n, Wc));
        }
        if (fp64tc) {  // FP64-equivalent digit planes of this iteration's W
          BLWS_TRY(oz_planes_from_rows(ctx, q, W, ld, m, n, Or));
          BLWS_TRY(oz_planes_from_cols(ctx, q, W, ld, 0, m, n, Oc));
        }
        return blws_run_a(ctx, q, Wop, a);
      }));
      BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
      BLWS_TRY(graph_harvest(ctx));
      if (!a.guard || extra == 2 || (a.k + 1) * bw > N || !(blws_guard_ratio(ctx, a) > ctx->cfg.guard)) break;
      ++a.k;
      a.reorth = true;
      ++info->restarts;
    }
    BLWS_TRY(blws_run_mid(ctx, s, Wop, a));  // the EVD's host stage
    // FP64-equivalent mode: A = (U diag(theta)) V^T over the sv computed pairs
    // (theta is zero past the count) as a digit-plane product, when it is
    // large enough for gemm to route it there
    // mixed mode: the same product from split TF32 operands on the tensor cores
    const bool pre = (fp64tc && sv >= 64) || (mixed && sv >= 16 && std::min(m, n) >= 16);
    // phase 2: Ritz lift, count, thresholds, the fused epilogue and its
    // residual norm, copied back with the count
    GraphKey kb2;
    kb2.u(0x52504341u).u(2).u(m).u(n).u(ld).u(mixed).u(fp64tc).u(a.r).u(a.k).u(a.w).u(pre);
    kb2.p(Uw).p(Vw).p(sig).p(D).p(Ecur).p(Enext).p(Y).p(W).p(Apre).d(lam).p(zpart).u(nparts);
    BLWS_TRY(graph_phase(ctx, s, kb2, [&](cudaStream_t q) -> blws_status {
      BLWS_TRY(blws_run_b(ctx, q, Wop, a, Uw, m, Vw, n, sig, count_dev, dyn));
      thresholds<<<1, 256, 0, q>>>(sv, sig, eps, dyn, th);
      BLWS_CHECK_LAUNCH(ctx);
      if (pre) {
        double* Us = nullptr;
        BLWS_TRY(ctx->get(BUF_P2, (size_t)m * sv, &Us));  // CholeskyQR scratch, free here
        scale_columns<<<std::min(ceil_div((long long)m * sv, 256), ctx->sms * 8), 256, 0, q>>>(
            m, sv, Uw, th, Us);
        BLWS_CHECK_LAUNCH(ctx);
        BLWS_TRY(gemm(ctx, q, false, true, m, n, sv, 1.0, Us, m, Vw, n, 0.0, Apre, ld, mixed));
        rpca_epilogue<EP_PRE, double><<<egrid, 256, 0, q>>>(m, n, ld, Uw, m, th, Vw, n, count_dev, D,
                                                            Ecur, Enext, Y, W, Apre, mu, mu_next,
                                                            lam, zpart, dyn);
      } else if (mixed)
        rpca_epilogue<EP_ITER, float><<<egrid, 256, 0, q>>>(m, n, ld, Uw, m, th, Vw, n, count_dev, D,
                                                            Ecur, Enext, Y, W, nullptr, mu, mu_next,
                                                            lam, zpart, dyn);
      else
        rpca_epilogue<EP_ITER, double><<<egrid, 256, 0, q>>>(m, n, ld, Uw, m, th, Vw, n, count_dev, D,
                                                             Ecur, Enext, Y, W, nullptr, mu, mu_next,
                                                             lam, zpart, dyn);
      BLWS_CHECK_LAUNCH(ctx);
      reduce_sum<<<1, 256, 0, q>>>(nparts, zpart, scal + SLOT_NORM);
      BLWS_CHECK_LAUNCH(ctx);
      BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * SLOT_MAX,
                                         cudaMemcpyDeviceToHost, q));
      return BLWS_OK;
    }));
    BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    svp = *reinterpret_cast<int*>(ctx->host_pinned + SLOT_COUNT);
    const double z2 = ctx->host_pinned[SLOT_NORM];
    if (!isfinite(z2)) return ctx->fail(BLWS_ENONFINITE, "rpca_solve: iterate became non-finite");
    res = sqrt(z2) / d_norm;
    if (*reinterpret_cast<int*>(ctx->host_pinned + SLOT_TCERR))
      return ctx->fail(BLWS_ETIMEOUT, "rpca_solve: a tensor-core wait ran out");
    if (p.trace && it <= p.trace_len) {
      p.trace[3 * (it - 1) + 0] = res;
      p.trace[3 * (it - 1) + 1] = svp;
      p.trace[3 * (it - 1) + 2] = sv;
    }
    w = sv;
    // [Lin09] rank prediction for the next iteration
    int nsv = svp < sv ? std::min(svp + 1, n) : std::min(svp + (int)lround(0.05 * n), n);
    sv = std::max(1, std::min(nsv, bcap));
    mu = mu_next;
    if (res < p.tol) {
      converged = true;
      break;
    }
    if (mixed && res < p.mixed_tol) {
      // the refinement tail: FP64-equivalent products (BF16 digit planes on the
      // tensor cores, errors at the FP64 level) from here on
      mixed = false;
      fp64tc = true;
      ctx->oz_tail = true;
    }
  }
  if (!converged) it = p.max_iter;
  // outputs: A = U diag(th) V^T of the last SVT; E = the E of that iteration
  rpca_epilogue<EP_FINAL, double><<<egrid, 256, 0, s>>>(m, n, ld, Uw, m, th, Vw, n, count_dev,
                                                        nullptr, nullptr, nullptr, nullptr, nullptr,
                                                        A, 0.0, 1.0, 0.0, nullptr, nullptr);
  BLWS_CHECK_LAUNCH(ctx);
  if (Ecur != E) {
    BLWS_TRY_CUDA(ctx, cudaMemcpy2DAsync(E, sizeof(double) * ld, Ecur, sizeof(double) * ld,
                                         sizeof(double) * m, n, cudaMemcpyDeviceToDevice, s));
  }
  unsigned long long* nz = reinterpret_cast<unsigned long long*>(scal + SLOT_NNZ);
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(nz, 0, sizeof(unsigned long long), s));
  count_nonzero<<<eb, 256, 0, s>>>(m, n, ld, E, nz);
  BLWS_CHECK_LAUNCH(ctx);
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, scal, sizeof(double) * SLOT_MAX,
                                     cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  info->iters = it;
  info->rank = svp;
  info->nnzE = (int64_t)*reinterpret_cast<unsigned long long*>(ctx->host_pinned + SLOT_NNZ);
  info->residual = res;
  info->status = converged ? BLWS_OK : BLWS_ENOCONV;
  info->mixed_iters = mixed_iters;
  return converged ? BLWS_OK : BLWS_ENOCONV;
}

}  // namespace blws
