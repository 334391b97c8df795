// FP64 GEMM and reductions on CUDA cores (DFMA).
//
// On GB300 FP64 runs at 1/64 of the FP32 rate (about 2 DFMA per clock per
// SM), so every FP64 product here is bound by the DFMA pipe, not by memory:
// the tiling only has to keep all 152 SMs busy.  Tiles of BM x BN outputs
// per 256-thread CTA; when the tile count cannot fill the GPU the K range is
// split and the partial sums are reduced in a fixed order (deterministic, no
// atomics).
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include "ops.cuh"
#include "tune.cuh"

namespace blws {

namespace {

constexpr int kThreads = 256;
constexpr int kBK = 16;

// CT: the arithmetic type of the products and of the in-CTA sums (double,
// or float in the mixed-precision mode); inputs, outputs and the split-K
// reduction are FP64 either way.
template <typename CT, bool TA, bool TB, int BM, int BN>
__global__ void __launch_bounds__(kThreads)
gemm_f64_kernel(int M, int N, int K, int kchunk, double alpha, const double* __restrict__ A,
                int lda, const double* __restrict__ B, int ldb, double beta, double* C, int ldc,
                double* __restrict__ part, int sym) {
  // TX x TY threads over the tile, TM x TN outputs each: 16 x 16 threads, or
  // for tiles narrower than 16 columns 256 / BN threads down the rows
  constexpr int TX = BN >= 16 ? 16 : kThreads / BN, TY = kThreads / TX;
  constexpr int TM = BM / TX, TN = BN / TY;
  static_assert(TM >= 1 && TN >= 1 && TM * TX == BM && TN * TY == BN, "tile shape");
  __shared__ CT As[kBK][BM + 1];
  __shared__ CT Bs[kBK][BN + 1];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  // sym: the result is symmetric (M = N); a tile wholly below the diagonal is
  // left to its mirror image
  if (sym && m0 > n0 + BN - 1) return;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  CT acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = CT(0);

  for (int k0 = kbeg; k0 < kend; k0 += kBK) {
#pragma unroll 4
    for (int e = threadIdx.x; e < BM * kBK; e += kThreads) {
      int i, kk;
      if (!TA) { i = e % BM; kk = e / BM; } else { kk = e % kBK; i = e / kBK; }
      const int gi = m0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < M && gk < kend) v = TA ? A[gk + (size_t)gi * lda] : A[gi + (size_t)gk * lda];
      As[kk][i] = (CT)v;
    }
#pragma unroll 4
    for (int e = threadIdx.x; e < kBK * BN; e += kThreads) {
      int kk, j;
      if (!TB) { kk = e % kBK; j = e / kBK; } else { j = e % BN; kk = e / BN; }
      const int gj = n0 + j, gk = k0 + kk;
      double v = 0.0;
      if (gj < N && gk < kend) v = TB ? B[gj + (size_t)gk * ldb] : B[gk + (size_t)gj * ldb];
      Bs[kk][j] = (CT)v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      CT a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + TX * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ty + TY * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gi = m0 + tx + TX * i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = n0 + ty + TY * j;
      if (gj >= N) continue;
      const double av = (double)acc[i][j];
      if (part) {
        part[(size_t)blockIdx.z * M * N + gi + (size_t)gj * M] = av;
      } else if (!sym) {
        double* c = C + gi + (size_t)gj * ldc;
        *c = beta == 0.0 ? alpha * av : fma(alpha, av, beta * *c);
      } else if (gi <= gj) {  // (beta = 0) the upper triangle and its mirror, each written once
        C[gi + (size_t)gj * ldc] = alpha * av;
        C[gj + (size_t)gi * ldc] = alpha * av;
      }
    }
  }
}

// C = alpha (sum of the split-K partials) + beta C.  Each output is summed by
// a group of G lanes (G a power of two up to 32, chosen so that small outputs
// with many splits still fill the GPU): lane q of the group adds partials q,
// q + G, ... in order (loads issued 8 at a time), then the group adds its lanes
// with a fixed shuffle tree -- a fixed order for given M, N, splits.
__global__ void splitk_reduce(int M, int N, int splits, int G, double alpha, const double* __restrict__ part,
                              double beta, double* C, int ldc, int sym) {
  const size_t total = (size_t)M * N;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t nth = (size_t)gridDim.x * blockDim.x;
  const int q = (int)(tid % G);
  // every lane of a warp runs the same number of iterations (the shuffles need them all)
  const size_t span = (total * G + nth - 1) / nth * nth;
  for (size_t t = tid; t < span; t += nth) {
    const size_t e = t / G;
    double acc = 0.0;
    if (e < total) {
      // sym (M = N): an element below the diagonal sums its mirror's partials
      size_t src = e;
      if (sym) {
        const size_t i = e % M, j = e / M;
        if (i > j) src = j + i * (size_t)M;
      }
      int z = q;
      for (; z + 7 * G < splits; z += 8 * G) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = part[(size_t)(z + u * G) * total + src];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
      }
      for (; z < splits; z += G) acc += part[(size_t)z * total + src];
    }
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (q == 0 && e < total) {
      const int i = (int)(e % M), j = (int)(e / M);
      double* c = C + i + (size_t)j * ldc;
      *c = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *c);
    }
  }
}

// FP32 sums inside one CTA cover at most this much of K (the rest is summed
// in FP64 by the split-K reduction)
constexpr int kF32MaxChunk = 256;

// target: CTAs the K split aims for (0: no split beyond the FP32 chunk rule)
template <typename CT, bool TA, bool TB, int BM, int BN>
blws_status launch_tiles(Ctx* ctx, cudaStream_t s, int M, int N, int K, double alpha,
                         const double* A, int lda, const double* B, int ldb, double beta,
                         double* C, int ldc, bool sym, int target) {
  const int tm = ceil_div(M, BM), tn = ceil_div(N, BN);
  const int tiles = tm * tn;
  int splits = 1;
  if (tiles < target && K > 2 * kBK) {
    splits = ceil_div(target, tiles);
    splits = min(splits, ceil_div(K, 2 * kBK));
    splits = max(splits, 1);
  }
  if (sizeof(CT) < sizeof(double)) splits = max(splits, ceil_div(K, kF32MaxChunk));
  int kchunk = ceil_div(ceil_div(K, splits), kBK) * kBK;
  splits = ceil_div(K, kchunk);
  double* part = nullptr;
  if (splits > 1) BLWS_TRY(ctx->get(BUF_SPLITK, (size_t)splits * M * N, &part));
  dim3 grid(tm, tn, splits);
  gemm_f64_kernel<CT, TA, TB, BM, BN><<<grid, kThreads, 0, s>>>(M, N, K, kchunk, alpha, A, lda, B,
                                                                ldb, beta, C, ldc, part, sym ? 1 : 0);
  BLWS_CHECK_LAUNCH(ctx);
  if (splits > 1) {
    const size_t total = (size_t)M * N;
    // lanes per output: enough to fill ~8 x 256 threads per SM, at most 32 and the split count
    int G = 1;
    while (G < 32 && 2 * G <= splits && total * (size_t)(2 * G) <= (size_t)ctx->sms * 8 * 256) G *= 2;
    const int blocks = (int)std::min<size_t>((total * G + 255) / 256, (size_t)ctx->sms * 8);
    splitk_reduce<<<blocks, 256, 0, s>>>(M, N, splits, G, alpha, part, beta, C, ldc, sym ? 1 : 0);
    BLWS_CHECK_LAUNCH(ctx);
  }
  return BLWS_OK;
}

constexpr int kShapes[5][2] = {{64, 64}, {64, 32}, {128, 16}, {16, 16}, {32, 8}};

// The tile shape that wastes the fewest FMAs on padding (the DFMA pipe, not
// shared-memory traffic, bounds every shape here); ties go to the earlier,
// larger tile.  32 x 8 serves block widths just above a multiple of 16
// (b = 101 pads to 104 instead of 112).
int padding_tile(int M, int N) {
  int best = 0;
  long long best_work = -1;
  for (int t = 0; t < 5; ++t) {
    const long long work = (long long)ceil_div(M, kShapes[t][0]) * kShapes[t][0] *
                           ((long long)ceil_div(N, kShapes[t][1]) * kShapes[t][1]);
    if (best_work < 0 || work < best_work) {
      best = t;
      best_work = work;
    }
  }
  return best;
}

// DFMA-bound: balance the SMs.  The fixed rule aims for about 8 CTAs per SM
// (of which ~4 are resident at once), which keeps the tail of the last wave
// under ~1/8 of the run; the inner dimension is split (chunks >= 32) until
// that many CTAs exist.  The autotuner picks among 0, 2, 4 and 8 per SM.
int split_target(const Ctx* ctx, int q) { return q == 0 ? 0 : (1 << q) * ctx->sms; }
constexpr int kDefaultSplit = 3;

template <typename CT, bool TA, bool TB>
blws_status launch_choice(Ctx* ctx, cudaStream_t s, int tile, int target, int M, int N, int K,
                          double alpha, const double* A, int lda, const double* B, int ldb,
                          double beta, double* C, int ldc, bool sym) {
  switch (tile) {
    case 0: return launch_tiles<CT, TA, TB, 64, 64>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym, target);
    case 1: return launch_tiles<CT, TA, TB, 64, 32>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym, target);
    case 2: return launch_tiles<CT, TA, TB, 128, 16>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym, target);
    case 3: return launch_tiles<CT, TA, TB, 16, 16>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym, target);
    default: return launch_tiles<CT, TA, TB, 32, 8>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym, target);
  }
}

// ------------------------------------------------------------ autotuner --
// With blws_config.tune, the tile shape and the K split of each product come
// from timing every (shape, split) pair on the product's own dimensions the
// first time a size bucket is met: each dimension is rounded up on a ladder
// of quarter-octaves (exact up to 32), so one measurement serves the products
// within ~25% of it.  Choices are process-wide (per SM count), kept in memory
// and, when the environment variable BLWS_TUNE_FILE names a file, read from it
// at first use and appended to it as they are made, so later processes start
// tuned.  A choice is kept unless it beats the fixed rule by 5%, so timing
// noise does not move products off the rule for nothing.  Inside a graph
// capture no timing can run: an untuned bucket there breaks the capture, and
// the phase runs directly (and tunes).
TuneKey tune_key(const Ctx* ctx, int ct_bytes, bool ta, bool tb, bool sym, int M, int N, int K) {
  return TuneKey{{ctx->sms, ct_bytes == 8 ? kTuneF64 : kTuneF32, ta, tb, sym, tune_bucket(M), tune_bucket(N),
                  tune_bucket(K)}};
}

template <typename CT, bool TA, bool TB>
blws_status tune_shape(Ctx* ctx, cudaStream_t s, int M, int N, int K, bool sym, const TuneKey& key,
                       TuneChoice* out) {
  const int lda = TA ? K : M, ldb = TB ? N : K;
  const size_t na = (size_t)lda * (TA ? M : K), nb = (size_t)ldb * (TB ? K : N), nc = (size_t)M * N;
  double* w = nullptr;
  BLWS_TRY(ctx->get(BUF_TUNE, na + nb + nc, &w));
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(w, 0, sizeof(double) * (na + nb + nc), s));
  const double* A = w;
  const double* B = w + na;
  double* C = w + na + nb;
  cudaEvent_t e0, e1;
  BLWS_TRY_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ctx->fail(BLWS_ECUDA, "autotuner events");
  }
  const TuneChoice rule{padding_tile(M, N), kDefaultSplit};
  TuneChoice best = rule;
  float best_ms = -1.0f, rule_ms = -1.0f;
  blws_status st = BLWS_OK;
  for (int t = 0; t < 5 && st == BLWS_OK; ++t)
    for (int q = 0; q <= 3 && st == BLWS_OK; ++q) {
      const int target = split_target(ctx, q);
      // one launch to warm up, three timed
      st = launch_choice<CT, TA, TB>(ctx, s, t, target, M, N, K, 1.0, A, lda, B, ldb, 0.0, C, M, sym);
      if (st != BLWS_OK) break;
      if (cudaEventRecord(e0, s) != cudaSuccess) st = ctx->fail(BLWS_ECUDA, "autotuner event");
      for (int r = 0; r < 3 && st == BLWS_OK; ++r)
        st = launch_choice<CT, TA, TB>(ctx, s, t, target, M, N, K, 1.0, A, lda, B, ldb, 0.0, C, M, sym);
      if (st != BLWS_OK) break;
      float ms = 0.0f;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = ctx->fail(BLWS_ECUDA, "autotuner timing");
        break;
      }
      if (t == rule.a && q == rule.b) rule_ms = ms;
      if (best_ms < 0.0f || ms < best_ms) {
        best_ms = ms;
        best = TuneChoice{t, q};
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BLWS_TRY(st);
  if (!(best_ms < 0.95f * rule_ms)) best = rule;
  tune_store(key, best);
  *out = best;
  return BLWS_OK;
}

template <typename CT, bool TA, bool TB>
blws_status gemm_t(Ctx* ctx, cudaStream_t s, int M, int N, int K, double alpha, const double* A,
                   int lda, const double* B, int ldb, double beta, double* C, int ldc, bool sym) {
  TuneChoice c{padding_tile(M, N), kDefaultSplit};
  if (ctx->cfg.tune) {
    const TuneKey key = tune_key(ctx, (int)sizeof(CT), TA, TB, sym, M, N, K);
    if (!tune_lookup(key, &c)) {
      if (ctx->capturing) {
        ctx->capture_broken = true;
        return ctx->fail(BLWS_ECUDA, "untuned product shape inside a graph capture");
      }
      BLWS_TRY((tune_shape<CT, TA, TB>(ctx, s, M, N, K, sym, key, &c)));
    }
  }
  return launch_choice<CT, TA, TB>(ctx, s, c.a, split_target(ctx, c.b), M, N, K, alpha, A, lda, B,
                                   ldb, beta, C, ldc, sym);
}

// ------------------------------------------------------------ reductions --
__global__ void sumsq_partial(int M, int N, const double* __restrict__ A, int ld, double* part) {
  __shared__ double red[256];
  double acc = 0.0;
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double v = A[(e % M) + (e / M) * (size_t)ld];
    acc = fma(v, v, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sum_final(int n, const double* __restrict__ part, double* out) {
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

// one CTA per column (tall columns: thousands of rows, a hundred-odd
// columns), sums in a fixed order
__global__ void __launch_bounds__(256) col_norms_kernel(int M, int N, const double* __restrict__ A, int ld,
                                                        double* out) {
  __shared__ double red[8];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const double* a = A + (size_t)blockIdx.x * ld;
  double acc = 0.0;
  for (int i = threadIdx.x; i < M; i += 256) acc = fma(a[i], a[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[blockIdx.x] = sqrt(t);
  }
}

__global__ void max_final(int n, const double* __restrict__ v, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fmax(acc, v[i]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void scale_kernel(int M, int N, double beta, double* C, int ldc) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    double* c = C + (e % M) + (e / M) * (size_t)ldc;
    *c = beta == 0.0 ? 0.0 : beta * *c;
  }
}

}  // namespace

namespace {

bool oz_mode(const Ctx* ctx) {
  return ctx->cfg.precision == BLWS_PREC_FP64_TC || ctx->cfg.precision == BLWS_PREC_MIXED || ctx->oz_tail;
}

blws_status gemm_any(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                     const double* A, int lda, const double* B, int ldb, double beta, double* C,
                     int ldc, bool fp32, bool sym) {
  if (fp32) {
    if (!ta && !tb) return gemm_t<float, false, false>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
    if (ta && !tb) return gemm_t<float, true, false>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
    if (!ta && tb) return gemm_t<float, false, true>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
    return gemm_t<float, true, true>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
  }
  if (!ta && !tb) return gemm_t<double, false, false>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
  if (ta && !tb) return gemm_t<double, true, false>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
  if (!ta && tb) return gemm_t<double, false, true>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
  return gemm_t<double, true, true>(ctx, s, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
}

}  // namespace

blws_status gemm(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                 const double* A, int lda, const double* B, int ldb, double beta, double* C,
                 int ldc, bool fp32) {
  if (M <= 0 || N <= 0) return BLWS_OK;
  if (K <= 0) {  // C = beta C
    const size_t total = (size_t)M * N;
    scale_kernel<<<(int)std::min<size_t>((total + 255) / 256, (size_t)ctx->sms * 8), 256, 0, s>>>(
        M, N, beta, C, ldc);
    BLWS_CHECK_LAUNCH(ctx);
    return BLWS_OK;
  }
  // A^T A (the Gram matrices): symmetric, so one triangle of tiles is computed
  const bool sym = ta && !tb && A == B && lda == ldb && M == N && beta == 0.0;
  // FP64-level products of the tensor-core modes (in the mixed mode: the
  // eigen stage's refinement, blocks too wide for the TF32 accumulator, the
  // refinement tail) as digit-plane products once they are large enough
  if (!fp32 && oz_mode(ctx) && (double)M * N * K >= kOzGemmMin && std::min(M, N) >= 16 && K >= 64)
    return oz_gemm(ctx, s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
  // mixed precision: the FP32-level block products on the tensor cores (TF32 hi + lo)
  if (fp32 && ctx->cfg.precision == BLWS_PREC_MIXED && (double)M * N * K >= kTcGemmMin &&
      std::min(M, N) >= 16 && K >= 32)
    return tc_gemm(ctx, s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym);
  return gemm_any(ctx, s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, fp32, sym);
}

blws_status gemm_sym(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int n, int K, double alpha,
                     const double* A, int lda, const double* B, int ldb, double* C, int ldc, bool fp32) {
  if (n <= 0) return BLWS_OK;
  if (K <= 0) return gemm(ctx, s, ta, tb, n, n, K, alpha, A, lda, B, ldb, 0.0, C, ldc, fp32);
  if (!fp32 && oz_mode(ctx) && (double)n * n * K >= kOzGemmMin && n >= 16 && K >= 64)
    return oz_gemm(ctx, s, ta, tb, n, n, K, alpha, A, lda, B, ldb, 0.0, C, ldc, true);
  if (fp32 && ctx->cfg.precision == BLWS_PREC_MIXED && (double)n * n * K >= kTcGemmMin && n >= 16 &&
      K >= 32 && n <= 256)
    return tc_gemm(ctx, s, ta, tb, n, n, K, alpha, A, lda, B, ldb, 0.0, C, ldc, true);
  return gemm_any(ctx, s, ta, tb, n, n, K, alpha, A, lda, B, ldb, 0.0, C, ldc, fp32, true);
}

blws_status sumsq(Ctx* ctx, cudaStream_t s, int M, int N, const double* A, int ld, double* out) {
  double* part = nullptr;
  const int blocks = ctx->sms * 2;
  BLWS_TRY(ctx->get(BUF_RED, (size_t)blocks, &part));
  sumsq_partial<<<blocks, 256, 0, s>>>(M, N, A, ld, part);
  BLWS_CHECK_LAUNCH(ctx);
  sum_final<<<1, 256, 0, s>>>(blocks, part, out);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

blws_status col_norms(Ctx* ctx, cudaStream_t s, int M, int N, const double* A, int ld,
                      double* out, double* colmax) {
  if (N > 0) {
    col_norms_kernel<<<N, 256, 0, s>>>(M, N, A, ld, out);
    BLWS_CHECK_LAUNCH(ctx);
  }
  if (colmax) {
    max_final<<<1, 256, 0, s>>>(N, out, colmax);
    BLWS_CHECK_LAUNCH(ctx);
  }
  return BLWS_OK;
}

}  // namespace blws

// ------------------------------------------------ allocation-free product --
// blws_apply_noalloc: the product with the augmented matrix for callers that
// cannot allocate device memory.  Its only scratch (the split-K partial sums
// of the two GEMMs) lives in this file-scope array, which every GPU that
// loads the library holds until the process exits.
namespace blws {
namespace {

constexpr size_t kNoAllocScratchDoubles = (size_t)2 << 20;  // 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
int g_noalloc_sms[kNoAllocMaxDevices] = {0};

// Device address of the scratch array in the current context, and the SM
// count (looked up once per device).  The address is looked up on every call
// (no allocation, no synchronisation): it belongs to a context, and a cached
// copy would go stale after cudaDeviceReset or point into another context
// when the caller runs in a driver-API context of its own.
blws_status noalloc_setup(int dev, double** addr, int* sms) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return BLWS_ENOTSUP;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
    cudaGetLastError();
    return BLWS_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_sms[dev]) {
    int count = 0;
    if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return BLWS_ECUDA;
    }
    g_noalloc_sms[dev] = count;
  }
  *addr = static_cast<double*>(p);
  *sms = g_noalloc_sms[dev];
  return BLWS_OK;
}

// The split-K factor of this path.  It is deliberately coarser than the
// allocating path's (about two CTAs per SM instead of eight, and only for an
// inner dimension above 4 k-blocks), to bound the static scratch; the tile
// shape follows N alone instead of the padding-minimising search.  So the
// results agree with blws_apply to rounding, not bit for bit.
template <int BM, int BN>
int noalloc_splits(int sms, int M, int N, int K, int* kchunk) {
  const int tiles = ceil_div(M, BM) * ceil_div(N, BN);
  const int target = 2 * sms;
  int splits = 1;
  if (tiles < target && K > 4 * kBK) {
    splits = ceil_div(target, tiles);
    splits = min(splits, ceil_div(K, 4 * kBK));
    splits = max(splits, 1);
  }
  *kchunk = ceil_div(ceil_div(K, splits), kBK) * kBK;
  return ceil_div(K, *kchunk);
}

template <bool TA, int BM, int BN>
size_t noalloc_need(int sms, int M, int N, int K) {
  int kchunk;
  const int splits = noalloc_splits<BM, BN>(sms, M, N, K, &kchunk);
  return splits > 1 ? (size_t)splits * M * N : 0;
}

template <bool TA, int BM, int BN>
cudaError_t noalloc_gemm(cudaStream_t s, int sms, double* scratch, int M, int N, int K,
                         const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
  int kchunk;
  const int splits = noalloc_splits<BM, BN>(sms, M, N, K, &kchunk);
  double* part = splits > 1 ? scratch : nullptr;
  dim3 grid(ceil_div(M, BM), ceil_div(N, BN), splits);
  gemm_f64_kernel<double, TA, false, BM, BN><<<grid, kThreads, 0, s>>>(M, N, K, kchunk, 1.0, A, lda, B, ldb,
                                                               0.0, C, ldc, part, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const size_t total = (size_t)M * N;
  int G = 1;  // the same lane-group rule as the context path
  while (G < 32 && 2 * G <= splits && total * (size_t)(2 * G) <= (size_t)sms * 8 * 256) G *= 2;
  const int blocks = (int)std::min<size_t>((total * G + 255) / 256, (size_t)sms * 8);
  splitk_reduce<<<blocks, 256, 0, s>>>(M, N, splits, G, 1.0, part, 0.0, C, ldc, 0);
  return cudaGetLastError();
}

template <bool TA>
size_t noalloc_need_any(int sms, int M, int N, int K) {
  if (N <= 16) return noalloc_need<TA, 128, 16>(sms, M, N, K);
  if (N <= 32) return noalloc_need<TA, 64, 32>(sms, M, N, K);
  return noalloc_need<TA, 64, 64>(sms, M, N, K);
}

template <bool TA>
cudaError_t noalloc_gemm_any(cudaStream_t s, int sms, double* scratch, int M, int N, int K,
                             const double* A, int lda, const double* B, int ldb, double* C,
                             int ldc) {
  if (N <= 16) return noalloc_gemm<TA, 128, 16>(s, sms, scratch, M, N, K, A, lda, B, ldb, C, ldc);
  if (N <= 32) return noalloc_gemm<TA, 64, 32>(s, sms, scratch, M, N, K, A, lda, B, ldb, C, ldc);
  return noalloc_gemm<TA, 64, 64>(s, sms, scratch, M, N, K, A, lda, B, ldb, C, ldc);
}

}  // namespace

}  // namespace blws

extern "C" blws_status blws_apply_noalloc(const double* W, int m, int n, int ldw, const double* X,
                                          int ldx, int b, double* P, int ldp, void* stream) {
  using namespace blws;
  if (!W || !X || !P) return BLWS_EINVAL;
  if (m < 1 || n < 1 || b < 1 || ldw < m || ldx < m + n || ldp < m + n) return BLWS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BLWS_ECUDA;
  }
  double* scratch = nullptr;
  int sms = 0;
  blws_status st = noalloc_setup(dev, &scratch, &sms);
  if (st != BLWS_OK) return st;
  // P_u = W X_v (m x b, inner n) and P_v = W^T X_u (n x b, inner m); they run
  // one after the other on the stream, so each may use the whole array
  if (noalloc_need_any<false>(sms, m, b, n) > kNoAllocScratchDoubles ||
      noalloc_need_any<true>(sms, n, b, m) > kNoAllocScratchDoubles)
    return BLWS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (noalloc_gemm_any<false>(s, sms, scratch, m, b, n, W, ldw, X + m, ldx, P, ldp) != cudaSuccess ||
      noalloc_gemm_any<true>(s, sms, scratch, n, b, m, W, ldw, X, ldx, P + m, ldp) != cudaSuccess)
    return BLWS_ECUDA;
  return BLWS_OK;
}

// ------------------------------------------------------ autotuner table --
namespace blws {
namespace {
std::mutex g_tune_mutex;
std::map<TuneKey, TuneChoice> g_tune;
bool g_tune_loaded = false;

bool tune_valid(const TuneKey& k, const TuneChoice& c) {
  if (k.v[1] == kTuneDigits) return c.a >= 1 && c.a <= 4096 && c.b == 0;
  return (k.v[1] == kTuneF32 || k.v[1] == kTuneF64) && c.a >= 0 && c.a < 5 && c.b >= 0 && c.b <= 3;
}

// (the mutex is held)
void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("BLWS_TUNE_FILE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  TuneKey k;
  TuneChoice c;
  while (std::fscanf(f, "tune %d %d %d %d %d %d %d %d %d %d\n", &k.v[0], &k.v[1], &k.v[2], &k.v[3],
                     &k.v[4], &k.v[5], &k.v[6], &k.v[7], &c.a, &c.b) == 10)
    if (tune_valid(k, c)) g_tune[k] = c;
  std::fclose(f);
}
}  // namespace

int tune_bucket(int x) {
  if (x <= 32) return x;
  int p = 32;
  while (2 * p < x) p *= 2;  // p < x <= 2p
  const int step = p / 4;
  return ceil_div(x, step) * step;
}

bool tune_lookup(const TuneKey& k, TuneChoice* c) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load();
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *c = it->second;
  return true;
}

void tune_store(const TuneKey& k, const TuneChoice& c) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load();
  if (!g_tune.emplace(k, c).second) return;  // another context tuned it first
  const char* path = std::getenv("BLWS_TUNE_FILE");
  if (!path || !*path) return;
  if (FILE* f = std::fopen(path, "a")) {
    std::fprintf(f, "tune %d %d %d %d %d %d %d %d %d %d\n", k.v[0], k.v[1], k.v[2], k.v[3], k.v[4],
                 k.v[5], k.v[6], k.v[7], c.a, c.b);
    std::fclose(f);
  }
}

size_t tune_count() {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load();
  return g_tune.size();
}

}  // namespace blws

extern "C" size_t blws_tune_count(void) { return blws::tune_count(); }
