// Sparse operator pieces for matrix completion: the CSR -> CSC mirror of the
// observed pattern, the products S X and S^T X (CSR SpMM), the low-rank term
// of the "sparse residual plus low-rank" operator, and the sampled product
// x_ij = sum_t U_it theta_t V_jt on Omega (SDDMM) fused with the host's update.
#include <algorithm>

#include "blws_core.cuh"
#include "mc_kernels.cuh"

namespace blws {

namespace {

__global__ void count_cols(int nnz, const int* __restrict__ colidx, int* cnt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x)
    atomicAdd(&cnt[colidx[e]], 1);  // integer histogram: order-independent
}

// exclusive scan of cnt[0:n] into ptr[0:n+1] (one CTA, sequential chunks)
__global__ void scan_ptr(int n, const int* __restrict__ cnt, int* ptr, int* cursor) {
  __shared__ int sums[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int chunk = (n + nt - 1) / nt;
  const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += cnt[i];
  sums[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int t = 0; t < nt; ++t) {
      const int v = sums[t];
      sums[t] = acc;
      acc += v;
    }
    ptr[n] = acc;
  }
  __syncthreads();
  int acc = sums[tid];
  for (int i = lo; i < hi; ++i) {
    const int ci = cnt[i];  // cursor may alias cnt: read before writing
    ptr[i] = acc;
    cursor[i] = acc;
    acc += ci;
  }
}

__global__ void scatter_csc(int m, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                            int* cursor, int* rowidx, int* perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int pos = atomicAdd(&cursor[colidx[e]], 1);
      rowidx[pos] = i;
      perm[pos] = e;
    }
  }
}

// sort each column segment by row (the scatter above leaves it in arrival
// order), which makes the CSC mirror deterministic: one CTA per column, a
// bitonic sort of (row, CSR position) pairs in shared memory (rows within a
// column are distinct, so the order is unique); a segment longer than the
// shared buffer falls back to an insertion sort by one thread.
constexpr int kSortMax = 4096;

__global__ void __launch_bounds__(256)
sort_segments(int n, const int* __restrict__ colptr, int* rowidx, int* perm) {
  __shared__ int key[kSortMax];
  __shared__ int val[kSortMax];
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    const int lo = colptr[j], len = colptr[j + 1] - lo;
    if (len <= 1) continue;
    if (len > kSortMax) {
      if (threadIdx.x == 0) {
        for (int a = lo + 1; a < lo + len; ++a) {
          const int r = rowidx[a], p = perm[a];
          int b = a - 1;
          while (b >= lo && rowidx[b] > r) {
            rowidx[b + 1] = rowidx[b];
            perm[b + 1] = perm[b];
            --b;
          }
          rowidx[b + 1] = r;
          perm[b + 1] = p;
        }
      }
      __syncthreads();
      continue;
    }
    int P = 1;
    while (P < len) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      key[i] = i < len ? rowidx[lo + i] : 0x7fffffff;
      val[i] = i < len ? perm[lo + i] : 0;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int h = k >> 1; h > 0; h >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int l = i ^ h;
          if (l > i) {
            const bool up = (i & k) == 0;
            const int a = key[i], b = key[l];
            if ((a > b) == up) {
              key[i] = b;
              key[l] = a;
              const int t = val[i];
              val[i] = val[l];
              val[l] = t;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      rowidx[lo + i] = key[i];
      perm[lo + i] = val[i];
    }
    __syncthreads();
  }
}

// Xt (rows x b, row-major) = X (rows x b, column-major, ld)
__global__ void to_rowmajor(int rows, int b, const double* __restrict__ X, int ld, double* Xt) {
  const size_t total = (size_t)rows * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), c = (int)(e / rows);
    Xt[(size_t)i * b + c] = X[i + (size_t)c * ld];
  }
}

// One warp per output row: P[i, c] = sum_e val(e) Xt[idx(e), c], lanes over c.
template <int CPL, bool PERM>
__global__ void spmm_rows(int rows, int b, const int* __restrict__ ptr, const int* __restrict__ idx,
                          const int* __restrict__ perm, const double* __restrict__ val,
                          const double* __restrict__ Xt, double* P, int ldp) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= rows) return;
  double acc[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) acc[c] = 0.0;
  const int lo = ptr[warp], hi = ptr[warp + 1];
#pragma unroll 4
  for (int e = lo; e < hi; ++e) {  // unrolled: several rows of Xt in flight
    const double v = val[PERM ? perm[e] : e];
    const double* x = Xt + (size_t)idx[e] * b;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int col = lane + 32 * c;
      if (col < b) acc[c] = fma(v, x[col], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int col = lane + 32 * c;
    if (col < b) P[warp + (size_t)col * ldp] = acc[c];
  }
}

template <bool PERM>
blws_status spmm(Ctx* ctx, cudaStream_t s, int rows, int b, const int* ptr, const int* idx,
                 const int* perm, const double* val, const double* Xt, double* P, int ldp) {
  const int blocks = ceil_div((long long)rows * 32, 256);
  if (b <= 32) spmm_rows<1, PERM><<<blocks, 256, 0, s>>>(rows, b, ptr, idx, perm, val, Xt, P, ldp);
  else if (b <= 64) spmm_rows<2, PERM><<<blocks, 256, 0, s>>>(rows, b, ptr, idx, perm, val, Xt, P, ldp);
  else if (b <= 128) spmm_rows<4, PERM><<<blocks, 256, 0, s>>>(rows, b, ptr, idx, perm, val, Xt, P, ldp);
  else if (b <= 256) spmm_rows<8, PERM><<<blocks, 256, 0, s>>>(rows, b, ptr, idx, perm, val, Xt, P, ldp);
  else if (b <= 512) spmm_rows<16, PERM><<<blocks, 256, 0, s>>>(rows, b, ptr, idx, perm, val, Xt, P, ldp);
  else return ctx->fail(BLWS_EINVAL, "sparse block width %d > 512", b);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

__global__ void scale_rows(int r, int b, const double* __restrict__ sl, double* C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * b; e += gridDim.x * blockDim.x)
    C[e] *= sl[e % r];
}

// SDDMM on Omega, one warp per row i of the pattern, one lane per observed
// entry (i, j): the row's scaled u = Ut[i, :] th sits in shared memory and
// each lane walks its own row of Vt, so a warp has 32 independent gathers in
// flight and no per-entry reduction:
//   x = sum_t Ut[i, t] th_t Vt[j, t]  (Ut, Vt row-major with stride c),
//   mode 0 (SVT):  r = m - x;  y += delta r;            acc r^2
//   mode 1 (PROX): r = m - x;  y = delta r (next sparse values);  acc r^2
constexpr int kSddWarps = 8;

__global__ void __launch_bounds__(kSddWarps * 32)
sddmm_update(int rows, int c, const int* __restrict__ rowptr, const int* __restrict__ colidx,
             const double* __restrict__ mval, const double* __restrict__ Ut, const double* __restrict__ th,
             const double* __restrict__ Vt, double delta, int mode, double* y, double* part) {
  extern __shared__ double su[];  // [kSddWarps][c]
  __shared__ double red[kSddWarps];
  const int wib = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int warp = blockIdx.x * kSddWarps + wib;
  double* u = su + (size_t)wib * c;
  double acc2 = 0.0;
  if (warp < rows) {
    for (int t = lane; t < c; t += 32) u[t] = Ut[(size_t)warp * c + t] * th[t];
    __syncwarp();
    const int e1 = rowptr[warp + 1];
    for (int e = rowptr[warp] + lane; e < e1; e += 32) {
      const double* v = Vt + (size_t)colidx[e] * c;
      double x0 = 0.0, x1 = 0.0, x2 = 0.0, x3 = 0.0;
      int t = 0;
      for (; t + 3 < c; t += 4) {
        x0 = fma(u[t], v[t], x0);
        x1 = fma(u[t + 1], v[t + 1], x1);
        x2 = fma(u[t + 2], v[t + 2], x2);
        x3 = fma(u[t + 3], v[t + 3], x3);
      }
      for (; t < c; ++t) x0 = fma(u[t], v[t], x0);
      const double r = mval[e] - ((x0 + x1) + (x2 + x3));
      acc2 = fma(r, r, acc2);
      y[e] = mode == 0 ? fma(delta, r, y[e]) : delta * r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  if (lane == 0) red[wib] = acc2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sacc = 0.0;
    for (int w = 0; w < kSddWarps; ++w) sacc += red[w];
    part[blockIdx.x] = sacc;
  }
}

__global__ void sum_parts(int n, const double* __restrict__ part, double* out) {
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

}  // namespace

blws_status build_csc(Ctx* ctx, cudaStream_t s, int m, int n, int nnz, const int* rowptr,
                      const int* colidx, int** colptr, int** rowidx, int** perm) {
  int *cp, *ri, *pm, *cnt;
  BLWS_TRY(ctx->get(BUF_CSC_PTR, (size_t)2 * (n + 1), &cp));
  BLWS_TRY(ctx->get(BUF_CSC_ROW, (size_t)std::max(nnz, 1), &ri));
  BLWS_TRY(ctx->get(BUF_CSC_PERM, (size_t)std::max(nnz, 1), &pm));
  cnt = cp + (n + 1);
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s));
  if (nnz > 0) {
    count_cols<<<std::min(ceil_div(nnz, 256), ctx->sms * 8), 256, 0, s>>>(nnz, colidx, cnt);
    BLWS_CHECK_LAUNCH(ctx);
  }
  // cursor reuses the count array after the scan has read it: scan writes
  // ptr and cursor from cnt in the same thread, chunk by chunk
  scan_ptr<<<1, 1024, 0, s>>>(n, cnt, cp, cnt);
  BLWS_CHECK_LAUNCH(ctx);
  if (nnz > 0) {
    scatter_csc<<<ceil_div(m, 256), 256, 0, s>>>(m, rowptr, colidx, cnt, ri, pm);
    BLWS_CHECK_LAUNCH(ctx);
    sort_segments<<<std::min(n, ctx->sms * 16), 256, 0, s>>>(n, cp, ri, pm);
    BLWS_CHECK_LAUNCH(ctx);
  }
  *colptr = cp;
  *rowidx = ri;
  *perm = pm;
  return BLWS_OK;
}

blws_status apply_sparse(Ctx* ctx, cudaStream_t s, const Operator& op, const double* X, int ldx,
                         int b, double* P, int ldp) {
  const int m = op.m, n = op.n, N = m + n;
  double* Xt = nullptr;
  BLWS_TRY(ctx->get(BUF_P2, (size_t)N * b, &Xt));  // free during the apply
  const int eb = std::min(ceil_div((long long)N * b, 256), ctx->sms * 8);
  to_rowmajor<<<eb, 256, 0, s>>>(N, b, X, ldx, Xt);  // rows 0..m-1: u-part, m..: v-part
  BLWS_CHECK_LAUNCH(ctx);
  // P_u = S X_v ; P_v = S^T X_u
  BLWS_TRY(spmm<false>(ctx, s, m, b, op.rowptr, op.colidx, nullptr, op.val, Xt + (size_t)m * b, P, ldp));
  BLWS_TRY(spmm<true>(ctx, s, n, b, op.colptr, op.rowidx, op.perm, op.val, Xt, P + m, ldp));
  if (op.rl > 0) {
    double* C = nullptr;
    BLWS_TRY(ctx->get(BUF_MC_X, (size_t)2 * op.rl * b, &C));
    double* C2 = C + (size_t)op.rl * b;
    // P_u += Ul diag(sl) (Vl^T X_v) ; P_v += Vl diag(sl) (Ul^T X_u)
    BLWS_TRY(gemm(ctx, s, true, false, op.rl, b, n, 1.0, op.Vl, n, X + m, ldx, 0.0, C, op.rl));
    BLWS_TRY(gemm(ctx, s, true, false, op.rl, b, m, 1.0, op.Ul, m, X, ldx, 0.0, C2, op.rl));
    scale_rows<<<ceil_div((long long)2 * op.rl * b, 256), 256, 0, s>>>(op.rl, 2 * b, op.sl, C);
    BLWS_CHECK_LAUNCH(ctx);
    BLWS_TRY(gemm(ctx, s, false, false, m, b, op.rl, 1.0, op.Ul, m, C, op.rl, 1.0, P, ldp));
    BLWS_TRY(gemm(ctx, s, false, false, n, b, op.rl, 1.0, op.Vl, n, C2, op.rl, 1.0, P + m, ldp));
  }
  return BLWS_OK;
}

blws_status sddmm(Ctx* ctx, cudaStream_t s, int m, int n, int c, const int* rowptr,
                  const int* colidx, const double* mval, const double* U, int ldu,
                  const double* th, const double* V, int ldv, double delta, int mode, double* y,
                  double* sumsq_out, double* Ut, double* Vt) {
  if (c > 0) {
    to_rowmajor<<<std::min(ceil_div((long long)m * c, 256), ctx->sms * 8), 256, 0, s>>>(m, c, U, ldu, Ut);
    BLWS_CHECK_LAUNCH(ctx);
    to_rowmajor<<<std::min(ceil_div((long long)n * c, 256), ctx->sms * 8), 256, 0, s>>>(n, c, V, ldv, Vt);
    BLWS_CHECK_LAUNCH(ctx);
  }
  double* part = nullptr;
  const int blocks = ceil_div((long long)m, kSddWarps);
  BLWS_TRY(ctx->get(BUF_RED, (size_t)std::max(blocks, ctx->sms * 8), &part));
  if (c > 512) return ctx->fail(BLWS_EINVAL, "rank %d > 512", c);
  const int ssm = kSddWarps * std::max(c, 1) * (int)sizeof(double);
  sddmm_update<<<blocks, kSddWarps * 32, ssm, s>>>(m, c, rowptr, colidx, mval, Ut, th, Vt, delta, mode, y, part);
  BLWS_CHECK_LAUNCH(ctx);
  sum_parts<<<1, 256, 0, s>>>(blocks, part, sumsq_out);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

}  // namespace blws
