// FP32 first stage of the eigen-decomposition of T_k (Algorithm 3, "EVD of
// T_k") by the tridiagonal route (Golub & Van Loan, Sections 8.3-8.4):
//   1. Householder tridiagonalisation Q^T T Q = tridiag(d, e): one CTA, the
//      lower triangle of T packed in shared memory (FP32), one reflector per
//      column; each step's symmetric rank-2 update is applied in the same
//      pass over the trailing triangle as the next step's matrix-vector
//      product;
//   2. every eigenvalue of the tridiagonal matrix by multisection on Sturm
//      counts (one warp per eigenvalue, 32 probes per step);
//   3. eigenvectors by inverse iteration (Wilkinson), each eigenvalue its own
//      shift, from a hashed random start, two solves (one warp per
//      eigenvalue, the substitutions in FP64 so that a chain of small
//      pivots cannot overflow).  Eigenvalues closer than kGroupTol ||T|| form
//      a group whose vectors are orthonormalised together by CholeskyQR2
//      after each solve, so a tight cluster still comes out as an
//      orthonormal basis of its joint eigenspace;
//   4. back-transformation Z = Q Y with the reflectors gathered eight at a
//      time in compact WY form (Schreiber & Van Loan), written out in FP64.
// The result has FP32 accuracy (residual and orthogonality ~1e-6) and is the
// starting point of the FP64 Ogita-Aishima refinement in eig.cu.  Every
// reduction has a fixed order: the stage is deterministic.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

#include "ops.cuh"

namespace cg = cooperative_groups;

namespace blws {

namespace {

constexpr int kTriThreads = 1024;
// threads per CTA of the group orthonormalisation: in the 2000 x 2000 solve,
// 1024: 120.3 ms, 512: 122.0, 384: 121.6, 256: 125.6 per solve
#ifndef BLWS_TRI_QR_THREADS
#define BLWS_TRI_QR_THREADS 1024
#endif
constexpr int kQrThreads = BLWS_TRI_QR_THREADS;
constexpr float kGroupTol = kTriGroupTol;
constexpr float kInvPert = 1.2e-7f;  // inverse iteration: pivots kept >= this x ||T||
constexpr int kQrSmemFloats = 56 * 1024;  // group kernel: shared-memory budget (floats)
constexpr int kQrMaxGroup = 192;          // group kernel: widest group (2 c^2 <= the budget)
constexpr int kQrTileThreads = 64;        // group kernel: Gram tiles from which a thread takes a tile
constexpr float kPivMin = 1e-30f;    // Sturm counts: pivots kept away from zero by this (T scaled to <= 1)

// packed lower triangle, column-major: element (i, j), i >= j
__device__ __forceinline__ int pk(int n, int i, int j) { return j * n - (j * (j - 1)) / 2 + (i - j); }

// sum over the CTA, returned to every thread (fixed order: each warp reduces
// the per-warp partials with the same shuffle tree)
__device__ float block_sum(float v, float* red) {
  __syncthreads();  // red may still be read from the previous call
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31;
  if (lane == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// ------------------------------------------------- 1. tridiagonalisation --
// T (n x n FP64, ld n, symmetric; its lower triangle is read) is scaled by a
// power of two to max |T_ij| in [0.5, 1).  Reflector k, H_k = I - tau_k v v^T
// with v_{k+1} = 1, is stored in V(:, k) (zeros above row k + 1).
//
// Step k: (1) column k receives the rank-2 update left pending by step k-1
// (one warp), which gives alpha, sigma and the diagonal; (2) the reflector;
// (3) one pass over the trailing triangle (rows and columns > k) applies the
// pending update to every element and forms p = A22 v in the same loads, in
// items of 32 columns x 64 rows (one warp each): lane i holds two rows; for
// each column it adds A(r, c) v_c to its rows' sums (the part left of the
// diagonal) and A(r, c) v_r to a per-column sum (the part on and below it),
// which a 31-shuffle reduce-scatter hands to lane c.  Lanes read consecutive
// rows of one column: no bank conflicts.  The partial sums go to a small
// global scratch (L1-resident) and are added per row in a fixed order;
// (4) K = tau p^T v / 2 and w = p - K v become the next pending update.
constexpr int kItemCols = 32, kItemRows = 64;
constexpr int kMaxGroups = (kTriOneCtaMaxN + kItemCols - 1) / kItemCols;
constexpr int kMaxChunks = (kTriOneCtaMaxN + kItemRows - 1) / kItemRows;

__global__ void __launch_bounds__(kTriThreads)
tri_reduce_kernel(int n, const double* __restrict__ T, float* __restrict__ V, float* __restrict__ dv,
                  float* __restrict__ ev, float* __restrict__ tauv, float* __restrict__ part,
                  float* __restrict__ tscale) {
  extern __shared__ float sm[];
  __shared__ float red[32];
  __shared__ double redd[32];
  __shared__ float col[3];  // alpha, sigma and the diagonal entry of the current column
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int np = n * (n + 1) / 2;
  float* A = sm;  // packed lower triangle
  // per row (global index): x, y the pending update A -= pv pw^T + pw pv^T,
  // z this step's reflector: one 16-byte load per column in the items
  float4* cv = reinterpret_cast<float4*>(A + np + ((4 - (np & 3)) & 3));
  float* Lp = part;                     // [group][row]: sums left of the diagonal
  float* Up = part + kMaxGroups * n;    // [chunk][column]: sums on and below the diagonal
  // scale: largest |T_ij| over the lower triangle (a warp per column)
  double mx = 0.0;
  for (int j = wid; j < n; j += nw) {
#pragma unroll 4
    for (int i = j + lane; i < n; i += 32) mx = fmax(mx, fabs(T[i + (size_t)j * n]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) redd[wid] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < nw; ++w) mx = fmax(mx, redd[w]);
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  const double scale = ldexp(1.0, -ex);
  if (tid == 0) *tscale = (float)ldexp(1.0, ex);  // T = 2^ex x the scaled matrix
  for (int j = wid; j < n; j += nw) {
    const int base = pk(n, j, j) - j;
#pragma unroll 4
    for (int i = j + lane; i < n; i += 32) A[base + i] = (float)(T[i + (size_t)j * n] * scale);
  }
  for (int t = tid; t < n; t += nt) cv[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // trailing rows k+1 .. n-1 (local 0 .. m-1)
    // (1) column k
    if (wid == 0) {
      const int base = pk(n, k, k) - k;  // + r: A(r, k), r >= k
      const float pvk = cv[k].x, pwk = cv[k].y;
      float ssq = 0.0f;
      for (int r = k + lane; r < n; r += 32) {
        const float4 q = cv[r];
        const float a = A[base + r] - fmaf(q.x, pwk, q.y * pvk);
        A[base + r] = a;
        if (r >= k + 2) ssq = fmaf(a, a, ssq);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
      __syncwarp();
      if (lane == 0) {
        col[0] = A[base + k + 1];
        col[1] = ssq;
        col[2] = A[base + k];
      }
    }
    __syncthreads();
    // (2) reflector: H x = beta e_1 (same scalars in every thread)
    const float alpha = col[0], sigma = col[1];
    float tau = 0.0f, beta = alpha, vscale = 0.0f;
    if (sigma > 0.0f) {
      const float nrm = sqrtf(fmaf(alpha, alpha, sigma));
      beta = alpha >= 0.0f ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      vscale = 1.0f / (alpha - beta);
    }
    if (tid == 0) {
      dv[k] = col[2];
      ev[k] = beta;
      tauv[k] = tau;
    }
    const int c0 = pk(n, k + 1, k);  // A(k+1, k)
    for (int t = tid; t < n; t += nt) {
      float v = 0.0f;
      if (t == k + 1) v = 1.0f;
      else if (t > k + 1 && tau != 0.0f) v = A[c0 + (t - k - 1)] * vscale;
      V[t + (size_t)k * n] = v;
      cv[t].z = v;
    }
    __syncthreads();
    // (3) pending update and product, one pass
    const int G = (m + kItemCols - 1) / kItemCols, H = (m + kItemRows - 1) / kItemRows;
    for (int it = wid; it < G * H; it += nw) {
      const int g = it % G, h = it / G;
      const int cb = g * kItemCols, rb = h * kItemRows;
      if (rb + kItemRows - 1 < cb) continue;  // above the diagonal
      const int r0 = rb + lane, r1 = r0 + 32;
      const float4 q0 = r0 < m ? cv[k + 1 + r0] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float4 q1 = r1 < m ? cv[k + 1 + r1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float pv0 = q0.x, pw0 = q0.y, v0 = q0.z, pv1 = q1.x, pw1 = q1.y, v1 = q1.z;
      float l0 = 0.0f, l1 = 0.0f, acc[32];
      int base = pk(n, k + 1 + cb, k + 1 + cb) - cb;  // + r: A(k+1+r, k+1+c)
      if (rb >= cb + kItemCols && rb + kItemRows <= m && cb + kItemCols <= m) {
        // every element present and left of the diagonal
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int C = k + 1 + cb + j;
          const float4 q = cv[C];
          const float pvc = q.x, pwc = q.y, vc = q.z;
          const float a0 = fmaf(-pw0, pvc, fmaf(-pv0, pwc, A[base + r0]));
          const float a1 = fmaf(-pw1, pvc, fmaf(-pv1, pwc, A[base + r1]));
          A[base + r0] = a0;
          A[base + r1] = a1;
          l0 = fmaf(a0, vc, l0);
          l1 = fmaf(a1, vc, l1);
          acc[j] = fmaf(a0, v0, a1 * v1);
          base += n - C - 1;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = cb + j, C = k + 1 + c;
          float a0 = 0.0f, a1 = 0.0f, vc = 0.0f;
          if (c < m) {
            const float4 q = cv[C];
            const float pvc = q.x, pwc = q.y;
            vc = q.z;
            if (r0 >= c && r0 < m) {
              a0 = fmaf(-pw0, pvc, fmaf(-pv0, pwc, A[base + r0]));
              A[base + r0] = a0;
            }
            if (r1 >= c && r1 < m) {
              a1 = fmaf(-pw1, pvc, fmaf(-pv1, pwc, A[base + r1]));
              A[base + r1] = a1;
            }
          }
          if (r0 > c) l0 = fmaf(a0, vc, l0);
          if (r1 > c) l1 = fmaf(a1, vc, l1);
          acc[j] = fmaf(a0, v0, a1 * v1);
          base += n - C - 1;
        }
      }
      // reduce-scatter over the lanes: lane j ends with the sum of acc[j]
#pragma unroll
      for (int sft = 16; sft >= 1; sft >>= 1) {
        const bool up = (lane & sft) != 0;
#pragma unroll
        for (int q = 0; q < sft; ++q) {
          const float send = up ? acc[q] : acc[q + sft];
          const float keep = up ? acc[q + sft] : acc[q];
          acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
        }
      }
      if (cb + lane < m) Up[h * n + cb + lane] = acc[0];
      if (r0 < m) Lp[g * n + r0] = l0;
      if (r1 < m) Lp[g * n + r1] = l1;
    }
    __syncthreads();
    // (4) p = tau A22 v, K, w: the next pending update
    float p = 0.0f, pvv = 0.0f;
    if (tid < m) {
      const int r = tid, gr = r / kItemCols;
      float lv[kMaxGroups], uv[kMaxChunks];  // independent loads, then a fixed-order sum
#pragma unroll
      for (int g = 0; g < kMaxGroups; ++g) lv[g] = g <= gr ? Lp[g * n + r] : 0.0f;
#pragma unroll
      for (int h = 0; h < kMaxChunks; ++h)
        uv[h] = (h < H && h * kItemRows + kItemRows - 1 >= gr * kItemCols) ? Up[h * n + r] : 0.0f;
      float sl = 0.0f, su = 0.0f;
#pragma unroll
      for (int g = 0; g < kMaxGroups; ++g) sl += lv[g];
#pragma unroll
      for (int h = 0; h < kMaxChunks; ++h) su += uv[h];
      p = tau * (sl + su);
      pvv = p * cv[k + 1 + r].z;
    }
    const float K = 0.5f * tau * block_sum(pvv, red);
    if (tid < m) {
      float4 q = cv[k + 1 + tid];
      q.y = p - K * q.z;
      q.x = q.z;
      cv[k + 1 + tid] = q;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {  // the last 2 x 2 block receives the last pending update
      const int a = n - 2, b = n - 1;
      const float4 qa = cv[a], qb = cv[b];
      const float daa = A[pk(n, a, a)] - 2.0f * qa.x * qa.y;
      const float dba = A[pk(n, b, a)] - fmaf(qb.x, qa.y, qb.y * qa.x);
      const float dbb = A[pk(n, b, b)] - 2.0f * qb.x * qb.y;
      dv[a] = daa;
      ev[a] = dba;
      dv[b] = dbb;
      tauv[a] = 0.0f;
    } else {
      dv[0] = A[0];
    }
  }
}

// ------------------------------------ 1b. tridiagonalisation on a cluster --
// The same reduction spread over a cluster of kCl CTAs, for matrices
// whose packed triangle does not fit one CTA (kTriOneCtaMaxN < n <=
// kTriMaxN).  (For smaller n the single CTA is faster: three cluster barriers
// and the distributed-shared-memory broadcasts per step cost more than the
// divided item work saves.)  Column groups of 32 are owned round-robin
// (group g by CTA g mod kCl); a CTA keeps all rows of its columns, packed,
// in its own shared memory, and a full copy of the per-row vectors (the
// pending update and the reflector).  Step k:
//   (A) the owner of column k applies the pending update to it, forms the
//       reflector and writes it into every CTA's vectors (distributed shared
//       memory); cluster barrier;
//   (B) every CTA runs the fused update-and-product items over its columns:
//       column sums are complete inside the owner, row sums are partial;
//       each CTA writes its row partials and its columns' sums to CTA 0;
//       cluster barrier;
//   (C) CTA 0 adds them up in a fixed order, forms p, K and w and writes the
//       next pending update into every CTA; cluster barrier.
// Two cluster sizes: 4 CTAs up to kTriCl4MaxN (a quarter of the packed
// triangle per CTA fits shared memory), 8 CTAs (the portable maximum) above,
// up to kTriMaxN.
constexpr int kTriCl4MaxN = 576;
template <int kCl>
__host__ __device__ constexpr int cl_groups() { return (kTriMaxN / kItemCols + kCl - 1) / kCl; }  // groups per CTA
constexpr int kClChunks = (kTriMaxN + kItemRows - 1) / kItemRows;

template <int kCl>
__host__ __device__ inline int cl_owner(int j) { return (j / kItemCols) % kCl; }

// words of packed columns the CTA of `rank` holds
template <int kCl>
__host__ __device__ inline int cl_words(int n, int rank) {
  int w = 0;
  for (int j = 0; j < n; ++j)
    if (cl_owner<kCl>(j) == rank) w += n - j;
  return w;
}

template <int kCl>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kTriThreads)
tri_reduce_cluster_kernel(int n, const double* __restrict__ T, float* __restrict__ V, float* __restrict__ dv,
                          float* __restrict__ ev, float* __restrict__ tauv, float* __restrict__ part,
                          float* __restrict__ tscale) {
  constexpr int kClGroups = cl_groups<kCl>();
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ float4 smc[];
  float4* cv = smc;                                        // x, y: pending update; z: reflector
  float* rowpart = reinterpret_cast<float*>(cv + n);      // [kCl][n], filled in CTA 0
  float* ucol = rowpart + (size_t)kCl * n;             // [n], filled in CTA 0
  int* colstart = reinterpret_cast<int*>(ucol + n);       // A(r, j) at A[colstart[j] + r], own j
  float* A = reinterpret_cast<float*>(colstart + n);
  __shared__ float red[32];
  __shared__ double redd[32];
  __shared__ double cmax[kCl];
  __shared__ float s_tau, s_col[3];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  float* Lp = part + (size_t)rank * (kClGroups + kClChunks) * n;  // [local group][row]
  float* Up = Lp + (size_t)kClGroups * n;                         // [chunk][column]
  if (tid == 0) {
    int off = 0;
    for (int j = 0; j < n; ++j) {
      colstart[j] = INT_MIN / 2;
      if (cl_owner<kCl>(j) == rank) {
        colstart[j] = off - j;
        off += n - j;
      }
    }
  }
  // scale: the largest |T_ij| over the whole lower triangle
  double mx = 0.0;
  for (int j = wid; j < n; j += nw) {
    if (cl_owner<kCl>(j) != rank) continue;
#pragma unroll 4
    for (int i = j + lane; i < n; i += 32) mx = fmax(mx, fabs(T[i + (size_t)j * n]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) redd[wid] = mx;
  __syncthreads();
  if (tid == 0) {
    double bm = 0.0;
    for (int w = 0; w < nw; ++w) bm = fmax(bm, redd[w]);
    for (int q = 0; q < kCl; ++q) *cl.map_shared_rank(&cmax[rank], q) = bm;
  }
  cl.sync();
  mx = 0.0;
  for (int q = 0; q < kCl; ++q) mx = fmax(mx, cmax[q]);
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  const double scale = ldexp(1.0, -ex);
  if (rank == 0 && tid == 0) *tscale = (float)ldexp(1.0, ex);
  for (int j = wid; j < n; j += nw) {
    if (cl_owner<kCl>(j) != rank) continue;
    const int base = colstart[j];
#pragma unroll 4
    for (int i = j + lane; i < n; i += 32) A[base + i] = (float)(T[i + (size_t)j * n] * scale);
  }
  for (int t = tid; t < n; t += nt) cv[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  cl.sync();
  const int ngr = (n + kItemCols - 1) / kItemCols, H = (n + kItemRows - 1) / kItemRows;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    // (A) column k at its owner
    if (rank == cl_owner<kCl>(k)) {
      const int base = colstart[k];
      if (wid == 0) {
        const float pvk = cv[k].x, pwk = cv[k].y;
        float ssq = 0.0f;
        for (int r = k + lane; r < n; r += 32) {
          const float4 q = cv[r];
          const float a = A[base + r] - fmaf(q.x, pwk, q.y * pvk);
          A[base + r] = a;
          if (r >= k + 2) ssq = fmaf(a, a, ssq);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
        __syncwarp();
        if (lane == 0) {
          s_col[0] = A[base + k + 1];
          s_col[1] = ssq;
          s_col[2] = A[base + k];
        }
      }
      __syncthreads();
      const float alpha = s_col[0], sigma = s_col[1];
      float tau = 0.0f, beta = alpha, vscale = 0.0f;
      if (sigma > 0.0f) {
        const float nrm = sqrtf(fmaf(alpha, alpha, sigma));
        beta = alpha >= 0.0f ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        vscale = 1.0f / (alpha - beta);
      }
      if (tid == 0) {
        dv[k] = s_col[2];
        ev[k] = beta;
        tauv[k] = tau;
        for (int q = 0; q < kCl; ++q) *cl.map_shared_rank(&s_tau, q) = tau;
      }
      for (int t = tid; t < n; t += nt) {
        float v = 0.0f;
        if (t == k + 1) v = 1.0f;
        else if (t > k + 1 && tau != 0.0f) v = A[base + t] * vscale;
        V[t + (size_t)k * n] = v;
        if (t > k)
          for (int q = 0; q < kCl; ++q) cl.map_shared_rank(cv, q)[t].z = v;
      }
    }
    cl.sync();
    const float tau = s_tau;
    // (B) items over my column groups in the trailing block
    int nit = 0;
    for (int g = rank; g < ngr; g += kCl)
      if (kItemCols * g + kItemCols - 1 >= k + 1) nit += H - max(kItemCols * g, k + 1) / kItemRows;
    for (int it = wid; it < nit; it += nw) {
      int g = rank, rem = it, h = 0;
      for (;; g += kCl) {
        if (kItemCols * g + kItemCols - 1 < k + 1) continue;
        const int h0 = max(kItemCols * g, k + 1) / kItemRows;
        if (rem < H - h0) {
          h = h0 + rem;
          break;
        }
        rem -= H - h0;
      }
      const int cb = kItemCols * g, rb = kItemRows * h, gl = g / kCl;
      const int r0 = rb + lane, r1 = r0 + 32;
      const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float4 q0 = (r0 > k && r0 < n) ? cv[r0] : z4, q1 = (r1 > k && r1 < n) ? cv[r1] : z4;
      float l0 = 0.0f, l1 = 0.0f, acc[32];
      const bool full = cb >= k + 1 && cb + kItemCols <= n && rb >= cb + kItemCols && rb + kItemRows <= n;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = cb + j;
        const bool cin = full || (c > k && c < n);
        const float4 qc = cin ? cv[c] : z4;
        const int base = cin ? colstart[c] : 0;
        const bool in0 = full || (cin && r0 >= c && r0 < n), in1 = full || (cin && r1 >= c && r1 < n);
        float a0 = 0.0f, a1 = 0.0f;
        if (in0) {
          a0 = fmaf(-q0.y, qc.x, fmaf(-q0.x, qc.y, A[base + r0]));
          A[base + r0] = a0;
        }
        if (in1) {
          a1 = fmaf(-q1.y, qc.x, fmaf(-q1.x, qc.y, A[base + r1]));
          A[base + r1] = a1;
        }
        if (r0 > c) l0 = fmaf(a0, qc.z, l0);
        if (r1 > c) l1 = fmaf(a1, qc.z, l1);
        acc[j] = fmaf(a0, q0.z, a1 * q1.z);
      }
#pragma unroll
      for (int sft = 16; sft >= 1; sft >>= 1) {
        const bool up = (lane & sft) != 0;
#pragma unroll
        for (int q = 0; q < sft; ++q) {
          const float send = up ? acc[q] : acc[q + sft];
          const float keep = up ? acc[q + sft] : acc[q];
          acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
        }
      }
      if (cb + lane > k && cb + lane < n) Up[(size_t)h * n + cb + lane] = acc[0];
      if (r0 > k && r0 < n) Lp[(size_t)gl * n + r0] = l0;
      if (r1 > k && r1 < n) Lp[(size_t)gl * n + r1] = l1;
    }
    __syncthreads();
    {
      float* rp0 = cl.map_shared_rank(rowpart, 0);
      float* uc0 = cl.map_shared_rank(ucol, 0);
      for (int r = k + 1 + tid; r < n; r += nt) {
        float sl = 0.0f;
        for (int g = rank; g < ngr && kItemCols * g < r; g += kCl)
          if (kItemCols * g + kItemCols - 1 >= k + 1) sl += Lp[(size_t)(g / kCl) * n + r];
        rp0[(size_t)rank * n + r] = sl;
        if (cl_owner<kCl>(r) == rank) {
          const int g = r / kItemCols;
          float su = 0.0f;
          for (int h = max(kItemCols * g, k + 1) / kItemRows; h < H; ++h) su += Up[(size_t)h * n + r];
          uc0[r] = su;
        }
      }
    }
    cl.sync();
    // (C) CTA 0: p = tau (row sums + column sums), K, w; the next pending update everywhere
    if (rank == 0) {
      float p = 0.0f, pvv = 0.0f, v = 0.0f;
      const int r = k + 1 + tid;
      if (tid < m) {
        float sum = ucol[r];
#pragma unroll
        for (int q = 0; q < kCl; ++q) sum += rowpart[(size_t)q * n + r];
        p = tau * sum;
        v = cv[r].z;
        pvv = p * v;
      }
      const float K = 0.5f * tau * block_sum(pvv, red);
      if (tid < m) {
        const float w = p - K * v;
        for (int q = 0; q < kCl; ++q) {
          float4* rc = cl.map_shared_rank(cv, q);
          rc[r].x = v;
          rc[r].y = w;
        }
      }
    }
    cl.sync();
  }
  if (tid == 0 && n >= 2) {  // the last 2 x 2 block receives the last pending update
    const int a = n - 2, b = n - 1;
    const float4 qa = cv[a], qb = cv[b];
    if (rank == cl_owner<kCl>(a)) {
      dv[a] = A[colstart[a] + a] - 2.0f * qa.x * qa.y;
      ev[a] = A[colstart[a] + b] - fmaf(qb.x, qa.y, qb.y * qa.x);
      tauv[a] = 0.0f;
    }
    if (rank == cl_owner<kCl>(b)) dv[b] = A[colstart[b] + b] - 2.0f * qb.x * qb.y;
  }
}

template <int kCl>
int cl_smem_bytes(int n) {
  int w = 0;
  for (int r = 0; r < kCl; ++r) w = std::max(w, cl_words<kCl>(n, r));
  return n * (int)sizeof(float4) + (kCl + 1) * n * (int)sizeof(float) + n * (int)sizeof(int) +
         w * (int)sizeof(float);
}


// ----------------------------- 1c. tridiagonalisation by rows on a cluster --
// The same Householder reduction with the whole symmetric matrix stored (both
// triangles) and its rows dealt out round-robin: row i lives in CTA i mod kCl
// (kCl = 1, 2, 4 or 8 CTAs of one thread-block cluster) as local row
// i / kCl, and local row l belongs to warp l mod (warps per CTA).  A warp then owns whole
// rows: the trailing update and the product p = A22 v of a row are one pass
// over it with a warp-level sum, and no column sums have to be gathered
// across warps.  Every CTA keeps the per-index vectors (pending update
// pv, pw, the current reflector v, and p) in full.  Step k:
//   (1) the warp owning row k applies the pending update to it, forms the
//       reflector and writes v (and tau) into every CTA; cluster barrier;
//   (2) every warp updates its trailing rows and forms p_i = tau a_i . v,
//       written into every CTA; each CTA's sum of p_i v_i goes to every CTA;
//       cluster barrier;
//   (3) every CTA forms K = tau / 2 sum p_i v_i (the CTA sums in rank order)
//       and the next pending pair (v_j, w_j = p_j - K v_j) of every index
//       itself -- no third barrier; the reflectors of consecutive steps live
//       in two slots, so the next owner can write its own meanwhile.
// Every sum has a fixed order, so the result is deterministic.
constexpr int kRowsMaxN1 = 236, kRowsMaxN2 = 330, kRowsMaxN4 = 468, kRowsMaxN8 = 656;
// threads per CTA of the reduction by rows: measured in the 2000 x 2000 solve
// (4-CTA cluster at n = 303), 1024: 123.1 ms, 768: 120.7, 512: 120.9 per solve
#ifndef BLWS_TRI_ROWS_THREADS
#define BLWS_TRI_ROWS_THREADS 768
#endif
constexpr int kTriRowsThreads = BLWS_TRI_ROWS_THREADS;  // threads per CTA (a multiple of 32, <= 1024)

template <int kCl>
__host__ __device__ constexpr int rows_per_cta(int n) { return (n + kCl - 1) / kCl; }


// Shared memory of the kernel below: the vectors (n float4), p of the local
// rows, and the rows themselves -- sized for the larger of the cluster phase
// (R rows of n) and the single-CTA phase (a trailing block of at most
// kRowsSwitchM squared).  The cluster phase runs while the trailing block is
// wider than kRowsSwitchM, on at least BLWS_TRI_MIN_CL CTAs.  Measured in the
// 2000 x 2000 rank-100 FP64-equivalent solve (T_k of 303): 96 and 4 CTAs took
// 135.8-136.0 ms per solve, 232 on the 2 CTAs whose shares fit 139.9 ms, the
// other pairs tried (32-160, 2-8 CTAs) in between.
#ifndef BLWS_TRI_SWITCH_M
#define BLWS_TRI_SWITCH_M 96
#endif
constexpr int kRowsSwitchM = BLWS_TRI_SWITCH_M;
static_assert(kRowsSwitchM >= 2, "the single-CTA phase holds at least the last 2 x 2 block");
#ifndef BLWS_TRI_MIN_CL
#define BLWS_TRI_MIN_CL 4
#endif

// CTAs of the reduction by rows: the smallest cluster whose share of the full
// matrix fits one CTA (0: none), and at least BLWS_TRI_MIN_CL when a cluster
// phase runs at all (n above the switch point)
inline int rows_cluster(int n) {
  int c = 0;
  if (n <= kRowsMaxN1) c = 1;
  else if (n <= kRowsMaxN2) c = 2;
  else if (n <= kRowsMaxN4) c = 4;
  else if (n <= kRowsMaxN8) c = 8;
  if (c && n > kRowsSwitchM) c = std::max(c, BLWS_TRI_MIN_CL);
  return c;
}

// the pending rank-2 term pv_i pw_j + pw_i pv_j of element (i, j), rounded the
// same way for (j, i): both products, then their sum (each operation is
// commutative), so the stored matrix stays exactly symmetric
__device__ __forceinline__ float sym_upd(const float4& qi, const float4& qj) {
  return __fadd_rn(__fmul_rn(qi.x, qj.y), __fmul_rn(qi.y, qj.x));
}

template <int kCl>
__device__ __forceinline__ void rows_sync() {
  if constexpr (kCl > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// the same shared-memory object in CTA r of the cluster
template <int kCl, typename P>
__device__ __forceinline__ P* rows_remote(P* p, int r) {
  if constexpr (kCl > 1) {
    return cg::this_cluster().map_shared_rank(p, r);
  } else {
    return p;
  }
}

template <int kCl>
int rows_smem_bytes(int n) {
  const int R = rows_per_cta<kCl>(n);
  const int S = kCl > 1 ? std::min(n, kRowsSwitchM) : 0;
  return n * (int)sizeof(float4) + n * (int)sizeof(float) + std::max(R * n, S * S) * (int)sizeof(float);
}

// One Householder step k over the rows this CTA holds, KC CTAs taking part.
// Local row l is global row i = base + l KC + rank, stored at A + l ldA, and
// element (i, j) of it at (A + l ldA)[j - base] (only j >= k + 1 > base is
// touched).  sh_part has KC entries, pv (p of every index) n.  The step's
// reflector goes to cv[.].z on even steps and cv[.].w on odd ones, so the
// next step's owner can write its reflector while the others still read this
// one; two cluster barriers per step: after the reflector, after p.
template <int KC>
__device__ __forceinline__ void rows_step(int k, int n, int rank, int R, int base, float* A, int ldA,
                                          float4* cv, float* pv, float* red, float* sh_part, float* sh_tau,
                                          float* __restrict__ V, float* __restrict__ dv, float* __restrict__ ev,
                                          float* __restrict__ tauv) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const bool odd = (k & 1) != 0;
  // (1) row k: pending update, reflector into every CTA
  const int lk = (k - base) / KC;
  if (rank == (k - base) % KC && wid == lk % nw) {
    float* row = A + (size_t)lk * ldA - base;
    const float4 qk = cv[k];
    float ssq = 0.0f;
    for (int j = k + lane; j < n; j += 32) {
      const float4 q = cv[j];
      const float a = row[j] - sym_upd(qk, q);
      row[j] = a;
      if (j >= k + 2) ssq = fmaf(a, a, ssq);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
    __syncwarp();
    const float alpha = row[k + 1];
    float tau = 0.0f, beta = alpha, vscale = 0.0f;
    if (ssq > 0.0f) {
      // the serial part of the step: a correctly rounded reciprocal and one
      // fast quotient (2 ulp) keep it short; the FP32 stage is refined in
      // FP64 afterwards
      const float nrm = sqrtf(fmaf(alpha, alpha, ssq));
      beta = alpha >= 0.0f ? -nrm : nrm;
      tau = __fdividef(beta - alpha, beta);
      vscale = __frcp_rn(alpha - beta);
    }
    if (lane == 0) {
      dv[k] = row[k];
      ev[k] = beta;
      tauv[k] = tau;
#pragma unroll
      for (int r = 0; r < KC; ++r) *rows_remote<KC>(sh_tau, r) = tau;
    }
    for (int j = k + 1 + lane; j < n; j += 32) {
      const float v = j == k + 1 ? 1.0f : (tau != 0.0f ? row[j] * vscale : 0.0f);
#pragma unroll
      for (int r = 0; r < KC; ++r) {
        float4* rc = rows_remote<KC>(cv, r);
        if (odd) rc[j].w = v;
        else rc[j].z = v;
      }
    }
  }
  rows_sync<KC>();
  // (2) trailing rows: pending update and p_i = tau a_i . v, two rows per pass;
  // p_i into every CTA
  const float tau = *sh_tau;
  const int l0 = (k - base + KC - rank) / KC;  // first local row with a global index > k
  float pvw = 0.0f;                            // this warp's sum of p_i v_i
  for (int l = l0 + ((wid - l0 % nw) + nw) % nw; l < R; l += 2 * nw) {
    const int i0 = base + l * KC + rank, i1 = base + (l + nw) * KC + rank;
    if (i0 >= n) break;
    const bool two = l + nw < R && i1 < n;
    float* r0 = A + (size_t)l * ldA - base;
    float* r1 = A + (size_t)(l + nw) * ldA - base;
    const float4 q0 = cv[i0];
    const float4 q1 = two ? cv[i1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float s0 = 0.0f, s1 = 0.0f;
    if (two) {
#pragma unroll 2
      for (int j = k + 1 + lane; j < n; j += 32) {
        const float4 q = cv[j];
        const float vj = odd ? q.w : q.z;
        const float a0 = r0[j] - sym_upd(q0, q);
        const float a1 = r1[j] - sym_upd(q1, q);
        r0[j] = a0;
        r1[j] = a1;
        s0 = fmaf(a0, vj, s0);
        s1 = fmaf(a1, vj, s1);
      }
    } else {
#pragma unroll 2
      for (int j = k + 1 + lane; j < n; j += 32) {
        const float4 q = cv[j];
        const float a0 = r0[j] - sym_upd(q0, q);
        r0[j] = a0;
        s0 = fmaf(a0, odd ? q.w : q.z, s0);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const float p0 = tau * s0, p1 = tau * s1;
    if (lane < KC) {
      float* rp = rows_remote<KC>(pv, lane);
      rp[i0] = p0;
      if (two) rp[i1] = p1;
    }
    pvw = fmaf(p0, odd ? q0.w : q0.z, pvw);
    if (two) pvw = fmaf(p1, odd ? q1.w : q1.z, pvw);
  }
  if (lane == 0) red[wid] = pvw;
  __syncthreads();
  if (wid == 0) {
    float t = lane < nw ? red[lane] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane < KC) rows_remote<KC>(sh_part, lane)[rank] = t;
  }
  rows_sync<KC>();
  // (3) in every CTA, for every index: K and the next pending pair
  // (v_j, w_j = p_j - K v_j) -- only the pair's two words are written, as
  // the next step's owner may already be writing its reflector into the
  // other slot
  float K = 0.0f;
#pragma unroll
  for (int r = 0; r < KC; ++r) K += sh_part[r];
  K *= 0.5f * tau;
  for (int j = k + 1 + tid; j < n; j += blockDim.x) {
    const float v = odd ? cv[j].w : cv[j].z;
    *reinterpret_cast<float2*>(&cv[j]) = make_float2(v, pv[j] - K * v);
  }
  // reflector k out to global memory, off the serial step: CTA r writes the
  // indices i = r (mod KC) (zero above k + 1, v_{k+1} = 1)
  for (int i = rank + KC * tid; i < n; i += KC * (int)blockDim.x)
    V[i + (size_t)k * n] = i > k ? (odd ? cv[i].w : cv[i].z) : 0.0f;
  __syncthreads();  // the pairs are read by every warp of this CTA next
}

// The reduction by rows.  kCl > 1: the cluster phase runs while the trailing
// block is larger than kRowsSwitchM; then every CTA writes its trailing rows to
// `stage` (global, at least kRowsSwitchM^2 floats), CTA 0 gathers the block
// (rows and columns ks .. n-1) into its own shared memory and finishes alone,
// with block barriers instead of cluster barriers, and the other CTAs leave.
template <int kCl>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kTriRowsThreads)
tri_rows_kernel(int n, const double* __restrict__ T, float* __restrict__ V, float* __restrict__ dv,
                float* __restrict__ ev, float* __restrict__ tauv, float* __restrict__ tscale,
                float* __restrict__ stage) {
  extern __shared__ float4 smr[];
  __shared__ float red[32];
  __shared__ double redd[32];
  __shared__ float sh_part[kCl];  // every CTA's sum of p_i v_i (written by that CTA)
  __shared__ float sh_tau;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  int rank = 0;
  if constexpr (kCl > 1) rank = (int)cg::this_cluster().block_rank();
  const int R = rows_per_cta<kCl>(n);
  const int S = kCl > 1 ? min(n, kRowsSwitchM) : 0;
  float4* cv = smr;                                   // x, y: pending update; z / w: reflector
  float* pv = reinterpret_cast<float*>(cv + n);       // p_i of every index
  float* A = pv + n;                                  // the rows
  // scale: largest |T_ij| over the lower triangle (every CTA finds the same)
  double mx = 0.0;
  for (int j = wid; j < n; j += nw) {
#pragma unroll 4
    for (int i = j + lane; i < n; i += 32) mx = fmax(mx, fabs(T[i + (size_t)j * n]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) redd[wid] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < nw; ++w) mx = fmax(mx, redd[w]);
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  const double scale = ldexp(1.0, -ex);
  if (tid == 0 && rank == 0) *tscale = (float)ldexp(1.0, ex);  // T = 2^ex x the scaled matrix
  // own rows, both triangles from the lower one: (i, j) = T[max + min n]
  for (int l = wid; l < R; l += nw) {
    const int i = l * kCl + rank;
    if (i >= n) break;
    float* row = A + (size_t)l * n;
    for (int j = lane; j < n; j += 32)
      row[j] = (float)((j >= i ? T[j + (size_t)i * n] : T[i + (size_t)j * n]) * scale);
  }
  for (int t = tid; t < n; t += blockDim.x) cv[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  rows_sync<kCl>();  // every CTA running and initialised before any remote write
  const int ks = kCl > 1 ? n - S : n;  // first step of the single-CTA phase
  int k = 0;
  for (; k + 2 < n && k < ks; ++k)
    rows_step<kCl>(k, n, rank, R, 0, A, n, cv, pv, red, sh_part, &sh_tau, V, dv, ev, tauv);
  int fbase = 0, fld = n;  // layout of the rows for the last 2 x 2 block
  if constexpr (kCl > 1) {
    // gather the trailing block (m0 = n - ks rows and columns) into CTA 0
    const int m0 = n - ks;
    for (int l = wid; l < R; l += nw) {
      const int i = l * kCl + rank;
      if (i >= n) break;
      if (i < ks) continue;
      const float* row = A + (size_t)l * n;
      for (int j = ks + lane; j < n; j += 32) stage[(size_t)(i - ks) * m0 + (j - ks)] = row[j];
    }
    __threadfence();
    rows_sync<kCl>();
    if (rank != 0) return;  // no remote access follows
    __threadfence();
    for (int e = tid; e < m0 * m0; e += blockDim.x) A[e] = stage[e];
    __syncthreads();
    for (; k + 2 < n; ++k) rows_step<1>(k, n, 0, m0, ks, A, m0, cv, pv, red, sh_part, &sh_tau, V, dv, ev, tauv);
    fbase = ks;
    fld = m0;
  }
  // the last 2 x 2 block receives the last pending update (one CTA holds it:
  // CTA 0 after the gather, or the only one)
  if (tid == 0) {
    if (n >= 2) {
      const int a = n - 2, b = n - 1;
      const float4 qa = cv[a], qb = cv[b];
      const float* ra = A + (size_t)(a - fbase) * fld - fbase;
      const float* rb = A + (size_t)(b - fbase) * fld - fbase;
      dv[a] = ra[a] - sym_upd(qa, qa);
      ev[a] = ra[b] - sym_upd(qa, qb);
      tauv[a] = 0.0f;
      dv[b] = rb[b] - sym_upd(qb, qb);
    } else {
      dv[0] = A[0];
    }
  }
}

// ------------------------------------------------------ 2. eigenvalues --
// lam[j] = the (j+1)-th smallest eigenvalue of tridiag(d, e), one warp each.
__device__ __forceinline__ int sturm_count(int n, const float* sd, const float* se2, float x) {
  float q = sd[0] - x;
  if (fabsf(q) <= kPivMin) q = -kPivMin;
  int c = q < 0.0f;
  for (int i = 1; i < n; ++i) {
    q = (sd[i] - x) - __fdividef(se2[i - 1], q);
    if (fabsf(q) <= kPivMin) q = -kPivMin;
    c += q < 0.0f;
  }
  return c;
}

__global__ void __launch_bounds__(256)
tri_bisect_kernel(int n, const float* __restrict__ dv, const float* __restrict__ ev, float* __restrict__ lam) {
  __shared__ float sd[kTriMaxN], se2[kTriMaxN];
  __shared__ float rlo[8], rhi[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float lo = 3.0e38f, hi = -3.0e38f;
  for (int i = tid; i < n; i += blockDim.x) {
    const float d = dv[i];
    const float el = i > 0 ? fabsf(ev[i - 1]) : 0.0f, er = i + 1 < n ? fabsf(ev[i]) : 0.0f;
    sd[i] = d;
    if (i + 1 < n) se2[i] = ev[i] * ev[i];
    lo = fminf(lo, d - el - er);
    hi = fmaxf(hi, d + el + er);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) {
    rlo[wid] = lo;
    rhi[wid] = hi;
  }
  __syncthreads();
  lo = rlo[0];
  hi = rhi[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    lo = fminf(lo, rlo[w]);
    hi = fmaxf(hi, rhi[w]);
  }
  const float tn = fmaxf(fabsf(lo), fabsf(hi));
  const float tol = 2.4e-7f * tn + kPivMin;
  lo -= 1e-6f * tn + kPivMin;  // count(lo) = 0 and count(hi) = n
  hi += 1e-6f * tn + kPivMin;
  const int j = blockIdx.x * (blockDim.x >> 5) + wid;
  if (j >= n) return;
  for (int it = 0; it < 12 && hi - lo > tol; ++it) {
    const float x = lo + (hi - lo) * (float)(lane + 1) * (1.0f / 33.0f);
    const unsigned below = __ballot_sync(0xffffffffu, sturm_count(n, sd, se2, x) <= j);
    const int f = __ffs(~below) - 1;  // first probe with more than j eigenvalues below it (-1: none)
    const float xl = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 31);
    const float xh = __shfl_sync(0xffffffffu, x, f >= 0 ? f : 31);
    if (f != 0) lo = xl;           // lanes before f all have count <= j
    if (f >= 0) hi = xh;
  }
  if (lane == 0) lam[j] = 0.5f * (lo + hi);
}

// ----------------------------------------------- 3. inverse iteration --
__device__ __forceinline__ float hash_uniform(uint32_t col, uint32_t row) {
  // integer hash (xorshift-multiply finaliser) of (col, row) to [-1, 1)
  uint32_t x = col * 0x9E3779B1u ^ (row + 0x632BE5ABu) * 0x85EBCA77u;
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return (float)(x >> 8) * (1.0f / 8388608.0f) - 1.0f;
}

// One warp per eigenvalue g.  First call: the group of g (grp[g]: its first
// column for groups of two or more, else -1; gtop[g]: the group's largest
// eigenvalue from the multisection, in T's units), the LU factorisation with
// partial pivoting of tridiag(d, e) - lam_g I (F, kept for the second call)
// and a hashed random start; second call: F and the start from Y.  Lane 0
// runs the substitutions from shared memory.  A chain of small pivots can
// grow the solution past the FP32 range: whenever an entry exceeds 2^100 the
// running values are scaled by 2^-100 and the row is recorded, and the
// entries computed before it are scaled down with the normalisation.  Y(r, g)
// at r * n + g receives the normalised solution; a solution that cannot be
// normalised (too many rescalings, a non-finite entry, zero) sets *fail.
constexpr int kMaxRescale = 8;
constexpr float kRescaleAt = 1.2676506e30f;  // 2^100
constexpr float kRescaleBy = 7.888609e-31f;  // 2^-100

template <bool kFirst>
__global__ void __launch_bounds__(32)
tri_solve_kernel(int n, const float* __restrict__ dv, const float* __restrict__ ev,
                 const float* __restrict__ lam, const float* __restrict__ tscale, float4* __restrict__ F,
                 float* __restrict__ Y, int* __restrict__ grp, float* __restrict__ gtop, int* fail) {
  extern __shared__ float4 smf[];
  float4* sF = smf;                                // n
  float* sy = reinterpret_cast<float*>(sF + n);    // right-hand side, then solution (n)
  float* sb = sy + n;                              // after the forward elimination (n)
  float* sd = sb + n;                              // d, e (first call)
  float* se = sd + n;
  __shared__ int nres, rrow[kMaxRescale];
  const int g = blockIdx.x, lane = threadIdx.x;
  const float tn = fmaxf(fabsf(lam[0]), fabsf(lam[n - 1]));
  const float pmin = fmaxf(kInvPert * tn, kPivMin);
  if (kFirst) {
#pragma unroll 4
    for (int r = lane; r < n; r += 32) {
      sd[r] = dv[r];
      se[r] = r + 1 < n ? ev[r] : 0.0f;
      sy[r] = hash_uniform((uint32_t)g, (uint32_t)r);
    }
    __syncwarp();
    if (lane == 0) {
      const float gtol = kGroupTol * tn;
      int i = g, j = g + 1;
      while (i > 0 && lam[i] - lam[i - 1] < gtol) --i;
      while (j < n && lam[j] - lam[j - 1] < gtol) ++j;
      grp[g] = j - i >= 2 ? i : -1;
      gtop[g] = lam[j - 1] * *tscale;  // largest eigenvalue of the group (FP32 estimate, T's units)
      const float x = lam[g];
      float al = sd[0] - x, be = se[0];  // pending row k: (k, k) and (k, k+1)
      for (int k = 0; k + 1 < n; ++k) {
        const float ck = se[k], ak1 = sd[k + 1] - x, bk1 = se[k + 1];
        float u1, u2, u3, lk;
        uint32_t sw;
        if (fabsf(al) >= fabsf(ck)) {  // keep row k
          u1 = al; u2 = be; u3 = 0.0f; sw = 0u;
          if (fabsf(u1) < pmin) u1 = u1 < 0.0f ? -pmin : pmin;
          const float ru = __frcp_rn(u1);
          lk = ck * ru;
          al = fmaf(-lk, be, ak1);
          be = bk1;
          u1 = ru;
        } else {                       // interchange rows k and k+1
          u2 = ak1; u3 = bk1; sw = 1u;
          const float rc = __frcp_rn(ck);
          lk = al * rc;
          al = fmaf(-lk, ak1, be);
          be = -lk * bk1;
          u1 = fabsf(ck) < pmin ? __frcp_rn(ck < 0.0f ? -pmin : pmin) : rc;
        }
        // stored: 1/U(k,k), U(k,k+1), U(k,k+2), multiplier whose last mantissa
        // bit carries the interchange (a one-ulp change, immaterial here)
        sF[k] = make_float4(u1, u2, u3, __uint_as_float((__float_as_uint(lk) & ~1u) | sw));
      }
      if (fabsf(al) < pmin) al = al < 0.0f ? -pmin : pmin;
      sF[n - 1] = make_float4(__frcp_rn(al), 0.0f, 0.0f, 0.0f);
    }
    __syncwarp();
    for (int k = lane; k < n; k += 32) F[(size_t)k * n + g] = sF[k];
  } else {
    if (*fail) return;
#pragma unroll 4
    for (int k = lane; k < n; k += 32) {
      sF[k] = F[(size_t)k * n + g];
      sy[k] = Y[(size_t)k * n + g];
    }
    __syncwarp();
  }
  if (lane == 0) {
    float yk = sy[0];
    for (int k = 0; k + 1 < n; ++k) {  // L^{-1} P y
      const float4 f = sF[k];
      float yk1 = sy[k + 1];
      if (__float_as_uint(f.w) & 1u) {
        const float t = yk;
        yk = yk1;
        yk1 = t;
      }
      yk1 = fmaf(-f.w, yk, yk1);
      sb[k] = yk;
      yk = yk1;
    }
    int nr = 0;
    float x1 = yk * sF[n - 1].x, x2 = 0.0f;  // U x = y
    if (fabsf(x1) > kRescaleAt) {
      x1 *= kRescaleBy;  // nothing computed before it
    }
    sy[n - 1] = x1;
    for (int k = n - 2; k >= 0; --k) {
      const float4 f = sF[k];
      float xk = fmaf(-f.z, x2, fmaf(-f.y, x1, sb[k])) * f.x;
      if (fabsf(xk) > kRescaleAt) {
        xk *= kRescaleBy;
        x1 *= kRescaleBy;
        x2 *= kRescaleBy;
        if (nr < kMaxRescale) rrow[nr] = k;
        ++nr;
      }
      sy[k] = xk;
      x2 = x1;
      x1 = xk;
    }
    nres = nr;
  }
  __syncwarp();
  const int nr = nres;
  // entries above a rescaled row were computed before it: scale them down
  float mx = 0.0f;
  for (int r = lane; r < n; r += 32) {
    float v = sy[r];
    for (int e = 0; e < min(nr, kMaxRescale); ++e)
      if (r > rrow[e]) v *= kRescaleBy;
    sy[r] = v;
    mx = fmaxf(mx, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncwarp();
  const bool ok = nr <= kMaxRescale && mx > 0.0f && mx <= 3.0e38f;
  const float rm = ok ? 1.0f / mx : 0.0f;
  float ss = 0.0f;
  for (int r = lane; r < n; r += 32) {
    const float v = sy[r] * rm;
    ss = fmaf(v, v, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const float inv = ok ? rm * rsqrtf(ss) : 0.0f;
  if (!ok && lane == 0) *fail = 1;
  for (int r = lane; r < n; r += 32) Y[(size_t)r * n + g] = sy[r] * inv;
}

// CholeskyQR2 (FP32) of each group's n x c block of Y, one CTA per group
// (the CTA of the group's first column; the others return at once).  The
// block and its Gram matrix are staged in shared memory (sm_floats), the
// block with an odd leading dimension so that warps reading down a column
// and threads walking a row both hit distinct banks, the Gram matrix with
// rows padded to a multiple of four floats (the solve reads L four at a time).  A group too wide for
// that sets *fail (the matrix then goes to Jacobi).
// The Cholesky factor is built column by column with one barrier per column:
// every thread reads the pivot itself, and column k of L goes to the unused
// upper triangle (L(a, k) at G[k + a c], the diagonal in dg) while the
// trailing update reads the lower one.  When the second pass's Gram matrix is
// within kNearId of the identity, G = I + E, its Cholesky factor is taken as
// I + tril(E) (error O(|E|^2) ~ 1e-7, the FP32 level) without the column
// by column factorisation.
constexpr float kNearId = 3e-4f;

__global__ void __launch_bounds__(kQrThreads)
tri_group_qr_kernel(int n, int sm_floats, const int* __restrict__ grp, float* __restrict__ Y, int* fail) {
  extern __shared__ __align__(16) float smq[];
  __shared__ float dg[kQrMaxGroup];
  __shared__ int near_sh;
  const int i = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (grp[i] != i || *fail) return;
  int j = i + 1;
  while (j < n && grp[j] == i) ++j;
  const int c = j - i;
  const int lds = c | 1;
  const int ldg = (c + 3) & ~3;           // Gram rows 16-byte aligned
  const int goff = (n * lds + 3) & ~3;
  if ((long long)goff + (long long)c * ldg > sm_floats || c > kQrMaxGroup) {
    // too wide to stage: the caller falls back to Jacobi for this matrix
    if (tid == 0) *fail = 1;
    return;
  }
  float* Yb = smq;  // block element (r, a) at Yb[r * lds + a]
  float* G = smq + goff;  // G(a, b) at G[a + b * ldg]
  const int ldb = lds;
  for (int r = wid; r < n; r += nw)
    for (int a = lane; a < c; a += 32) Yb[r * ldb + a] = Y[(size_t)r * n + i + a];
  if (tid == 0) near_sh = 1;
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    // Gram matrix in 4 x 4 tiles (upper triangle of tiles), mirrored.  Few
    // tiles: a warp per tile, lanes over rows, summed by shuffles.  Many: a
    // thread per tile summing over every S-th row (S = 4, 2 or 1, as many
    // row slices as the threads allow), the slices of a tile in adjacent
    // lanes, combined by shuffles
    const int t4 = (c + 3) / 4, ntile = t4 * (t4 + 1) / 2;
    auto put_tile = [&](int ta, int tb, const float(&acc)[4][4]) {
      bool near = true;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int a = 4 * ta + u, b = 4 * tb + q;
          if (a < c && b < c) {
            G[a + b * ldg] = acc[u][q];
            G[b + a * ldg] = acc[u][q];
            near = near && fabsf(acc[u][q] - (a == b ? 1.0f : 0.0f)) <= kNearId;
          }
        }
      if (!near) near_sh = 0;
    };
    auto tile_sum = [&](int ta, int tb, int r0, int step, float(&acc)[4][4]) {
      for (int r = r0; r < n; r += step) {
        const float* yr = Yb + (size_t)r * ldb;
        float ya[4], yb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ya[u] = 4 * ta + u < c ? yr[4 * ta + u] : 0.0f;
          yb[u] = 4 * tb + u < c ? yr[4 * tb + u] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[u][q] = fmaf(ya[u], yb[q], acc[u][q]);
      }
    };
    auto unrank = [&](int e, int& ta, int& tb) {  // e -> (ta, tb), ta <= tb
      int rem = e;
      ta = 0;
      while (rem >= t4 - ta) {
        rem -= t4 - ta;
        ++ta;
      }
      tb = ta + rem;
    };
    if (ntile < kQrTileThreads) {
      for (int e = wid; e < ntile; e += nw) {
        int ta, tb;
        unrank(e, ta, tb);
        float acc[4][4] = {};
        tile_sum(ta, tb, lane, 32, acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[u][q] += __shfl_xor_sync(0xffffffffu, acc[u][q], o);
        if (lane == 0) put_tile(ta, tb, acc);
      }
    } else {
      const int S = ntile * 4 <= nt ? 4 : (ntile * 2 <= nt ? 2 : 1);
      for (int base = 0; base < ntile; base += nt / S) {
        const int e = base + tid / S, sl = tid % S;
        int ta = 0, tb = 0;
        float acc[4][4] = {};
        if (e < ntile) {
          unrank(e, ta, tb);
          tile_sum(ta, tb, sl, S, acc);
        }
        for (int o = 1; o < S; o <<= 1)
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[u][q] += __shfl_xor_sync(0xffffffffu, acc[u][q], o);
        if (e < ntile && sl == 0) put_tile(ta, tb, acc);
      }
    }
    __syncthreads();
    if (pass == 1 && near_sh) {
      // G = I + E with |E| <= kNearId: L = I + tril(E) to within |E|^2 ~ 1e-7
      // (the FP32 level), which is G itself below the diagonal and its mirror
      // above (where the solve reads it), with the square-rooted diagonal
      for (int a = tid; a < c; a += nt) dg[a] = sqrtf(G[a + a * ldg]);
      __syncthreads();
    } else {
      // G = L L^T: column kk of L into the upper triangle and dg, one barrier per column
      for (int kk = 0; kk < c; ++kk) {
        float p = G[kk + kk * ldg];
        if (!(p > 1e-8f)) {  // too ill-conditioned for CholeskyQR2 in FP32
          if (tid == 0) *fail = 1;
          p = 1.0f;
        }
        const float ri = rsqrtf(p);
        if (tid == 0) dg[kk] = p * ri;  // sqrt(p)
        for (int a = kk + 1 + tid; a < c; a += nt) G[kk + a * ldg] = G[a + kk * ldg] * ri;
        // trailing update of the lower triangle: a warp per column, lanes over rows
        for (int b = kk + 1 + wid; b < c; b += nw) {
          const float gb = G[b + kk * ldg] * ri * ri;
          for (int a = b + lane; a < c; a += 32) G[a + b * ldg] = fmaf(-G[a + kk * ldg], gb, G[a + b * ldg]);
        }
        __syncthreads();
      }
    }
    if (tid == 0) near_sh = 1;  // the next pass's Gram matrix decides afresh
    // Y <- Y L^{-T}, one row per thread
    for (int r = tid; r < n; r += nt) {
      float* yr = Yb + (size_t)r * ldb;
      for (int a = 0; a < c; ++a) {
        float acc = yr[a];
        const float* La = G + (size_t)a * ldg;  // L(a, b) at La[b], four at a time
        int b = 0;
        for (; b + 4 <= a; b += 4) {
          const float4 l = *reinterpret_cast<const float4*>(La + b);
          acc = fmaf(-yr[b], l.x, acc);
          acc = fmaf(-yr[b + 1], l.y, acc);
          acc = fmaf(-yr[b + 2], l.z, acc);
          acc = fmaf(-yr[b + 3], l.w, acc);
        }
        for (; b < a; ++b) acc = fmaf(-yr[b], La[b], acc);
        yr[a] = acc / dg[a];
      }
    }
    __syncthreads();
  }
  for (int r = wid; r < n; r += nw)
    for (int a = lane; a < c; a += 32) Y[(size_t)r * n + i + a] = Yb[r * ldb + a];
}

// ------------------------------------------------- 4. back-transformation --
// Reflectors k0 .. k0+7 (block b, k0 = 8 b) compose as H_k0 ... H_k0+7 =
// I - Vb Tb Vb^T with Tb upper triangular (forward, columnwise accumulation):
// Tb(j, j) = tau_j, Tb(0:j, j) = -tau_j Tb(0:j, 0:j) (Vb(:, 0:j)^T v_j).
constexpr int kWY = 8;

__global__ void __launch_bounds__(64)
tri_wy_kernel(int n, const float* __restrict__ V, const float* __restrict__ tauv, float* __restrict__ Tw) {
  __shared__ float gv[kWY][kWY];
  const int b = blockIdx.x, k0 = b * kWY, nref = n - 2;
  const int cnt = min(kWY, nref - k0);
  const int tid = threadIdx.x;
  if (tid < kWY * kWY) {
    const int a = tid % kWY, c = tid / kWY;
    float acc = 0.0f;
    if (a < c && c < cnt) {
      const float* va = V + (size_t)(k0 + a) * n;
      const float* vc = V + (size_t)(k0 + c) * n;
      for (int r = 0; r < n; ++r) acc = fmaf(va[r], vc[r], acc);
    }
    gv[a][c] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    float t[kWY][kWY] = {};
    for (int c = 0; c < cnt; ++c) {
      const float tc = tauv[k0 + c];
      for (int a = 0; a < c; ++a) {
        float s = 0.0f;
        for (int l = a; l < c; ++l) s = fmaf(t[a][l], gv[l][c], s);
        t[a][c] = -tc * s;
      }
      t[c][c] = tc;
    }
    for (int e = 0; e < kWY * kWY; ++e) Tw[(size_t)b * kWY * kWY + e] = t[e % kWY][e / kWY];
  }
}

// X(:, col) = H_0 H_1 ... H_{n-3} Y(:, col) in FP32 arithmetic (the FP32 stage's
// accuracy; the FP64 refinement follows), written as FP64; one warp per column, each
// lane holding kBackRows rows (32 kBackRows >= n: the kernel is instantiated
// for a few heights, so a small T_k does not carry the largest one's rows); the
// CTA stages kBackStage WY blocks at a time in shared memory.
constexpr int kBackWarps = 8;
constexpr int kBackStage = 2;

template <int kBackRows>
__global__ void __launch_bounds__(kBackWarps * 32)
tri_back_kernel(int n, const float* __restrict__ V, const float* __restrict__ Tw, const float* __restrict__ Y,
                double* __restrict__ X) {
  __shared__ float sv[kBackStage * kWY][kBackRows * 32];
  __shared__ float st[kBackStage][kWY * kWY];
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * kBackWarps + (threadIdx.x >> 5);
  const int nref = n - 2, nblk = nref > 0 ? (nref + kWY - 1) / kWY : 0;
  float z[kBackRows];
#pragma unroll
  for (int t = 0; t < kBackRows; ++t) {
    const int r = lane + 32 * t;
    z[t] = (col < n && r < n) ? Y[(size_t)r * n + col] : 0.0f;
  }
  for (int bt = nblk - 1; bt >= 0; bt -= kBackStage) {
    const int b0 = max(bt - kBackStage + 1, 0), nb = bt - b0 + 1;  // blocks b0 .. bt
    __syncthreads();
#pragma unroll 8
    for (int e = threadIdx.x; e < nb * kWY * kBackRows * 32; e += blockDim.x) {
      const int r = e % (kBackRows * 32), q = e / (kBackRows * 32);  // q: reflector within the stage
      const int k = b0 * kWY + q;
      sv[q][r] = (r < n && k < nref) ? V[r + (size_t)k * n] : 0.0f;
    }
    for (int e = threadIdx.x; e < nb * kWY * kWY; e += blockDim.x)
      st[e / (kWY * kWY)][e % (kWY * kWY)] = Tw[(size_t)b0 * kWY * kWY + e];
    __syncthreads();
    for (int q = nb - 1; q >= 0; --q) {
      // y = Vb^T z, u = Tb y, z -= Vb u
      float y[kWY];
#pragma unroll
      for (int a = 0; a < kWY; ++a) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < kBackRows; ++t) acc = fmaf(sv[q * kWY + a][lane + 32 * t], z[t], acc);
        y[a] = acc;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < kWY; ++a) y[a] += __shfl_xor_sync(0xffffffffu, y[a], o);
      float u[kWY];
#pragma unroll
      for (int a = 0; a < kWY; ++a) {
        float s = 0.0f;
#pragma unroll
        for (int c = a; c < kWY; ++c) s = fmaf(st[q][a + c * kWY], y[c], s);
        u[a] = s;
      }
#pragma unroll
      for (int t = 0; t < kBackRows; ++t) {
        float zt = z[t];
#pragma unroll
        for (int a = 0; a < kWY; ++a) zt = fmaf(-sv[q * kWY + a][lane + 32 * t], u[a], zt);
        z[t] = zt;
      }
    }
  }
  if (col >= n) return;
#pragma unroll
  for (int t = 0; t < kBackRows; ++t) {
    const int r = lane + 32 * t;
    if (r < n) X[r + (size_t)col * n] = (double)z[t];
  }
}

}  // namespace

bool tri_fits(Ctx* ctx, int n) {
  if (n <= kTriOneCtaMaxN) return true;
  if (n > kTriMaxN) return false;
  if (ctx->tri_route == 0 && rows_cluster(n) > 0)
    return (size_t)rows_smem_bytes<8>(n) + 1024 <= ctx->smem_optin;
  const int bytes = n <= kTriCl4MaxN ? cl_smem_bytes<4>(n) : cl_smem_bytes<8>(n);
  return (size_t)bytes + 1024 <= ctx->smem_optin;
}

blws_status tri_stage(Ctx* ctx, cudaStream_t s, int n, const double* T, double* X, int* grp, float* gtop,
                      int* fail) {
  if (n < 1 || !tri_fits(ctx, n)) return ctx->fail(BLWS_EINVAL, "tri_stage: n = %d", n);
  const bool on_cluster = n > kTriOneCtaMaxN;
  const bool cl8 = n > kTriCl4MaxN;
  const size_t nn = (size_t)n * n;
  const int nblk = n > 2 ? (n - 2 + kWY - 1) / kWY : 0;
  // F (4 nn, first: 16-byte aligned), V, Y, reduction partial sums, WY factors, d, e, tau, lam, scale
  const size_t parts = (size_t)std::max({kMaxGroups + kMaxChunks, 4 * (cl_groups<4>() + kClChunks),
                                         8 * (cl_groups<8>() + kClChunks)}) * n;
  float* f = nullptr;
  BLWS_TRY(ctx->get(BUF_TRI, (nn * 6 + parts + (size_t)nblk * kWY * kWY + (size_t)n * 4 + 64) * sizeof(float),
                    (void**)&f));
  float4* F = reinterpret_cast<float4*>(f);
  float* V = f + 4 * nn;
  float* Y = V + nn;
  float* part = Y + nn;
  float* Tw = part + parts;
  float* dv = Tw + (size_t)nblk * kWY * kWY;
  float* ev = dv + n;
  float* tauv = ev + n;
  float* lam = tauv + n;
  float* tscale = lam + n;
  // the reduction by rows (section 1c) wherever a cluster's share fits, else
  // the packed kernels (also selectable with BLWS_TRI=packed at context creation)
  const int kc = ctx->tri_route == 0 ? rows_cluster(n) : 0;
  if (kc == 1) {
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_TRI_ROWS1, (const void*)tri_rows_kernel<1>, rows_smem_bytes<1>(n)));
  } else if (kc == 2) {
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_TRI_ROWS2, (const void*)tri_rows_kernel<2>, rows_smem_bytes<2>(n)));
  } else if (kc == 4) {
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_TRI_ROWS4, (const void*)tri_rows_kernel<4>, rows_smem_bytes<4>(n)));
  } else if (kc == 8) {
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_TRI_ROWS8, (const void*)tri_rows_kernel<8>, rows_smem_bytes<8>(n)));
  } else if (on_cluster && cl8) {
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_TRI_CL8, (const void*)tri_reduce_cluster_kernel<8>, cl_smem_bytes<8>(n)));
  } else if (on_cluster) {
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_TRI_CL, (const void*)tri_reduce_cluster_kernel<4>, cl_smem_bytes<4>(n)));
  } else {
    const int smem = (n * (n + 1) / 2 + 4 * n + 4) * (int)sizeof(float);
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_TRI, (const void*)tri_reduce_kernel, smem));
  }
  // the group kernel's shared memory: the largest staged block n x (c|1) plus c x c, capped
  const int qr_floats = std::min((int)(((size_t)n * (n | 1) + (size_t)n * ((n + 3) & ~3) + 4)), kQrSmemFloats);
  const int gsmem = qr_floats * (int)sizeof(float);
  BLWS_TRY(ctx->smem_limit(Ctx::ATTR_TRI_INV, (const void*)tri_group_qr_kernel, gsmem));
  const int ssmem = n * ((int)sizeof(float4) + 4 * (int)sizeof(float));
  BLWS_TRY_CUDA(ctx, cudaMemsetAsync(fail, 0, sizeof(int), s));
  if (kc == 1)
    tri_rows_kernel<1><<<1, kTriRowsThreads, rows_smem_bytes<1>(n), s>>>(n, T, V, dv, ev, tauv, tscale, Y);
  else if (kc == 2)
    tri_rows_kernel<2><<<2, kTriRowsThreads, rows_smem_bytes<2>(n), s>>>(n, T, V, dv, ev, tauv, tscale, Y);
  else if (kc == 4)
    tri_rows_kernel<4><<<4, kTriRowsThreads, rows_smem_bytes<4>(n), s>>>(n, T, V, dv, ev, tauv, tscale, Y);
  else if (kc == 8)
    tri_rows_kernel<8><<<8, kTriRowsThreads, rows_smem_bytes<8>(n), s>>>(n, T, V, dv, ev, tauv, tscale, Y);
  else if (on_cluster && cl8)
    tri_reduce_cluster_kernel<8><<<8, kTriThreads, cl_smem_bytes<8>(n), s>>>(n, T, V, dv, ev, tauv, part, tscale);
  else if (on_cluster)
    tri_reduce_cluster_kernel<4><<<4, kTriThreads, cl_smem_bytes<4>(n), s>>>(n, T, V, dv, ev, tauv, part, tscale);
  else
    tri_reduce_kernel<<<1, kTriThreads, (n * (n + 1) / 2 + 4 * n + 4) * (int)sizeof(float), s>>>(
        n, T, V, dv, ev, tauv, part, tscale);
  BLWS_CHECK_LAUNCH(ctx);
  tri_bisect_kernel<<<ceil_div(n, 8), 256, 0, s>>>(n, dv, ev, lam);
  BLWS_CHECK_LAUNCH(ctx);
  tri_solve_kernel<true><<<n, 32, ssmem, s>>>(n, dv, ev, lam, tscale, F, Y, grp, gtop, fail);
  BLWS_CHECK_LAUNCH(ctx);
  tri_group_qr_kernel<<<n, kQrThreads, gsmem, s>>>(n, qr_floats, grp, Y, fail);
  BLWS_CHECK_LAUNCH(ctx);
  tri_solve_kernel<false><<<n, 32, ssmem, s>>>(n, dv, ev, lam, tscale, F, Y, grp, gtop, fail);
  BLWS_CHECK_LAUNCH(ctx);
  tri_group_qr_kernel<<<n, kQrThreads, gsmem, s>>>(n, qr_floats, grp, Y, fail);
  BLWS_CHECK_LAUNCH(ctx);
  if (nblk > 0) {
    tri_wy_kernel<<<nblk, 64, 0, s>>>(n, V, tauv, Tw);
    BLWS_CHECK_LAUNCH(ctx);
  }
  const int bg = ceil_div(n, kBackWarps), bt = kBackWarps * 32;
  static_assert((kTriMaxN + 31) / 32 <= 23, "heights of the back-transformation");
  if (n <= 128) tri_back_kernel<4><<<bg, bt, 0, s>>>(n, V, Tw, Y, X);
  else if (n <= 256) tri_back_kernel<8><<<bg, bt, 0, s>>>(n, V, Tw, Y, X);
  else if (n <= 384) tri_back_kernel<12><<<bg, bt, 0, s>>>(n, V, Tw, Y, X);
  else if (n <= 512) tri_back_kernel<16><<<bg, bt, 0, s>>>(n, V, Tw, Y, X);
  else tri_back_kernel<23><<<bg, bt, 0, s>>>(n, V, Tw, Y, X);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

}  // namespace blws
