// Symmetric eigen-decomposition of the projected matrix T_k (Algorithm 3,
// "EVD of T_k" with eigenvalues in decreasing order).
//
// GB300 has FP64 at 1/64 of the FP32 rate, and a one-SM FP64 Jacobi on a
// few-hundred-wide T_k costs milliseconds.  So the decomposition is done in
// two stages:
//   1. cyclic two-sided Jacobi in FP32 with the parallel (round-robin)
//      ordering, n/2 disjoint rotations per round applied as 2 x 2 block
//      updates (Golub & Van Loan, Section 8.5): one CTA with T in shared
//      memory when it fits, else a cooperative grid with one grid barrier per
//      round;
//   2. FP64 iterative refinement of the eigenvector matrix by Ogita & Aishima
//      ("Iterative refinement for symmetric eigenvalue decomposition", 2018),
//      which uses only matrix products (FP64 GEMMs over the whole GPU):
//        R = I - X^T X,  S = X^T T X,  lam_i = s_ii / (1 - r_ii),
//        E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i)  if |lam_i - lam_j| > d,
//               r_ij / 2 otherwise,   X <- X + X E,
//      with d = 2 (||S - diag(lam)|| + ||T|| ||R||) (Frobenius bounds here),
//      widened by a safety factor.  Each step squares the error of
//      well-separated pairs; closer pairs stay as an (orthonormalised) basis
//      of their joint eigenspace;
//   3. each cluster that can change the count above eps or a threshold is
//      solved again on its own (shifted and rescaled to O(1)) by stages 1-2.
// Pairs are sorted by decreasing eigenvalue.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ops.cuh"

namespace cg = cooperative_groups;

namespace blws {

namespace {

constexpr int kJacobiMaxSweeps = 16;
// FP32 stage: stop when off(A)^2 <= tol2 ||A||_F^2, or when off(A) is near the
// FP32 rounding floor (<= 3e-5 ||A||_F) and a sweep no longer cuts off(A)^2 by
// more than 3x;
// the FP64 refinement does the rest.
constexpr float kJacobiTol2 = 1e-11f;
constexpr float kJacobiFloor2 = 1e-9f;
constexpr int kRefineSteps = 3;
// The first-order refinement is only applied to pairs whose gap exceeds
// kClusterGamma times the Ogita-Aishima width d: closer pairs may start with
// O(1) mixing after the FP32 stage, outside the refinement's convergence
// region, so they are kept as a joint subspace and resolved by the cluster
// level (sym_eig).
constexpr double kClusterGamma = 64.0;

__device__ inline bool jacobi_done(int sweep, float off, float tot, float prev_off) {
  (void)sweep;
  return off <= kJacobiTol2 * tot || (off <= kJacobiFloor2 * tot && off > 0.3f * prev_off);
}
constexpr int kCtaMaxN = 160;       // A and V (FP32) in shared memory up to this size

struct Rot {
  int p, q;
  float c, s;
};

// Round-robin pairing of N (even) indices, round r in [0, N-1): pair k.
__device__ inline void rr_pair(int N, int r, int k, int& p, int& q) {
  if (k == 0) {
    p = r;
    q = N - 1;
  } else {
    p = (r + k) % (N - 1);
    q = (r - k + (N - 1)) % (N - 1);
  }
  if (p > q) {
    int t = p; p = q; q = t;
  }
}

// Jacobi rotation annihilating a_pq (Golub & Van Loan, Algorithm 8.5.1):
// J = [[c, s], [-s, c]] on (p, q), A' = J^T A J.
__device__ inline void jacobi_rot(float app, float aqq, float apq, float& c, float& s) {
  if (fabsf(apq) <= 1e-30f * (fabsf(app) + fabsf(aqq)) || apq == 0.0f) {
    c = 1.0f;
    s = 0.0f;
    return;
  }
  const float tau = (aqq - app) / (2.0f * apq);
  const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
  c = rsqrtf(1.0f + t * t);
  s = t * c;
}

// Apply one round to the 2x2 block (i, j): reads Ain, writes Aout (may alias).
__device__ inline void apply_block(const float* Ain, float* Aout, int N, const Rot& ri, const Rot& rj,
                                   bool diag) {
  const size_t pi = ri.p, qi = ri.q, pj = rj.p, qj = rj.q;
  const float a = Ain[pi + pj * N], b = Ain[pi + qj * N], c = Ain[qi + pj * N], d = Ain[qi + qj * N];
  // M = A J_j (columns)
  const float m_ap = rj.c * a - rj.s * b, m_aq = rj.s * a + rj.c * b;  // row p_i
  const float m_cp = rj.c * c - rj.s * d, m_cq = rj.s * c + rj.c * d;  // row q_i
  // J_i^T M (rows)
  float n_pp = ri.c * m_ap - ri.s * m_cp, n_pq = ri.c * m_aq - ri.s * m_cq;
  float n_qp = ri.s * m_ap + ri.c * m_cp, n_qq = ri.s * m_aq + ri.c * m_cq;
  if (diag) {  // the annihilated pair
    n_pq = 0.0f;
    n_qp = 0.0f;
  }
  Aout[pi + pj * N] = n_pp;
  Aout[pi + qj * N] = n_pq;
  Aout[qi + pj * N] = n_qp;
  Aout[qi + qj * N] = n_qq;
}

// --------------------------------------------- single-CTA Jacobi (smem) --
__global__ void __launch_bounds__(1024)
jacobi_cta_kernel(int n, int N, const double* __restrict__ T, float* __restrict__ Vout,
                  int* __restrict__ sweeps_out) {
  extern __shared__ float sm[];
  float* A = sm;
  float* V = A + (size_t)N * N;
  __shared__ Rot rot[kCtaMaxN / 2];
  __shared__ float red_off[32], red_tot[32];
  __shared__ int stop;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int half = N / 2;
  for (int e = tid; e < N * N; e += nt) {
    const int i = e % N, j = e / N;
    A[e] = (i < n && j < n) ? (float)T[i + (size_t)j * n] : 0.0f;
    V[e] = (i == j) ? 1.0f : 0.0f;
  }
  if (tid == 0) stop = 0;
  __syncthreads();
  int sweep = 0;
  float prev_off = 3.0e38f;
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    for (int r = 0; r < N - 1; ++r) {
      for (int k = tid; k < half; k += nt) {
        Rot R;
        rr_pair(N, r, k, R.p, R.q);
        jacobi_rot(A[R.p + R.p * N], A[R.q + R.q * N], A[R.p + R.q * N], R.c, R.s);
        rot[k] = R;
      }
      __syncthreads();
      for (int e = tid; e < half * half; e += nt) {
        const int i = e % half, j = e / half;
        apply_block(A, A, N, rot[i], rot[j], i == j);
      }
      for (int e = tid; e < N * half; e += nt) {
        const int x = e % N, j = e / N;
        const Rot R = rot[j];
        const float vp = V[x + (size_t)R.p * N], vq = V[x + (size_t)R.q * N];
        V[x + (size_t)R.p * N] = R.c * vp - R.s * vq;
        V[x + (size_t)R.q * N] = R.s * vp + R.c * vq;
      }
      __syncthreads();
    }
    // convergence: off(A)^2 <= tol^2 ||A||_F^2
    float off = 0.0f, tot = 0.0f;
    for (int e = tid; e < N * N; e += nt) {
      const float v = A[e];
      tot += v * v;
      if (e % N != e / N) off += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (tid % 32 == 0) {
      red_off[tid / 32] = off;
      red_tot[tid / 32] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      float so = 0.0f, st = 0.0f;
      for (int w = 0; w < nt / 32; ++w) {
        so += red_off[w];
        st += red_tot[w];
      }
      red_tot[0] = so;  // broadcast this sweep's off(A)^2
      stop = jacobi_done(sweep, so, st, prev_off) ? 1 : 0;
    }
    __syncthreads();
    prev_off = red_tot[0];
    if (stop) {
      ++sweep;
      break;
    }
    __syncthreads();
  }
  for (int e = tid; e < N * N; e += nt) Vout[e] = V[e];
  if (tid == 0) *sweeps_out = sweep;
}

// --------------------------------- block-pair Jacobi (cooperative grid) --
// Blocks of kBS indices; each round pairs the nb blocks round-robin.  Phase 1:
// one CTA per block pair runs ONE cyclic Jacobi sweep on its (2 kBS)^2
// diagonal sub-block in shared memory and records the accumulated orthogonal
// Q (2 kBS x 2 kBS).  Phase 2: every off-diagonal block pair (a, b) becomes
// Q_a^T A_ab Q_b, and every row chunk of V becomes V Q_a.  One grid barrier
// per phase: 2 (nb - 1) barriers per sweep instead of one per scalar round.
// Block width: BS indices per block, 2 BS per pair (template parameters, so
// the shared-memory tiles and loop bounds are compile-time constants).
#ifndef BLWS_JACOBI_BS
#define BLWS_JACOBI_BS 8
#endif
constexpr int kBS = BLWS_JACOBI_BS;
constexpr int kBlockThreads = kBS >= 32 ? 512 : 256;

__device__ inline int blk_of_pair(int nb, int r, int k, int which) {
  int p, q;
  rr_pair(nb, r, k, p, q);
  return which ? q : p;
}

// global index of local row i (0..2 BS) of pair (bp, bq)
template <int BS>
__device__ inline int pair_index(int bp, int bq, int i) {
  return i < BS ? bp * BS + i : bq * BS + (i - BS);
}

template <int BS, int NT>
__global__ void __launch_bounds__(NT)
jacobi_block_kernel(int n, int N, const double* __restrict__ T, float* A, float* V, float* Qbuf,
                    float2* part, int* sweeps_out) {
  constexpr int kB2 = 2 * BS;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ float bsm[];
  float(*S1)[kB2 + 1] = reinterpret_cast<float(*)[kB2 + 1]>(bsm);
  float(*S2)[kB2 + 1] = reinterpret_cast<float(*)[kB2 + 1]>(bsm + kB2 * (kB2 + 1));
  float(*S3)[kB2 + 1] = reinterpret_cast<float(*)[kB2 + 1]>(bsm + 2 * kB2 * (kB2 + 1));
  float(*S4)[kB2 + 1] = reinterpret_cast<float(*)[kB2 + 1]>(bsm + 3 * kB2 * (kB2 + 1));
  __shared__ Rot rot[kB2 / 2];
  __shared__ float red_off[NT / 32], red_tot[NT / 32];
  const int tid = threadIdx.x, nt = NT;
  const int nb = N / BS, P = nb / 2;
  const size_t gtid = (size_t)blockIdx.x * nt + tid, gnt = (size_t)gridDim.x * nt;
  for (size_t e = gtid; e < (size_t)N * N; e += gnt) {
    const int i = (int)(e % N), j = (int)(e / N);
    A[e] = (i < n && j < n) ? (float)T[i + (size_t)j * n] : 0.0f;
    V[e] = (i == j) ? 1.0f : 0.0f;
  }
  grid.sync();
  int sweep = 0;
  float prev_off = 3.0e38f;
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    float off = 0.0f, tot = 0.0f;
    for (int r = 0; r < nb - 1; ++r) {
      const bool last = (r == nb - 2);
      // ---- phase 1: one inner sweep per diagonal block pair
      for (int k = blockIdx.x; k < P; k += gridDim.x) {
        const int bp = blk_of_pair(nb, r, k, 0), bq = blk_of_pair(nb, r, k, 1);
        for (int e = tid; e < kB2 * kB2; e += nt) {
          const int i = e % kB2, j = e / kB2;
          S1[i][j] = A[pair_index<BS>(bp, bq, i) + (size_t)pair_index<BS>(bp, bq, j) * N];
          S2[i][j] = (i == j) ? 1.0f : 0.0f;
        }
        __syncthreads();
        for (int ir = 0; ir < kB2 - 1; ++ir) {
          if (tid < kB2 / 2) {
            Rot R;
            rr_pair(kB2, ir, tid, R.p, R.q);
            jacobi_rot(S1[R.p][R.p], S1[R.q][R.q], S1[R.p][R.q], R.c, R.s);
            rot[tid] = R;
          }
          __syncthreads();
          for (int e = tid; e < (kB2 / 2) * (kB2 / 2); e += nt) {
            const int i = e % (kB2 / 2), j = e / (kB2 / 2);
            const Rot ri = rot[i], rj = rot[j];
            const float a = S1[ri.p][rj.p], b = S1[ri.p][rj.q], c = S1[ri.q][rj.p], d = S1[ri.q][rj.q];
            const float m_ap = rj.c * a - rj.s * b, m_aq = rj.s * a + rj.c * b;
            const float m_cp = rj.c * c - rj.s * d, m_cq = rj.s * c + rj.c * d;
            float n_pq = ri.c * m_aq - ri.s * m_cq, n_qp = ri.s * m_ap + ri.c * m_cp;
            if (i == j) { n_pq = 0.0f; n_qp = 0.0f; }
            S1[ri.p][rj.p] = ri.c * m_ap - ri.s * m_cp;
            S1[ri.p][rj.q] = n_pq;
            S1[ri.q][rj.p] = n_qp;
            S1[ri.q][rj.q] = ri.s * m_aq + ri.c * m_cq;
          }
          for (int e = tid; e < kB2 * (kB2 / 2); e += nt) {
            const int x = e % kB2, j = e / kB2;
            const Rot R = rot[j];
            const float vp = S2[x][R.p], vq = S2[x][R.q];
            S2[x][R.p] = R.c * vp - R.s * vq;
            S2[x][R.q] = R.s * vp + R.c * vq;
          }
          __syncthreads();
        }
        float lo = 0.0f, lt = 0.0f;
        for (int e = tid; e < kB2 * kB2; e += nt) {
          const int i = e % kB2, j = e / kB2;
          const float v = S1[i][j];
          A[pair_index<BS>(bp, bq, i) + (size_t)pair_index<BS>(bp, bq, j) * N] = v;
          Qbuf[(size_t)k * kB2 * kB2 + e] = S2[i][j];
          if (last) {
            lt += v * v;
            if (i != j) lo += v * v;
          }
        }
        off += lo;
        tot += lt;
        __syncthreads();
      }
      grid.sync();
      // ---- phase 2: off-diagonal block pairs (a < b) and row chunks of V
      const int npairs = P * (P - 1) / 2;
      const int nv = (N / kB2) * P;
      for (int item = blockIdx.x; item < npairs + nv; item += gridDim.x) {
        if (item < npairs) {
          // unrank item -> (a, b), a < b
          int a = 0, rem = item;
          while (rem >= P - 1 - a) { rem -= P - 1 - a; ++a; }
          const int b = a + 1 + rem;
          const int ap = blk_of_pair(nb, r, a, 0), aq = blk_of_pair(nb, r, a, 1);
          const int bp = blk_of_pair(nb, r, b, 0), bq = blk_of_pair(nb, r, b, 1);
          for (int e = tid; e < kB2 * kB2; e += nt) {
            const int i = e % kB2, j = e / kB2;
            S1[i][j] = A[pair_index<BS>(ap, aq, i) + (size_t)pair_index<BS>(bp, bq, j) * N];
            S2[i][j] = Qbuf[(size_t)a * kB2 * kB2 + e];
            S3[i][j] = Qbuf[(size_t)b * kB2 * kB2 + e];
          }
          __syncthreads();
          // S4 = Qa^T S1
          for (int e = tid; e < kB2 * kB2; e += nt) {
            const int i = e % kB2, j = e / kB2;
            float acc = 0.0f;
#pragma unroll 8
            for (int t = 0; t < kB2; ++t) acc = fmaf(S2[t][i], S1[t][j], acc);
            S4[i][j] = acc;
          }
          __syncthreads();
          float lo = 0.0f;
          for (int e = tid; e < kB2 * kB2; e += nt) {
            const int i = e % kB2, j = e / kB2;
            float acc = 0.0f;
#pragma unroll 8
            for (int t = 0; t < kB2; ++t) acc = fmaf(S4[i][t], S3[t][j], acc);
            const int gi = pair_index<BS>(ap, aq, i), gj = pair_index<BS>(bp, bq, j);
            A[gi + (size_t)gj * N] = acc;
            A[gj + (size_t)gi * N] = acc;
            lo += acc * acc;
          }
          if (last) {
            off += 2.0f * lo;
            tot += 2.0f * lo;
          }
          __syncthreads();
        } else {
          const int it2 = item - npairs;
          const int chunk = it2 % (N / kB2), a = it2 / (N / kB2);
          const int ap = blk_of_pair(nb, r, a, 0), aq = blk_of_pair(nb, r, a, 1);
          for (int e = tid; e < kB2 * kB2; e += nt) {
            const int i = e % kB2, j = e / kB2;
            S1[i][j] = V[(chunk * kB2 + i) + (size_t)pair_index<BS>(ap, aq, j) * N];
            S2[i][j] = Qbuf[(size_t)a * kB2 * kB2 + e];
          }
          __syncthreads();
          for (int e = tid; e < kB2 * kB2; e += nt) {
            const int i = e % kB2, j = e / kB2;
            float acc = 0.0f;
#pragma unroll 8
            for (int t = 0; t < kB2; ++t) acc = fmaf(S1[i][t], S2[t][j], acc);
            V[(chunk * kB2 + i) + (size_t)pair_index<BS>(ap, aq, j) * N] = acc;
          }
          __syncthreads();
        }
      }
      grid.sync();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (tid % 32 == 0) {
      red_off[tid / 32] = off;
      red_tot[tid / 32] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      float so = 0.0f, st = 0.0f;
      for (int w = 0; w < nt / 32; ++w) {
        so += red_off[w];
        st += red_tot[w];
      }
      part[blockIdx.x] = make_float2(so, st);
    }
    grid.sync();
    float so = 0.0f, st = 0.0f;
    for (int c = 0; c < (int)gridDim.x; ++c) {
      so += part[c].x;
      st += part[c].y;
    }
    grid.sync();
    const bool done = jacobi_done(sweep, so, st, prev_off);
    prev_off = so;
    if (done) {
      ++sweep;
      break;
    }
  }
  if (blockIdx.x == 0 && tid == 0) *sweeps_out = sweep;
}

// ------------------------------------------------------ refinement helpers --
__global__ void f32_to_f64_block(int n, int N, const float* __restrict__ V, double* __restrict__ X) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    X[e] = (double)V[i + (size_t)j * N];
  }
}

// R <- I - R (in place, R holds X^T X)
__global__ void identity_minus(int n, double* R) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    R[e] = (i == j ? 1.0 : 0.0) - R[e];
  }
}

// partial sums (per CTA): [0] sum_{i!=j} S_ij^2, [1] sum R_ij^2, [2] sum T_ij^2
// Off-diagonal entries inside a group of the FP32 stage (grp, may be null)
// are left out: the group's columns span its eigenspace without being
// eigenvectors one by one, and the refinement keeps them as one subspace.
__global__ void oa_norms_partial(int n, const double* __restrict__ S, const double* __restrict__ R,
                                 const double* __restrict__ T, const int* __restrict__ grp, double* part) {
  __shared__ double red[3][256];
  double a = 0.0, b = 0.0, c = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i != j && !(grp && grp[i] >= 0 && grp[i] == grp[j])) a = fma(S[e], S[e], a);
    b = fma(R[e], R[e], b);
    c = fma(T[e], T[e], c);
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
      red[2][threadIdx.x] += red[2][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = red[0][0];
    part[3 * blockIdx.x + 1] = red[1][0];
    part[3 * blockIdx.x + 2] = red[2][0];
  }
}

// lam_i = s_ii / (1 - r_ii); the diagonal part of ||S - D|| is added to the
// off-diagonal partials; writes lam[n] and delta (scal[0]).
__global__ void oa_lambda(int n, int nparts, const double* __restrict__ S, const double* __restrict__ R,
                          const double* __restrict__ part, double* lam, double* delta) {
  __shared__ double red[3][256];
  double dsum = 0.0, r2 = 0.0, t2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double l = S[i + (size_t)i * n] / (1.0 - R[i + (size_t)i * n]);
    lam[i] = l;
    const double dv = S[i + (size_t)i * n] - l;
    dsum = fma(dv, dv, dsum);
  }
  // the CTA partials of oa_norms_partial: thread t adds parts t, t + 256, ...
  // (fixed assignment and tree: deterministic)
  for (int c = threadIdx.x; c < nparts; c += blockDim.x) {
    dsum += part[3 * c + 0];
    r2 += part[3 * c + 1];
    t2 += part[3 * c + 2];
  }
  red[0][threadIdx.x] = dsum;
  red[1][threadIdx.x] = r2;
  red[2][threadIdx.x] = t2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
      red[2][threadIdx.x] += red[2][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    *delta = kClusterGamma * 2.0 * (sqrt(red[0][0]) + sqrt(red[2][0]) * sqrt(red[1][0]));
}

__global__ void oa_correction(int n, const double* __restrict__ S, const double* __restrict__ R,
                              const double* __restrict__ lam, const double* __restrict__ delta,
                              const int* __restrict__ grp, double* E) {
  const double d = *delta;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    const double rij = R[e];
    double v;
    if (i == j || (grp && grp[i] >= 0 && grp[i] == grp[j])) {
      v = 0.5 * rij;
    } else {
      const double gap = lam[j] - lam[i];
      v = (fabs(gap) > d) ? (S[e] + lam[j] * rij) / gap : 0.5 * rij;
    }
    E[e] = v;
  }
}

// rank of each eigenvalue in decreasing order (ties by index), then scatter
__global__ void sort_desc(int n, const double* __restrict__ lam_in, const double* __restrict__ X,
                          const int* __restrict__ grp_in, const float* __restrict__ gtop_in, double* lam_out,
                          double* Z, int* grp_out) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const double li = lam_in[i];
    int c = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double lj = lam_in[j];
      c += (lj > li || (lj == li && j < i)) ? 1 : 0;
    }
    atomicAdd(&cnt, c);  // integer count: order-independent
    __syncthreads();
    const int rank = cnt;
    if (threadIdx.x == 0) {
      lam_out[rank] = li;
      if (grp_out) {  // group id, then the group's top eigenvalue (n ints, n floats)
        grp_out[rank] = grp_in ? grp_in[i] : -1;
        reinterpret_cast<float*>(grp_out + n)[rank] = gtop_in ? gtop_in[i] : 0.0f;
      }
    }
    for (int x = threadIdx.x; x < n; x += blockDim.x) Z[x + (size_t)rank * n] = X[x + (size_t)i * n];
    __syncthreads();
  }
}

}  // namespace

// One level: FP32 Jacobi, FP64 refinement, sort.  *delta_dev receives the
// refinement's cluster width d (pairs closer than d are not resolved).
blws_status sym_eig_level(Ctx* ctx, cudaStream_t s, int n, const double* T, double* lam, double* Z,
                          double* delta_out, bool sorted = true, int* tri_fail = nullptr,
                          int* grp_sorted = nullptr) {
  if (n <= 0) return BLWS_OK;
  // FP32 stage: the tridiagonal route (tri_eig.cu) where the packed matrix fits
  // one CTA; otherwise, and for the block-diagonal second level (whose columns
  // must stay inside their blocks), Jacobi
  const bool tri = tri_fail != nullptr && n >= 3 && tri_fits(ctx, n);
  const bool small = n + (n & 1) <= kCtaMaxN;
  // padded size: even for the one-CTA solver; an even number of kBS blocks otherwise
  const int N = small ? n + (n & 1) : ceil_div(n, 2 * kBS) * 2 * kBS;
  // scratch: FP32 A0, A1, V (N^2 each) ; FP64 X, X2, R, S, TX, E (n^2 each); small vectors
  float* f = nullptr;
  BLWS_TRY(ctx->get(BUF_EIG, (size_t)3 * N * N * sizeof(float) + (size_t)6 * n * n * sizeof(double) +
                                 (size_t)(4 * n + 3 * 1024 + 64) * sizeof(double),
                    (void**)&f));
  float* A0 = f;
  float* A1 = A0 + (size_t)N * N;
  float* V = A1 + (size_t)N * N;
  double* X = reinterpret_cast<double*>(V + (size_t)N * N + ((N * N) & 1));  // 8-byte aligned
  double* X2 = X + (size_t)n * n;
  double* R = X2 + (size_t)n * n;
  double* S = R + (size_t)n * n;
  double* TX = S + (size_t)n * n;
  double* E = TX + (size_t)n * n;
  double* lam_u = E + (size_t)n * n;
  double* part = lam_u + n;
  double* delta = part + 3 * 1024;
  int* sweeps = reinterpret_cast<int*>(delta + 8);
  int* grp = reinterpret_cast<int*>(delta + 16);  // groups of the tridiagonal stage (n ints)
  float* gtop = reinterpret_cast<float*>(grp + n);  // their largest eigenvalues (n floats)

  if (tri_fail && !tri) BLWS_TRY_CUDA(ctx, cudaMemsetAsync(tri_fail, 0, sizeof(int), s));
  if (tri) {
    BLWS_TRY(tri_stage(ctx, s, n, T, X, grp, gtop, tri_fail));
  } else if (small) {
    const size_t smem = 2ull * N * N * sizeof(float);
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_JACOBI_CTA, (const void*)jacobi_cta_kernel, (int)smem));
    jacobi_cta_kernel<<<1, 1024, smem, s>>>(n, N, T, V, sweeps);
    BLWS_CHECK_LAUNCH(ctx);
  } else {
    // block-pair Jacobi: Qbuf (P x 2 kBS x 2 kBS) reuses A1
    auto kern = jacobi_block_kernel<kBS, kBlockThreads>;
    const int smem = 4 * (2 * kBS) * (2 * kBS + 1) * (int)sizeof(float);
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_JACOBI_BLOCK, (const void*)kern, smem));
    if (ctx->jacobi_block_per_sm == 0) {
      BLWS_TRY_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctx->jacobi_block_per_sm, kern,
                                                                       kBlockThreads, smem));
      if (ctx->jacobi_block_per_sm < 1) return ctx->fail(BLWS_ECUDA, "jacobi_block_kernel cannot be resident");
    }
    const int per_sm = ctx->jacobi_block_per_sm;
    const int P = N / kBS / 2;
    const int items = P * (P - 1) / 2 + (N / (2 * kBS)) * P;
    int grid = std::min(std::max(items, P), ctx->sms * per_sm);
    grid = std::max(std::min(grid, ctx->sms * per_sm), 1);
    float2* fpart = reinterpret_cast<float2*>(part);
    int nn = n, NN = N;
    void* args[] = {&nn, &NN, (void*)&T, &A0, &V, &A1, &fpart, &sweeps};
    BLWS_TRY_CUDA(ctx, cudaLaunchCooperativeKernel((void*)kern, grid, kBlockThreads, args, smem, s));
    ++ctx->launches;
  }
  const int eb = std::min(ceil_div((long long)n * n, 256), ctx->sms * 4);
  if (!tri) {
    f32_to_f64_block<<<eb, 256, 0, s>>>(n, N, V, X);
    BLWS_CHECK_LAUNCH(ctx);
  }
  const int nparts = std::min(eb, 1024);
  for (int step = 0; step < kRefineSteps; ++step) {
    BLWS_TRY(gemm(ctx, s, true, false, n, n, n, 1.0, X, n, X, n, 0.0, R, n));
    identity_minus<<<eb, 256, 0, s>>>(n, R);
    BLWS_CHECK_LAUNCH(ctx);
    BLWS_TRY(gemm(ctx, s, false, false, n, n, n, 1.0, T, n, X, n, 0.0, TX, n));
    BLWS_TRY(gemm_sym(ctx, s, true, false, n, n, 1.0, X, n, TX, n, S, n));  // X^T T X: one triangle
    oa_norms_partial<<<nparts, 256, 0, s>>>(n, S, R, T, tri ? grp : nullptr, part);
    BLWS_CHECK_LAUNCH(ctx);
    oa_lambda<<<1, 256, 0, s>>>(n, nparts, S, R, part, lam_u, delta);
    BLWS_CHECK_LAUNCH(ctx);
    oa_correction<<<eb, 256, 0, s>>>(n, S, R, lam_u, delta, tri ? grp : nullptr, E);
    BLWS_CHECK_LAUNCH(ctx);
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(X2, X, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
    BLWS_TRY(gemm(ctx, s, false, false, n, n, n, 1.0, X, n, E, n, 1.0, X2, n));
    std::swap(X, X2);
  }
  if (sorted) {
    sort_desc<<<std::min(n, ctx->sms * 4), 128, 0, s>>>(n, lam_u, X, tri ? grp : nullptr, tri ? gtop : nullptr,
                                                        lam, Z, grp_sorted);
    BLWS_CHECK_LAUNCH(ctx);
  } else {
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(lam, lam_u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(Z, X, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
  }
  if (delta_out)
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(delta_out, delta, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return BLWS_OK;
}

namespace {

// K = blockdiag over clusters of (sym(S) - mu_c I) / scale_c; cross-cluster
// entries 0.  S = X^T (T X) from two GEMMs is symmetric only up to rounding,
// and for an exactly degenerate cluster S - mu I is nothing but that rounding:
// without the symmetrisation K would be a non-symmetric noise matrix and its
// "eigenvectors" would not be orthogonal.
__global__ void cluster_blocks(int n2, const double* __restrict__ S, const int* __restrict__ blk,
                               const double* __restrict__ mu, const double* __restrict__ inv_scale,
                               double* K) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2 * n2; e += gridDim.x * blockDim.x) {
    const int a = e % n2, b = e / n2;
    double v = 0.0;
    if (blk[a] == blk[b])
      v = (0.5 * (S[e] + S[b + (size_t)a * n2]) - (a == b ? mu[a] : 0.0)) * inv_scale[a];
    K[e] = v;
  }
}

// Out(:, p) = In(:, perm[p])
__global__ void gather_cols(int rows, int cols, const double* __restrict__ In,
                            const int* __restrict__ perm, double* Out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)rows * cols;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % rows), p = (int)(e / rows);
    Out[e] = In[r + (size_t)perm[p] * rows];
  }
}

}  // namespace

// layout of the pinned host copies: eigenvalues (n), group ids and tops (2n
// ints), then the refinement width and the failure flag
size_t eig_host_bytes(int n) { return sizeof(double) * n + sizeof(int) * 2 * (size_t)n + 2 * sizeof(double); }

double* sym_eig_host_extra(Ctx* ctx, int n) {
  return reinterpret_cast<double*>(static_cast<char*>(ctx->host_eig) + eig_host_bytes(n));
}

blws_status eig_copy_back(Ctx* ctx, cudaStream_t s, int n, const double* lam, const int* dgrp,
                          const double* scal) {
  char* h = static_cast<char*>(ctx->host_eig);
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(h, lam, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(h + sizeof(double) * n, dgrp, sizeof(int) * 2 * n,
                                     cudaMemcpyDeviceToHost, s));
  double* tail = reinterpret_cast<double*>(h + sizeof(double) * n + sizeof(int) * 2 * (size_t)n);
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(tail, scal + SLOT_AUX2, sizeof(double), cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(tail + 1, scal + SLOT_TRIFAIL, sizeof(double), cudaMemcpyDeviceToHost, s));
  return BLWS_OK;
}

blws_status sym_eig_start(Ctx* ctx, cudaStream_t s, int n, const double* T, double* lam, double* Z) {
  if (n <= 0) return BLWS_OK;
  double* scal;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  const bool tri_enabled = ctx->eig_route != 1;
  int* dgrp = nullptr;  // sorted group ids and group tops of the tridiagonal stage (n ints, n floats)
  BLWS_TRY(ctx->get(BUF_EIG_GRP, (size_t)2 * n, &dgrp));
  BLWS_TRY(ctx->host_eig_get(eig_host_bytes(n) + sizeof(double)));
  BLWS_TRY(sym_eig_level(ctx, s, n, T, lam, Z, scal + SLOT_AUX2, true,
                         tri_enabled ? reinterpret_cast<int*>(scal + SLOT_TRIFAIL) : nullptr, dgrp));
  return eig_copy_back(ctx, s, n, lam, dgrp, scal);
}

blws_status sym_eig(Ctx* ctx, cudaStream_t s, int n, const double* T, double* lam, double* Z,
                    double eps) {
  if (n <= 0) return BLWS_OK;
  BLWS_TRY(sym_eig_start(ctx, s, n, T, lam, Z));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  return sym_eig_finish(ctx, s, n, T, lam, Z, eps);
}

blws_status sym_eig_finish(Ctx* ctx, cudaStream_t s, int n, const double* T, double* lam, double* Z,
                           double eps) {
  if (n <= 0) return BLWS_OK;
  double* scal;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  const bool tri_enabled = ctx->eig_route != 1;
  int* dgrp = nullptr;
  BLWS_TRY(ctx->get(BUF_EIG_GRP, (size_t)2 * n, &dgrp));
  // Second level for clusters: eigenvalues closer than the refinement width d
  // are only resolved as a joint subspace, with values accurate to ~d (the
  // FP32 stage's absolute accuracy, ~1e-7 ||T||).  Where that could change
  // the count above eps or a threshold sigma - eps, the cluster is solved
  // again on its own: K = (X_C^T T X_C - mu I) / scale has O(1) entries, so
  // the same two-stage solver resolves it to ~1e-7 of the cluster's width.
  char* hb = static_cast<char*>(ctx->host_eig);
  const double* hl = reinterpret_cast<const double*>(hb);
  const int* hg = reinterpret_cast<const int*>(hb + sizeof(double) * n);
  const double* htail = reinterpret_cast<const double*>(hb + sizeof(double) * n + sizeof(int) * 2 * (size_t)n);
  if (tri_enabled && (*reinterpret_cast<const int*>(htail + 1) != 0 || !std::isfinite(htail[0]))) {
    // the FP32 tridiagonal stage met a group it could not orthonormalise or a
    // solve it could not normalise: Jacobi instead
    ++ctx->tri_fallbacks;
    BLWS_TRY(sym_eig_level(ctx, s, n, T, lam, Z, scal + SLOT_AUX2, true, nullptr, dgrp));
    BLWS_TRY(eig_copy_back(ctx, s, n, lam, dgrp, scal));
    BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  }
  const double d = htail[0];
  if (!(d > 0.0)) return BLWS_OK;
  // Clusters: runs of sorted values closer than d, joined with the groups of
  // the tridiagonal stage (whose columns are a basis of the group's
  // eigenspace and whose values are Rayleigh quotients inside the group's
  // range, so a group is contiguous in sorted order).  A group's values can
  // sit below its largest eigenvalue: its top from the FP32 stage, widened
  // by 1e-5 ||T|| (the FP32 stage's accuracy with room to spare), bounds it.
  // A cluster is solved again when it can reach above eps - 3d.
  const double tnorm = std::max(std::fabs(hl[0]), std::fabs(hl[n - 1]));
  const float* htop = reinterpret_cast<const float*>(hg + n);
  struct Cl { int i, j; double mu, scale; };
  std::vector<Cl> cl;
  int n2 = 0;
  for (int i = 0; i < n;) {
    int j = i + 1;
    while (j < n && (hl[j - 1] - hl[j] <= d || (hg[j] >= 0 && hg[j] == hg[j - 1]))) ++j;
    double top = hl[i];
    for (int t = i; t < j; ++t)
      if (hg[t] >= 0) top = std::max(top, (double)htop[t] + 1e-5 * tnorm);
    const double hidden = top - hl[i];
    if (j - i >= 2 && top > eps - 3.0 * d) {
      cl.push_back({i, j, 0.5 * (hl[i] + hl[j - 1]), 0.5 * (hl[i] - hl[j - 1]) + d + hidden});
      n2 += j - i;
    }
    i = j;
  }
  if (cl.empty()) return BLWS_OK;
  // all clusters in one block-diagonal problem
  double* w;
  BLWS_TRY(ctx->get(BUF_EIG2, (size_t)n * n2 * 3 + (size_t)n2 * n2 * 3 + (size_t)n2 * 4, &w));
  double* Xu = w;                        // n x n2: the clusters' current vectors
  double* TX = Xu + (size_t)n * n2;      // n x n2
  double* Zc = TX + (size_t)n * n2;      // n x n2
  double* S = Zc + (size_t)n * n2;       // n2 x n2
  double* K = S + (size_t)n2 * n2;       // n2 x n2
  double* ZK = K + (size_t)n2 * n2;      // n2 x n2
  double* nu = ZK + (size_t)n2 * n2;     // n2
  double* bmu = nu + n2;                 // n2
  double* binv = bmu + n2;               // n2
  int* bid = reinterpret_cast<int*>(binv + n2);  // n2 ints, then n2 ints of perm
  int* perm = bid + n2;
  std::vector<double> hmu(n2), hinv(n2);
  std::vector<int> hid(n2);
  for (size_t c = 0, o = 0; c < cl.size(); ++c) {
    const int sz = cl[c].j - cl[c].i;
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(Xu + o * n, Z + (size_t)cl[c].i * n, sizeof(double) * n * sz,
                                       cudaMemcpyDeviceToDevice, s));
    for (int t = 0; t < sz; ++t) {
      hmu[o + t] = cl[c].mu;
      hinv[o + t] = 1.0 / cl[c].scale;
      hid[o + t] = (int)c;
    }
    o += sz;
  }
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(bmu, hmu.data(), sizeof(double) * n2, cudaMemcpyHostToDevice, s));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(binv, hinv.data(), sizeof(double) * n2, cudaMemcpyHostToDevice, s));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(bid, hid.data(), sizeof(int) * n2, cudaMemcpyHostToDevice, s));
  BLWS_TRY(gemm(ctx, s, false, false, n, n2, n, 1.0, T, n, Xu, n, 0.0, TX, n));
  BLWS_TRY(gemm_sym(ctx, s, true, false, n2, n, 1.0, Xu, n, TX, n, S, n2));
  cluster_blocks<<<std::min(ceil_div((long long)n2 * n2, 256), ctx->sms * 4), 256, 0, s>>>(
      n2, S, bid, bmu, binv, K);
  BLWS_CHECK_LAUNCH(ctx);
  // block-diagonal K: cross-block entries stay exactly zero through the Jacobi
  // rotations and the refinement, so unsorted column a belongs to block bid[a]
  BLWS_TRY(sym_eig_level(ctx, s, n2, K, nu, ZK, nullptr, false));
  std::vector<double> hnu(n2);
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(hnu.data(), nu, sizeof(double) * n2, cudaMemcpyDeviceToHost, s));
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  std::vector<int> hperm(n2);
  std::vector<double> hlam(n2);
  for (size_t c = 0, o = 0; c < cl.size(); ++c) {
    const int sz = cl[c].j - cl[c].i;
    for (int t = 0; t < sz; ++t) hperm[o + t] = (int)(o + t);
    std::stable_sort(hperm.begin() + o, hperm.begin() + o + sz,
                     [&](int a, int b) { return hnu[a] > hnu[b]; });
    for (int t = 0; t < sz; ++t) hlam[o + t] = cl[c].mu + cl[c].scale * hnu[hperm[o + t]];
    o += sz;
  }
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(perm, hperm.data(), sizeof(int) * n2, cudaMemcpyHostToDevice, s));
  BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(bmu, hlam.data(), sizeof(double) * n2, cudaMemcpyHostToDevice, s));
  gather_cols<<<std::min(ceil_div((long long)n2 * n2, 256), ctx->sms * 4), 256, 0, s>>>(n2, n2, ZK,
                                                                                      perm, K);
  BLWS_CHECK_LAUNCH(ctx);
  BLWS_TRY(gemm(ctx, s, false, false, n, n2, n2, 1.0, Xu, n, K, n2, 0.0, Zc, n));
  for (size_t c = 0, o = 0; c < cl.size(); ++c) {
    const int sz = cl[c].j - cl[c].i;
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(Z + (size_t)cl[c].i * n, Zc + o * n, sizeof(double) * n * sz,
                                       cudaMemcpyDeviceToDevice, s));
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(lam + cl[c].i, bmu + o, sizeof(double) * sz,
                                       cudaMemcpyDeviceToDevice, s));
    o += sz;
  }
  // the host vectors above are read by asynchronous copies: wait before they go
  BLWS_TRY_CUDA(ctx, cudaStreamSynchronize(s));
  return BLWS_OK;
}

}  // namespace blws
