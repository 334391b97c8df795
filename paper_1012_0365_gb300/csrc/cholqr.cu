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
// the whole GPU; the b x b factorisation runs on one thread-block cluster
// (one CTA for b above kCMaxB).
#include <cooperative_groups.h>

#include "ops.cuh"

namespace cg = cooperative_groups;

namespace blws {

namespace {

// 1 / sqrt(p) for a pivot p in (1e-30, 1e30): an FP32 estimate y0 and one
// third-order correction in FP64.  With e = 1 - p y0^2,
// 1/sqrt(p) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + ...); the estimate
// leaves |e| ~ 2^-22, so the dropped terms (~e^3) are below FP64 rounding.
// On this GPU an FP64 divide or square root is a long dependent chain of
// FP64 operations; this is four (two Newton steps would be six), and it gives
// both the pivot sqrt(p) = p y and its reciprocal y.
__device__ __forceinline__ double rsqrt_cubic(double p) {
  const double y0 = (double)rsqrtf((float)p);
  const double e = fma(-(p * y0), y0, 1.0);
  return fma(y0 * e, fma(e, 0.375, 0.5), y0);
}

constexpr double kPivMin = 1e-10;
constexpr double kPivMinF32 = 1e-6;
constexpr double kNearIdErr = 2e-16;     // error allowed in L, elementwise (FP64 Gram matrices)
constexpr double kNearIdErrF32 = 1e-10;  // the same with FP32 Gram matrices (resolved to ~1e-7)

// Near-identity shortcut.  When the equilibrated Gram matrix is I + E with
// every off-diagonal |E_ij| <= e_b = sqrt(err / b) (err = kNearIdErr: about
// 1.4e-9 at b = 101, the columns already orthonormal to that level, as after
// a first CholeskyQR pass), its Cholesky factor is L = I + tril(E) and
// L^-1 = I - tril(E), each to within b e_b^2 = err elementwise
// (L L^T = I + E + tril(E) tril(E)^T), so S and B follow without a
// factorisation.  The pivots are then 1 to that accuracy;
// a live column whose scale is within a factor 1 + 1e-6 of the deflation
// threshold takes the full path, so both paths deflate the same columns.
// The test reads the lower triangle only, like the factorisation, and a
// non-finite entry sends the matrix to the full path.  It is split into
// `parts` shares by columns (column j in share j mod parts, a warp per
// column, lanes over its rows); every thread of the block calls it for the
// block's share `part`, and it returns 1 (a block-wide vote) when that share
// rules the shortcut out.
__device__ int near_identity_slow(int b, const double* __restrict__ G, const double* d,
                                  const double* dinv, const int* dead, double thr, double err,
                                  int part, int parts) {
  const double eb = sqrt(err / b);
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int slow = 0;
  for (int j = part + parts * (int)(threadIdx.x >> 5); j < b; j += parts * nw) {
    if (dead[j]) continue;
    if (lane == 0 && !(d[j] > thr * (1.0 + 1e-6))) slow = 1;
    for (int i = j + 1 + lane; i < b; i += 32)
      if (!dead[i] && !(fabs(G[i + (size_t)j * b]) * dinv[i] * dinv[j] <= eb)) slow = 1;
  }
  return __syncthreads_or(slow);
}

// S(c, j) = L^-1(j, c) / d_c and B(c, j) = L(j, c) d_j from the shortcut,
// for the elements e = first, first + stride, ... of the b x b outputs.
__device__ void near_identity_write(int b, const double* __restrict__ G, const double* d,
                                    const double* dinv, const int* dead, double* __restrict__ S,
                                    double* __restrict__ Bout, int first, int stride) {
  for (int e = first; e < b * b; e += stride) {
    const int c = e % b, j = e / b;
    double sv = 0.0, bv = 0.0;
    if (j >= c && !dead[c]) {
      if (j == c) {
        sv = dinv[c];
        bv = d[c];
      } else if (!dead[j]) {
        const double f = G[j + (size_t)c * b] * dinv[j] * dinv[c];  // E(j, c), lower triangle
        sv = -f * dinv[c];
        bv = f * d[j];
      }
    }
    S[e] = sv;
    Bout[e] = bv;
  }
}

// One CTA: equilibrated Cholesky of G (b x b, ld b) with deflation, then
// S = D^-1 L^-T (upper, X = R S) and B = L^T D (upper, R = X B).
// work: 2 b^2 doubles (shared or global).
__global__ void __launch_bounds__(1024)
chol_equil_kernel(int b, const double* __restrict__ G, const double* __restrict__ scale_ptr,
                  double tol, double pivmin, double near_err, double* __restrict__ S,
                  double* __restrict__ Bout, double* gwork, int use_smem) {
  extern __shared__ double smem[];
  double* L = use_smem ? smem : gwork;          // b x b, ld b (lower used)
  double* Li = L + (size_t)b * b;               // inverse of L
  __shared__ double d[1024 + 1];                // column scales (b <= 1024)
  __shared__ double dinv[1024 + 1];             // 1 / d, then 1 / L_jj
  __shared__ int dead[1024 + 1];
  __shared__ double piv_sh, rpiv_sh;
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
  if (!near_identity_slow(b, G, d, dinv, dead, thr, near_err, 0, 1)) {
    near_identity_write(b, G, d, dinv, dead, S, Bout, tid, nt);
    return;
  }
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
      bool dj = dead[j] != 0 || !(p > pivmin);
      double y = 1.0;
      if (!dj) {
        y = rsqrt_cubic(p);
        if (!(d[j] * (p * y) > thr)) dj = true;
      }
      dead[j] = dj ? 1 : 0;
      piv_sh = dj ? 1.0 : p * y;
      rpiv_sh = dj ? 1.0 : y;
    }
    __syncthreads();
    const double lj = piv_sh;
    const double rlj = rpiv_sh;
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
  // Li = L^-1 (lower) by forward substitution, one warp per column: the lanes
  // split each dot product and reduce by shuffles (the column's entries depend
  // on each other in order, so parallelism is across and within columns).
  for (int i = tid; i < b; i += nt) dinv[i] = 1.0 / L[i + (size_t)i * b];
  __syncthreads();
  {
    const int lane = tid % 32, warp = tid / 32, nwarps = nt / 32;
    for (int c = warp; c < b; c += nwarps) {
      double* lic = Li + (size_t)c * b;
      for (int i = lane; i < c; i += 32) lic[i] = 0.0;
      if (lane == 0) lic[c] = dinv[c];
      __syncwarp();
      for (int i = c + 1; i < b; ++i) {
        double acc = 0.0;
        for (int k = c + lane; k < i; k += 32) acc = fma(L[i + (size_t)k * b], lic[k], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) lic[i] = -acc * dinv[i];
        __syncwarp();
      }
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

// ---------------------------------------------------------------------------
// The same factorisation spread over a cluster of kCC CTAs (b <= kCMaxB).
// One SM retires about two FP64 FMAs per clock, so the one-CTA kernel above
// is bound by a single SM's FP64 pipe; here the equilibrated matrix is cut
// into 16 x 16 tiles, owned round-robin by the CTAs of the cluster and read
// across CTAs through distributed shared memory.  Tile step jt:
//   (1) the owner of tile (jt, jt) factors it (pivot and deflation rules as
//       above), (2) cluster barrier, (3) the owners of tiles (it, jt), it > jt,
//       solve L_it,jt L_jt,jt^T = A_it,jt (dead columns set to zero),
//   (4) cluster barrier, (5) every CTA subtracts L_it,jt L_kt,jt^T from its
//       tiles (it, kt), it >= kt > jt.
// Then every CTA gathers the factor (packed lower triangle) and its warps
// compute the columns of L^-1 by forward substitution, writing rows of S and B.
constexpr int kCT = 16;      // tile size
constexpr int kCC = 8;       // CTAs per cluster (portable cluster size)
constexpr int kCMaxB = 192;  // largest b on this path (shared memory bound)
constexpr int kCThreads = 256;

struct CholLayout {  // offsets in doubles, identical in every CTA of the cluster
  int nt, ntiles, tiles_per_cta;
  size_t off_tiles, off_big, off_ld, off_xs, off_d, off_dinv, off_dl, off_dead, total;
  __host__ __device__ explicit CholLayout(int b) {
    nt = (b + kCT - 1) / kCT;
    ntiles = nt * (nt + 1) / 2;
    tiles_per_cta = (ntiles + kCC - 1) / kCC;
    const size_t big_panel = (size_t)nt * kCT * kCT;        // column of tiles
    const size_t big_packed = (size_t)b * (b + 1) / 2;      // packed lower triangle
    off_tiles = 0;
    off_big = off_tiles + (size_t)tiles_per_cta * kCT * kCT;
    off_ld = off_big + (big_panel > big_packed ? big_panel : big_packed);
    off_xs = off_ld + kCT * kCT;
    off_d = off_xs + (size_t)(kCThreads / 32) * b;
    off_dinv = off_d + nt * kCT;
    off_dl = off_dinv + nt * kCT;
    off_dead = off_dl + nt * kCT;  // ints, nt * kCT of them
    total = off_dead + (nt * kCT + 1) / 2;
  }
};

__device__ inline void tile_of_lin(int lin, int& it, int& jt) {
  it = (int)((sqrtf(8.0f * lin + 1.0f) - 1.0f) * 0.5f);
  while (it * (it + 1) / 2 > lin) --it;
  while ((it + 1) * (it + 2) / 2 <= lin) ++it;
  jt = lin - it * (it + 1) / 2;
}

__global__ void __cluster_dims__(kCC, 1, 1) __launch_bounds__(kCThreads)
chol_cluster_kernel(int b, const double* __restrict__ G, const double* __restrict__ scale_ptr,
                    double tol, double pivmin, double near_err, double* __restrict__ S,
                    double* __restrict__ Bout) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double smem[];
  const CholLayout lay(b);
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  double* tiles = smem + lay.off_tiles;
  double* big = smem + lay.off_big;   // panel copy during the factorisation, packed L after
  double* Ld = smem + lay.off_ld;     // copy of the diagonal tile of the step
  double* xs = smem + lay.off_xs;     // one column of L^-1 per warp
  double* d = smem + lay.off_d;
  double* dinv = smem + lay.off_dinv;
  double* dl = smem + lay.off_dl;     // 1 / L_jj
  int* dead = reinterpret_cast<int*>(smem + lay.off_dead);
  __shared__ double piv_sh, rpiv_sh;
  __shared__ double rdg[kCT];  // reciprocals of the diagonal of the step's tile
  __shared__ int votes_sh[kCC];  // the CTAs' near-identity votes
  // arrive at a cluster barrier now and wait for it before the first access
  // to another CTA's shared memory (the votes below): by then every CTA runs
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  const int nt = lay.nt;
  const double thr = tol * (*scale_ptr);
  auto owner = [](int it, int jt) { return (it * (it + 1) / 2 + jt) % kCC; };
  auto slot = [&](int it, int jt) { return tiles + (size_t)((it * (it + 1) / 2 + jt) / kCC) * 256; };

  for (int j = tid; j < nt * kCT; j += kCThreads) {
    double dj = 0.0;
    bool dz = true;
    if (j < b) {
      const double g = G[j + (size_t)j * b];
      dj = g > 0.0 ? sqrt(g) : 0.0;
      dz = !(dj > thr);
    }
    dead[j] = dz ? 1 : 0;
    d[j] = dz ? 1.0 : dj;
    dinv[j] = dz ? 1.0 : 1.0 / dj;
    const double t = thr / (dz ? 1.0 : dj);
    dl[j] = t * t;  // the pivot threshold until the factor is complete
  }
  __syncthreads();
  // the near-identity test, an eighth of the columns per CTA: every CTA
  // writes its vote into every CTA (once all have started), and after the
  // barrier all decide alike from their own copies; nothing is read from
  // another CTA's shared memory, so all may leave here
  {
    const int slow = near_identity_slow(b, G, d, dinv, dead, thr, near_err, rank, kCC);
    // every CTA of the cluster has started (the arrival at the top) before
    // any writes into another's shared memory
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    if (tid < kCC) cl.map_shared_rank(votes_sh, tid)[rank] = slow;
    cl.sync();
    int any = 0;
#pragma unroll
    for (int r = 0; r < kCC; ++r) any |= votes_sh[r];
    if (!any) {
      near_identity_write(b, G, d, dinv, dead, S, Bout, rank * kCThreads + tid, kCC * kCThreads);
      return;
    }
  }
  // my tiles of the equilibrated lower triangle; padding rows and columns
  // (index >= b) are identity, dead columns unit vectors
  for (int lin = rank; lin < lay.ntiles; lin += kCC) {
    int it, jt;
    tile_of_lin(lin, it, jt);
    double* T = tiles + (size_t)(lin / kCC) * 256;
    for (int e = tid; e < 256; e += kCThreads) {
      const int i = it * kCT + e % kCT, j = jt * kCT + e / kCT;
      double v = 0.0;
      if (i >= j) {
        if (i >= b || j >= b || dead[i] || dead[j]) v = (i == j) ? 1.0 : 0.0;
        else v = G[i + (size_t)j * b] * dinv[i] * dinv[j];
      }
      T[e] = v;
    }
  }
  __syncthreads();

  for (int jt = 0; jt < nt; ++jt) {
    // (1) factor the diagonal tile (the owner's 256 threads, one element each)
    if (rank == owner(jt, jt)) {
      double* T = slot(jt, jt);
      const int r = tid % kCT, k = tid / kCT;  // element (r, k) of the tile
      for (int c = 0; c < kCT; ++c) {
        const int j = jt * kCT + c;
        if (tid == 0) {
          const double p = T[c + kCT * c];
          // deflation d_j sqrt(p) <= thr tested as p <= (thr / d_j)^2, off the chain
          const bool dj = dead[j] != 0 || !(p > pivmin) || !(p > dl[j]);
          const double y = dj ? 1.0 : rsqrt_cubic(p);
          dead[j] = dj ? 1 : 0;
          piv_sh = dj ? 1.0 : p * y;
          rpiv_sh = dj ? 1.0 : y;
          T[c + kCT * c] = piv_sh;
        }
        __syncthreads();
        const bool dj = dead[j] != 0;
        if (k == c && r > c) T[r + kCT * c] = dj ? 0.0 : T[r + kCT * c] * rpiv_sh;
        __syncthreads();
        if (!dj && k > c && r >= k) T[r + kCT * k] -= T[r + kCT * c] * T[k + kCT * c];
        __syncthreads();
      }
    }
    cl.sync();  // (2)
    // (3) everyone copies the factored diagonal tile and its dead flags
    {
      const int o = owner(jt, jt);
      const double* rT = cl.map_shared_rank(slot(jt, jt), o);
      const int* rdead = cl.map_shared_rank(dead, o);
      for (int e = tid; e < 256; e += kCThreads) Ld[e] = rT[e];
      if (tid < kCT) {
        dead[jt * kCT + tid] = rdead[jt * kCT + tid];
        rdg[tid] = 1.0 / rT[tid + kCT * tid];  // 16 divisions side by side, none in the solve
      }
    }
    __syncthreads();
    for (int it = jt + 1 + tid / kCT; it < nt; it += kCThreads / kCT) {
      if (owner(it, jt) != rank) continue;
      double* T = slot(it, jt);
      const int r = tid % kCT;
      double x[kCT];
#pragma unroll
      for (int c = 0; c < kCT; ++c) {
        double acc = T[r + kCT * c];
#pragma unroll
        for (int k = 0; k < c; ++k) acc = fma(-x[k], Ld[c + kCT * k], acc);
        x[c] = dead[jt * kCT + c] ? 0.0 : acc * rdg[c];
      }
#pragma unroll
      for (int c = 0; c < kCT; ++c) T[r + kCT * c] = x[c];
    }
    cl.sync();  // (4)
    // (5) copy the factored column of tiles, update my trailing tiles
    for (int e = tid; e < (nt - jt - 1) * 256; e += kCThreads) {
      const int it = jt + 1 + e / 256;
      big[(size_t)it * 256 + e % 256] = cl.map_shared_rank(slot(it, jt), owner(it, jt))[e % 256];
    }
    __syncthreads();
    for (int lin = rank; lin < lay.ntiles; lin += kCC) {
      int it, kt;
      tile_of_lin(lin, it, kt);
      if (kt <= jt) continue;
      double* T = tiles + (size_t)(lin / kCC) * 256;
      const double* Pi = big + (size_t)it * 256;
      const double* Pk = big + (size_t)kt * 256;
      for (int e = tid; e < 256; e += kCThreads) {
        const int r = e % kCT, k = e / kCT;
        if (it == kt && r < k) continue;
        double acc = T[e];
#pragma unroll
        for (int c = 0; c < kCT; ++c) acc = fma(-Pi[r + kCT * c], Pk[k + kCT * c], acc);
        T[e] = acc;
      }
    }
    __syncthreads();
  }
  // gather the whole factor, packed by columns: (i, j) at j b - j (j - 1) / 2 + i - j
  cl.sync();
  for (int e = tid; e < lay.ntiles * 256; e += kCThreads) {
    const int lin = e / 256, rc = e % 256;
    int it, jt;
    tile_of_lin(lin, it, jt);
    const int i = it * kCT + rc % kCT, j = jt * kCT + rc / kCT;
    if (i < j || i >= b || j >= b) continue;
    const double* rT = cl.map_shared_rank(tiles + (size_t)(lin / kCC) * 256, lin % kCC);
    big[(size_t)j * b - (size_t)j * (j - 1) / 2 + (i - j)] = rT[rc];
  }
  cl.sync();  // no CTA reads another's shared memory after this point
  for (int j = tid; j < b; j += kCThreads) dl[j] = 1.0 / big[(size_t)j * b - (size_t)j * (j - 1) / 2];
  __syncthreads();
  // columns of L^-1, one warp each; S(c, j) = Li(j, c) / d_c, B(c, j) = L(j, c) d_j
  double* x = xs + (size_t)warp * b;
  for (int c = rank * (kCThreads / 32) + warp; c < b; c += kCC * (kCThreads / 32)) {
    for (int i = c + lane; i < b; i += 32) x[i] = (i == c) ? 1.0 : 0.0;
    __syncwarp();
    for (int k = c; k < b; ++k) {
      const double xk = x[k] * dl[k];
      const double* Lk = big + (size_t)k * b - (size_t)k * (k - 1) / 2 - k;  // Lk[i] = L(i, k)
      __syncwarp();
      if (lane == 0) x[k] = xk;
      for (int i = k + 1 + lane; i < b; i += 32) x[i] = fma(-Lk[i], xk, x[i]);
      __syncwarp();
    }
    const bool dc = dead[c] != 0;
    const double* Lc = big + (size_t)c * b - (size_t)c * (c - 1) / 2 - c;
    for (int j = lane; j < b; j += 32) {
      double sv = 0.0, bv = 0.0;
      if (j >= c && !dc) {
        if (!dead[j]) sv = x[j] * dinv[c];
        if (!dead[j] || c < j) bv = Lc[j] * d[j];
      }
      S[c + (size_t)j * b] = sv;
      Bout[c + (size_t)j * b] = bv;
    }
    __syncwarp();
  }
}

blws_status chol_equil(Ctx* ctx, cudaStream_t s, int b, const double* G, const double* scale,
                       double tol, double pivmin, double near_err, double* S, double* B, double* gwork) {
  if (b > 1024) return ctx->fail(BLWS_EINVAL, "block width %d exceeds 1024", b);
  if (b <= kCMaxB) {
    const size_t bytes = CholLayout(b).total * sizeof(double);
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_CHOL_CLUSTER, (const void*)chol_cluster_kernel, (int)bytes));
    chol_cluster_kernel<<<kCC, kCThreads, bytes, s>>>(b, G, scale, tol, pivmin, near_err, S, B);
    BLWS_CHECK_LAUNCH(ctx);
    return BLWS_OK;
  }
  const size_t need = 2ull * b * b * sizeof(double);
  const int use_smem = need <= 200 * 1024 ? 1 : 0;
  if (use_smem) {
    BLWS_TRY(ctx->smem_limit(Ctx::ATTR_CHOL, (const void*)chol_equil_kernel, (int)need));
  }
  chol_equil_kernel<<<1, 1024, use_smem ? need : 0, s>>>(b, G, scale, tol, pivmin, near_err, S, B,
                                                          gwork, use_smem);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

}  // namespace

blws_status chol_qr2(Ctx* ctx, cudaStream_t s, int N, int b, double* R, int ld, double* X,
                     double* tmp, double* B, const double* scale, double tol, bool fp32, bool one_pass) {
  // small scratch: G, S, B1, B2, work (2 b^2)
  double* sm = nullptr;
  BLWS_TRY(ctx->get(BUF_SMALL, 6ull * b * b, &sm));
  double* G = sm;
  double* S = G + (size_t)b * b;
  double* B1 = S + (size_t)b * b;
  double* B2 = B1 + (size_t)b * b;
  double* work = B2 + (size_t)b * b;
  // pass 1
  BLWS_TRY(gemm(ctx, s, true, false, b, b, N, 1.0, R, ld, R, ld, 0.0, G, b, fp32));
  // with FP32 Gram matrices a pivot is only resolved down to ~1e-6
  const double pivmin = fp32 ? kPivMinF32 : kPivMin;
  const double near_err = fp32 ? kNearIdErrF32 : kNearIdErr;
  BLWS_TRY(chol_equil(ctx, s, b, G, scale, tol, pivmin, near_err, S, B1, work));
  if (one_pass) {
    BLWS_TRY(gemm(ctx, s, false, false, N, b, b, 1.0, R, ld, S, b, 0.0, X, ld, fp32));
    BLWS_TRY_CUDA(ctx, cudaMemcpyAsync(B, B1, sizeof(double) * b * b, cudaMemcpyDeviceToDevice, s));
    return BLWS_OK;
  }
  BLWS_TRY(gemm(ctx, s, false, false, N, b, b, 1.0, R, ld, S, b, 0.0, tmp, ld, fp32));
  // pass 2 (columns are now unit or zero: same deflation rule against 1)
  BLWS_TRY(gemm(ctx, s, true, false, b, b, N, 1.0, tmp, ld, tmp, ld, 0.0, G, b, fp32));
  double* one = nullptr;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &one));
  BLWS_TRY(chol_equil(ctx, s, b, G, one + SLOT_ONE, 0.5, pivmin, near_err, S, B2, work));
  BLWS_TRY(gemm(ctx, s, false, false, N, b, b, 1.0, tmp, ld, S, b, 0.0, X, ld, fp32));
  // B = B2 B1
  BLWS_TRY(gemm(ctx, s, false, false, b, b, b, 1.0, B2, b, B1, b, 0.0, B, b));
  return BLWS_OK;
}

}  // namespace blws
