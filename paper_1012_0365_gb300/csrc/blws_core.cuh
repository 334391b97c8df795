// The BLWS procedure and the operator it is applied to.
#pragma once
#include "ops.cuh"

namespace blws {

// W (m x n): dense FP64 column-major, or CSR (+ CSC mirror) plus an optional
// low-rank term Ul diag(sl) Vl^T.  sym: W is a dense symmetric m x m matrix
// and the procedure runs on W itself (BL_EVD, Algorithm 3) instead of the
// augmented matrix; n is unused.
struct Operator {
  int m = 0, n = 0;
  bool sym = false;
  const double* W = nullptr;
  int ldw = 0;
  // sparse part
  int nnz = 0;
  const int* rowptr = nullptr;
  const int* colidx = nullptr;
  const double* val = nullptr;
  const int* colptr = nullptr;  // CSC mirror of the pattern
  const int* rowidx = nullptr;
  const int* perm = nullptr;    // CSC entry e is CSR entry perm[e]
  // mixed precision: TF32 planes of the dense W (row-major Wr: m rows,
  // column-major Wc: n rows); when set, products with W run on tensor cores
  const TcPlanes* Wr = nullptr;
  const TcPlanes* Wc = nullptr;
  // FP64-equivalent tensor-core products: digit planes of W (both orientations)
  const OzPlanes* Or = nullptr;
  const OzPlanes* Oc = nullptr;
  // low-rank part
  int rl = 0;
  const double* Ul = nullptr;
  const double* sl = nullptr;
  const double* Vl = nullptr;
};

struct BlwsArgs {
  double eps = 0.0;
  int r = 1;                 // Ritz pairs to output
  const double* U0 = nullptr;
  int ldu0 = 0;
  const double* V0 = nullptr;
  int ldv0 = 0;
  int w = 0;                 // warm columns
  const double* G = nullptr;  // extra start columns ((m+n) x g)
  int ldg = 0;
  int g = 0;
  int k = 3;                 // blocks
  bool cold = false;         // full reorthogonalisation (no previous subspace)
  uint32_t draw = 0;         // generator stream of the extra columns (per call)
  bool mixed = false;        // tall products in FP32 arithmetic (eigen-solver and
                             // Cholesky factorisations stay FP64)
  bool standard = false;     // warm columns [U0; 0] instead of [U0; V0] / sqrt(2)
  // Ritz-residual guard: stage (a) also forms the residual of the last block
  // and writes the largest ||W~ y - theta y|| / theta_1 over the pairs above
  // the threshold (read from eps_dev, device) to the pinned host copy the
  // eigen-solver's host stage reads (blws_guard_ratio)
  bool guard = false;
  const double* eps_dev = nullptr;
  // second projection of every residual against all earlier blocks, as on a
  // cold start (a call repeated by the guard with more blocks: the local
  // recurrence loses orthogonality to converged directions as k grows)
  bool reorth = false;
  // U0, V0 are the previous call's Ritz vectors (the solvers' own warm
  // starts, orthonormal to rounding): the start block takes one CholeskyQR
  // pass instead of two when it has no other columns (callers' warm starts
  // are orthonormalised in full)
  bool ritz_warm = false;
};

// the guard's ratio of the last stage (a) with a.guard, once s is synchronised
double blws_guard_ratio(Ctx* ctx, const BlwsArgs& a);

// P = W~ X: P[0:m] = W X[m:m+n], P[m:m+n] = W^T X[0:m]  (sym: P = W X, m rows)
blws_status apply_op(Ctx* ctx, cudaStream_t s, const Operator& op, const double* X, int ldx, int b,
                     double* P, int ldp);
blws_status apply_sparse(Ctx* ctx, cudaStream_t s, const Operator& op, const double* X, int ldx,
                         int b, double* P, int ldp);

// Size every workspace buffer one BLWS call of width <= bmax, <= kmax blocks needs.
blws_status blws_reserve(Ctx* ctx, int m, int n, int bmax, int kmax);

// One BLWS evaluation: writes U (m x r), V (n x r), sigma (r) and the count
// #{sigma > eps} to count_dev (device int).  With op.sym: U (m x r) holds the
// Ritz vectors of W itself, sigma its r largest Ritz values, V is not written.
blws_status blws_run(Ctx* ctx, cudaStream_t s, const Operator& op, const BlwsArgs& a, double* U,
                     int ldu, double* V, int ldv, double* sigma, int* count_dev);
// blws_run in three stages around its one synchronisation: (a) the start
// block, the k block steps and the device stage of the EVD of T_k; then, with
// s synchronised, (mid) the EVD's host stage; then (b) the Ritz lift and the
// count.  Stages a and b never wait on the host, so each can be captured in a
// CUDA graph; eps_dev (nullable) supplies the threshold of the count from
// device memory instead of a.eps.
blws_status blws_run_a(Ctx* ctx, cudaStream_t s, const Operator& op, const BlwsArgs& a);
blws_status blws_run_mid(Ctx* ctx, cudaStream_t s, const Operator& op, const BlwsArgs& a);
blws_status blws_run_b(Ctx* ctx, cudaStream_t s, const Operator& op, const BlwsArgs& a, double* U,
                       int ldu, double* V, int ldv, double* sigma, int* count_dev,
                       const double* eps_dev);

}  // namespace blws
