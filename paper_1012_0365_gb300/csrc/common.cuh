// Shared internals of the BLWS library: context, named workspace buffers,
// error plumbing and the counter-based generator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/blws.h"

namespace blws {

// ---------------------------------------------------------------- errors --
#define BLWS_TRY_CUDA(ctx, expr)                                                 \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      return (ctx)->fail(e_ == cudaErrorMemoryAllocation ? BLWS_ENOMEM : BLWS_ECUDA, \
                         "%s:%d %s: %s", __FILE__, __LINE__, #expr,              \
                         cudaGetErrorString(e_));                                \
    }                                                                            \
  } while (0)

// every kernel launch is followed by this check, which also counts it
#define BLWS_CHECK_LAUNCH(ctx)             \
  do {                                     \
    ++(ctx)->launches;                     \
    BLWS_TRY_CUDA(ctx, cudaGetLastError()); \
  } while (0)

#define BLWS_TRY(expr)               \
  do {                               \
    blws_status s_ = (expr);         \
    if (s_ != BLWS_OK) return s_;    \
  } while (0)

// ------------------------------------------------------------- workspace --
// Named device buffers owned by the context, each grown on demand.  Growth
// frees the old buffer after the work that may still use it has finished (the
// whole device, or only the context's own stream when it has one), so it
// happens outside steady state: a solver sizes its buffers once before its
// first iteration.
enum Buf {
  BUF_Q = 0,     // Lanczos basis Q_k, (m+n) x (k b)
  BUF_P,         // W~ X_l / residual R_l, (m+n) x b
  BUF_P2,        // CholeskyQR intermediate, (m+n) x b
  BUF_T,         // T_k and its eigenvectors, (k b)^2 each (several)
  BUF_SMALL,     // b x b scratch matrices and vectors
  BUF_SPLITK,    // split-K partial sums of the GEMMs
  BUF_EIG,       // eigen-solver scratch
  BUF_EIG2,      // eigen-solver second level (clusters)
  BUF_SCAL,      // device scalars (Slot)
  BUF_WARM_U,    // solver-held warm start U (m x b)
  BUF_WARM_V,    // solver-held warm start V (n x b)
  BUF_SIG,       // Ritz values
  BUF_Y,         // RPCA multiplier Y (m x n)
  BUF_W,         // RPCA SVT input W (m x n)
  BUF_E2,        // RPCA second E buffer (m x n)
  BUF_RED,       // reduction partials
  BUF_CSC_PTR,   // MC: CSC column pointers
  BUF_CSC_ROW,   // MC: CSC row indices
  BUF_CSC_PERM,  // MC: CSR position of each CSC entry
  BUF_MC_Y,      // MC: values of the sparse iterate on Omega (CSR order)
  BUF_MC_X,      // MC: low-rank factors of the current X (PROX)
  BUF_TC_W,      // mixed precision: TF32 planes of W (two orientations, hi and lo)
  BUF_TC_X,      // mixed precision: TF32 planes of the block X
  BUF_TC_PART,   // mixed precision: split-K partial sums (FP32)
  BUF_OZ_E,      // FP64-equivalent tensor-core products: scale exponents
  BUF_TRI,       // eigen-solver: tridiagonal-route scratch (FP32)
  BUF_EIG_GRP,   // eigen-solver: sorted group ids of the tridiagonal route
  BUF_OZ_G,      // FP64-equivalent general products: digit planes of both operands
  BUF_RPCA_A,    // RPCA, FP64-equivalent and mixed modes: A = U diag(theta) V^T as a product (m x n)
  BUF_TC_G,      // mixed precision: TF32 planes of both operands of a general product
  BUF_TUNE,      // GEMM autotuner: scratch operands of the shape being timed
  BUF_GUARD,     // Ritz-residual guard: Gram matrix of the last block residual, and R^T R Z
  BUF_COUNT_
};

// A CUDA graph of one solver phase, replayed while the phase's launches are
// unchanged (the key lists everything the launches depend on).
struct TimedPair {
  cudaEvent_t e0, e1;
  double work;
  int kind;  // 0 FP64 DFMA, 1 split TF32, 2 digit planes
};
struct GraphEntry {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  unsigned long long nlaunch = 0;   // kernels in the graph
  std::vector<TimedPair> ev;        // timed products inside it (timing on)
  unsigned long long last_use = 0;
};

struct Ctx {
  blws_config cfg;
  int device = 0;
  int sms = 0;
  size_t smem_optin = 0;
  void* buf[BUF_COUNT_] = {nullptr};
  size_t cap[BUF_COUNT_] = {0};
  double* host_pinned = nullptr;  // small pinned staging area for scalars
  // set when every call on this context uses this one stream (a server
  // worker): buffer growth then waits for that stream instead of the device
  cudaStream_t sole_stream = nullptr;
  unsigned long long launches = 0; // kernels launched through this context
  char last_error[512] = {0};

  blws_status fail(blws_status code, const char* fmt, ...);
  // device buffer `b` with at least `bytes` bytes (grown on demand)
  blws_status get(Buf b, size_t bytes, void** out);
  // free every workspace buffer but the scalar slots (the next call
  // allocates again what it needs)
  blws_status trim();
  // dynamic shared memory limit of a kernel.  The attribute belongs to the
  // kernel (process-wide, per device), not to a context: it only ever grows,
  // under a lock, so that contexts on other threads never lower it under a
  // launch that needs more (defined in capi.cu).
  enum SmemAttr { ATTR_CHOL, ATTR_CHOL_CLUSTER, ATTR_JACOBI_CTA, ATTR_JACOBI_BLOCK, ATTR_TRI, ATTR_TRI_INV, ATTR_TRI_CL, ATTR_TRI_CL8, ATTR_OZ,
                  ATTR_TRI_ROWS1, ATTR_TRI_ROWS2, ATTR_TRI_ROWS4, ATTR_TRI_ROWS8, ATTR_COUNT_ };
  blws_status smem_limit(SmemAttr which, const void* func, int bytes);
  int jacobi_block_per_sm = 0;  // occupancy of the block Jacobi kernel (queried once)
  // FP32 eigen stage: 0 the tridiagonal route where it applies, 1 Jacobi only
  // (environment BLWS_EIG=jacobi at context creation)
  int eig_route = 0;
  // timing of the product with the augmented matrix (step a2), on request
  // (blws_timing_start / blws_timing_stop): a pair of events around the
  // kernel(s) of each product, and the work m n b it did
  bool timing = false;
  cudaEvent_t* tev = nullptr;   // 2 * tcap events
  double* tw = nullptr;         // work of each timed product (tcap)
  int* tk = nullptr;            // its kernel kind (tcap)
  size_t tcap = 0, tused = 0;
  double twork = 0.0;
  double* trec_ms = nullptr;    // per-product times of the last blws_timing_stop
  double* trec_w = nullptr;
  int* trec_k = nullptr;
  size_t trec_n = 0;
  // events around one product's kernels (no-ops unless timing is on)
  blws_status time_begin(cudaStream_t s);
  blws_status time_end(cudaStream_t s, double work, int kind);
  // a mixed-precision solve in its refinement tail: FP64 products go to the
  // FP64-equivalent digit-plane kernels as in a BLWS_PREC_FP64_TC context
  bool oz_tail = false;
  // tridiagonal reduction: 0 by rows on a cluster where it fits, 1 the packed
  // kernels (environment BLWS_TRI=packed at context creation)
  int tri_route = 0;
  // ---- CUDA graphs of the outer-iteration phases (graph.cu) ----
  // replay on (blws_config.graphs, environment BLWS_GRAPH=0 turns it off)
  bool graphs_on = false;
  // a phase is being captured: workspace growth is refused (it would have to
  // synchronise) and breaks the capture, which then runs directly
  bool capturing = false;
  bool capture_broken = false;
  // bumped whenever a workspace buffer moves: keys hold it, so a graph never
  // outlives the addresses it was captured with
  unsigned long long gen = 0;
  unsigned long long graph_clock = 0;
  unsigned long long graph_replays = 0, graph_captures = 0;
  std::vector<GraphEntry> graphs;
  std::vector<std::vector<uint64_t>> seen;  // keys met once (captured on the second meeting)
  cudaStream_t gstream = nullptr;          // stream the graphs run on
  cudaEvent_t gfork = nullptr, gjoin = nullptr;
  std::vector<TimedPair> cap_ev;           // timed products of the capture in progress
  std::vector<TimedPair> pending_ev;       // timed products of replays not yet read
  std::vector<double> graph_ms, graph_w;   // their times and work, once read
  std::vector<int> graph_kind;
  // pinned host copies of the eigen-solver's results for its host stage
  // (eigenvalues, group ids and tops, refinement width, failure flag)
  void* host_eig = nullptr;
  size_t host_eig_cap = 0;
  blws_status host_eig_get(size_t bytes);
  void free_graphs();
  unsigned long long tri_fallbacks = 0;  // tridiagonal stage results replaced by Jacobi
  // device bytes the workspace holds now
  size_t held_bytes() const {
    size_t t = 0;
    for (int b = 0; b < BUF_COUNT_; ++b) t += cap[b];
    return t;
  }
  template <typename T>
  blws_status get(Buf b, size_t count, T** out) {
    void* p = nullptr;
    blws_status s = get(b, count * sizeof(T), &p);
    *out = reinterpret_cast<T*>(p);
    return s;
  }
};

// Device-side scalar slots used by the procedure (one small array).
enum Slot {
  SLOT_SCALE = 0,      // deflation scale: largest column norm of W~ X_1
  SLOT_COUNT = 1,      // #{sigma > eps} (stored as double)
  SLOT_NORM = 2,       // generic reduction result
  SLOT_AUX = 3,
  SLOT_ONE = 4,        // constant 1.0 (set at context creation)
  SLOT_FLAG = 5,       // int flag (non-finite input seen)
  SLOT_NNZ = 6,        // unsigned long long counter
  SLOT_AUX2 = 7,
  SLOT_TCERR = 8,      // int: a tensor-core kernel's bounded wait ran out
  SLOT_TRIFAIL = 9,    // int: the tridiagonal route met a group it cannot orthonormalise
  SLOT_EPS = 10,       // per-iteration scalars read by the kernels of a replayed
  SLOT_MU = 11,        //   graph: threshold eps = 1 / mu, mu, and the next mu
  SLOT_MU_NEXT = 12,
  SLOT_GUARD = 13,     // largest Ritz residual of a pair above eps, relative to the top Ritz value
  SLOT_MAX = 16
};

// ------------------------------------------------------- launch helpers --
inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------- Philox4x32-10 (Salmon,
// Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
// a counter-based generator; each (counter, key) maps to four 32-bit words.
struct Philox {
  static constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  static constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  __host__ __device__ static inline void round(uint32_t c[4], uint32_t k[2]) {
    uint64_t p0 = (uint64_t)M0 * c[0];
    uint64_t p1 = (uint64_t)M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k[0] += W0; k[1] += W1;
  }
  __host__ __device__ static inline void gen(const uint32_t ctr[4], uint64_t key, uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
#pragma unroll
    for (int i = 0; i < 10; ++i) round(c, k);
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
  }
};

// Standard normal from the generator by the Box-Muller transform.
__device__ inline double philox_normal(uint64_t key, uint32_t a, uint32_t b, uint32_t c) {
  uint32_t ctr[4] = {a, b, c, 0x243F6A88u}, o[4];
  Philox::gen(ctr, key, o);
  const double inv = 1.0 / 4294967296.0;
  double u1 = ((double)o[0] + 1.0) * inv;  // (0, 1]
  double u2 = (double)o[1] * inv;          // [0, 1)
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

}  // namespace blws

struct blws_ctx : public blws::Ctx {};
