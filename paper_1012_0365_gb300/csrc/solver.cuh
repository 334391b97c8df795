// Host solvers built on the BLWS procedure.
#pragma once
#include "blws_core.cuh"

namespace blws {

// ||W||_2: block Lanczos (8 columns, up to 8 blocks) from a seeded block,
// restarted from its own Ritz vectors until the leading Ritz value is stable
// to `stable` relative; returns it on the host.  The hosts use it for their
// starting point only (RPCA: mu_0 and Y_0; MC: k_0 and the first tau), which
// the optimum they converge to does not depend on; 1e-10 is far below what
// a change of the start can show in their results.
blws_status spectral_norm(Ctx* ctx, cudaStream_t s, const Operator& op, double* out_host,
                          double stable = 1e-10);

blws_status rpca_run(Ctx* ctx, cudaStream_t s, const double* D, int m, int n, int ld,
                     const rpca_params& p, double* A, double* E, rpca_info* info);

blws_status mc_run(Ctx* ctx, cudaStream_t s, int m, int n, int nnz, const int* rowptr,
                   const int* colidx, const double* vals, const mc_params& p, int max_rank,
                   double* U, double* theta, double* V, mc_info* info);

}  // namespace blws
