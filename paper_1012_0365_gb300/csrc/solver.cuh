// Host solvers built on the BLWS procedure.
#pragma once
#include "blws_core.cuh"

namespace blws {

// ||W||_2: block Lanczos (8 columns, up to 8 blocks) from a seeded block,
// restarted from its own Ritz vectors until the leading Ritz value is stable
// to `stable` relative (1e-14 with FP64 products, 1e-13 with the digit-plane
// ones); returns it on the host.
blws_status spectral_norm(Ctx* ctx, cudaStream_t s, const Operator& op, double* out_host,
                          double stable = 1e-14);

blws_status rpca_run(Ctx* ctx, cudaStream_t s, const double* D, int m, int n, int ld,
                     const rpca_params& p, double* A, double* E, rpca_info* info);

blws_status mc_run(Ctx* ctx, cudaStream_t s, int m, int n, int nnz, const int* rowptr,
                   const int* colidx, const double* vals, const mc_params& p, int max_rank,
                   double* U, double* theta, double* V, mc_info* info);

}  // namespace blws
