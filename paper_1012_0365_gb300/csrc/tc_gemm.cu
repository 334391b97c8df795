// Block products with the augmented matrix on the 5th-generation tensor cores
// (tcgen05), for the mixed-precision mode: P = [W X_v; W^T X_u] (Section 4,
// the product with W~ that skips its zero blocks) with split TF32 operands.
//
// Each operand x is carried as two TF32 planes, x ~ hi + lo (hi = tf32(x),
// lo = tf32(x - hi)), and each product is formed from three tensor-core
// products, A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 in tensor
// memory (the A_lo B_lo term is below the FP32 rounding of the sum).  The
// split-K partial sums are reduced in FP64 in a fixed order.
//
// Operands are K-major FP32 planes: element (r, k) of a plane at r * ld + k,
// ld a multiple of 32 floats.  W is therefore kept in two orientations (row
// major for W X_v, column major for W^T X_u) so that both products read their
// A operand along K.  One CTA (128 threads) owns a 128-row tile of one
// product and one K range:
//   warp 0, one thread:  TMA loads of the four operand tiles of a K block
//                        (128B swizzle) into a STAGES-deep ring;
//   warp 1, one thread:  12 tcgen05.mma per K block (4 K steps x 3 terms);
//   warp 2:              allocates and frees the tensor-memory accumulator;
//   all four warps:      read the 128 x NPAD accumulator back (tcgen05.ld,
//                        lane = row) and store the FP32 partial sums.
// Every mbarrier wait is bounded; a wait that runs out sets an error word
// and the CTA skips the rest of its work, frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ops.cuh"
#include "tc_ptx.cuh"

namespace blws {

namespace {

using namespace tc;

constexpr int kTcBM = 128;      // accumulator rows (tensor-memory lanes)
constexpr int kTcBK = 32;       // K block: 32 FP32 = one 128-byte swizzle row
constexpr int kTcThreads = 128;
constexpr int kTcMaxChunk = 256;  // K terms summed in FP32 inside the tensor core

struct TcJob {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;  // 64-byte aligned (CUtensorMap is)
  float* part;                         // [splits][NPAD][Mpad] partial sums (column-major)
  int M, K, tiles, splits, kchunk, Mpad;
};

struct TcJobs {
  TcJob job[2];
  int blocks0;  // CTAs of job 0; the rest belong to job 1
  int N;        // columns of the products (b)
  int* err;     // error word (nonzero: a wait ran out)
};

template <int NPAD>
__host__ __device__ constexpr int tmem_cols() {
  return NPAD <= 32 ? 32 : NPAD <= 64 ? 64 : NPAD <= 128 ? 128 : 256;
}

template <int NPAD, int STAGES>
__host__ __device__ constexpr size_t tc_smem_bytes() {
  return (size_t)STAGES * (2 * kTcBM * kTcBK * 4 + 2 * NPAD * kTcBK * 4) + 1024;
}

// ----------------------------------------------------------------- kernel --
template <int NPAD, int STAGES>
__global__ void __launch_bounds__(kTcThreads, 1) tc_tf32x3_kernel(const __grid_constant__ TcJobs jobs) {
  constexpr int A_BYTES = kTcBM * kTcBK * 4;
  constexpr int B_BYTES = NPAD * kTcBK * 4;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t NCOLS = tmem_cols<NPAD>();
  static_assert(NPAD % 16 == 0 && NPAD >= 16 && NPAD <= 256, "N of the MMA");
  static_assert(STAGE % 1024 == 0, "stage buffers keep the 1024-byte swizzle alignment");
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fail_sh;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int jb = (int)blockIdx.x < jobs.blocks0 ? 0 : 1;
  const TcJob& J = jobs.job[jb];
  const int local = jb ? (int)blockIdx.x - jobs.blocks0 : (int)blockIdx.x;
  const int tile = local % J.tiles, split = local / J.tiles;
  const int row0 = tile * kTcBM;
  const int kbeg = split * J.kchunk;
  const int kend = min(J.K, kbeg + J.kchunk);
  const int nk = (kend - kbeg + kTcBK - 1) / kTcBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    fail_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // producer: four TMA tiles per K block
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t round = (uint32_t)(kb / STAGES);
      if (kb >= STAGES && !mbar_wait(&empty_bar[s], (round & 1u) ^ 1u)) {
        fail_sh = 1;
        break;
      }
      uint8_t* st = smem + (size_t)s * STAGE;
      mbar_expect_tx(&full_bar[s], STAGE);
      const int kx = kbeg + kb * kTcBK;
      tma_load_2d(st, &J.a_hi, kx, row0, &full_bar[s]);
      tma_load_2d(st + A_BYTES, &J.a_lo, kx, row0, &full_bar[s]);
      tma_load_2d(st + 2 * A_BYTES, &J.b_hi, kx, 0, &full_bar[s]);
      tma_load_2d(st + 2 * A_BYTES + B_BYTES, &J.b_lo, kx, 0, &full_bar[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 K steps of 8 TF32 (32 bytes) x 3 terms per K block
    constexpr uint32_t idesc = tf32_idesc(kTcBM, NPAD);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t round = (uint32_t)(kb / STAGES);
      if (!mbar_wait(&full_bar[s], round & 1u)) {
        fail_sh = 1;
        break;
      }
      tc_fence_after();
      const uint32_t st = smem_u32(smem + (size_t)s * STAGE);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 8; ++kk) {
        const uint32_t off = kk * 32;
        const uint64_t a_hi = sw128_desc(st + off);
        const uint64_t a_lo = sw128_desc(st + A_BYTES + off);
        const uint64_t b_hi = sw128_desc(st + 2 * A_BYTES + off);
        const uint64_t b_lo = sw128_desc(st + 2 * A_BYTES + B_BYTES + off);
        mma_tf32(tbase, a_hi, b_hi, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tbase, a_hi, b_lo, idesc, 1u);
        mma_tf32(tbase, a_lo, b_hi, idesc, 1u);
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&done_bar);  // arrives once every MMA issued above has completed
  }
  __syncwarp();

  // epilogue: accumulator row = tensor-memory lane = thread
  const bool got = mbar_wait(&done_bar, 0);
  tc_fence_after();
  if (got && !fail_sh) {
    const int row = row0 + warp * 32 + lane;
    float* out = J.part + (size_t)split * NPAD * J.Mpad;
#pragma unroll 1
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < J.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < jobs.N) out[(size_t)(c0 + j) * J.Mpad + row] = v[j];
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(jobs.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS)
                 : "memory");
  }
}

// P(r, j) = sum over splits of the partial sums (FP64, split order)
__global__ void tc_reduce(int M, int N, int npad, int splits, int Mpad, const float* __restrict__ part,
                          double* __restrict__ P, int ldp) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % M), j = (int)(e / M);
    double acc = 0.0;
    for (int z = 0; z < splits; ++z) acc += (double)part[((size_t)z * npad + j) * Mpad + r];
    P[r + (size_t)j * ldp] = acc;
  }
}

// C = alpha (sum over splits) + beta C for a general product, each output
// summed by a group of G lanes (lane q adds splits q, q + G, ... in order, then
// a fixed shuffle tree); sym (M = N, beta = 0): an element below the diagonal
// is formed from its mirror's partials, so C is exactly symmetric
__global__ void tc_reduce_ab(int M, int N, int npad, int splits, int Mpad, const float* __restrict__ part,
                             double alpha, double beta, double* C, int ldc, int sym, int G) {
  const size_t total = (size_t)M * N;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t nth = (size_t)gridDim.x * blockDim.x;
  const int q = (int)(tid % G);
  const size_t span = (total * G + nth - 1) / nth * nth;  // the same trip count in every lane
  for (size_t t = tid; t < span; t += nth) {
    const size_t e = t / G;
    double acc = 0.0;
    if (e < total) {
      const int r = (int)(e % M), j = (int)(e / M);
      const bool mirror = sym && r > j;
      const int rr = mirror ? j : r, jj = mirror ? r : j;
      for (int z = q; z < splits; z += G) acc += (double)part[((size_t)z * npad + jj) * Mpad + rr];
    }
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (q == 0 && e < total) {
      const int r = (int)(e % M), j = (int)(e / M);
      double* c = C + r + (size_t)j * ldc;
      *c = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *c);
    }
  }
}

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split_tf32(double x, float& hi, float& lo) {
  hi = round_tf32((float)x);
  lo = round_tf32((float)(x - (double)hi));
}

// plane(r, k) = A[row0 + k + r * lda] for r < rows, k < inner; zero padding up to ld
__global__ void tc_planes_cols(int rows, int inner, int ld, const double* __restrict__ A, int lda,
                               int row0, float* __restrict__ hi, float* __restrict__ lo) {
  const size_t total = (size_t)rows * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % ld), r = (int)(e / ld);
    float h = 0.0f, l = 0.0f;
    if (k < inner) split_tf32(A[row0 + k + (size_t)r * lda], h, l);
    hi[e] = h;
    lo[e] = l;
  }
}

// transposed: plane(i, j) = A[i + j * lda] for i < m, j < n (plane row i, ld)
__global__ void tc_planes_rows(int m, int n, int ld, const double* __restrict__ A, int lda,
                               float* __restrict__ hi, float* __restrict__ lo) {
  __shared__ double t[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  for (int jj = ty; jj < 32; jj += 8) {
    const int i = i0 + tx, j = j0 + jj;
    t[jj][tx] = (i < m && j < n) ? A[i + (size_t)j * lda] : 0.0;
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    if (i < m && j < ld) {
      float h, l;
      split_tf32(t[tx][ii], h, l);
      hi[(size_t)i * ld + j] = h;
      lo[(size_t)i * ld + j] = l;
    }
  }
}

// ------------------------------------------------------------------- host --
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mutex;

blws_status get_encoder(Ctx* ctx) {
  std::lock_guard<std::mutex> lock(g_encode_mutex);
  if (g_encode) return BLWS_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  const cudaError_t e =
      cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return ctx->fail(BLWS_ENOTSUP, "cuTensorMapEncodeTiled is not available from the driver");
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return BLWS_OK;
}

// K-major plane (rows x inner, ld floats): box of kTcBK x box_rows, 128-byte swizzle
blws_status encode_plane(Ctx* ctx, CUtensorMap* map, const float* base, int rows, int inner, int ld,
                         int box_rows) {
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld % 4))
    return ctx->fail(BLWS_EINVAL, "tensor-core operand plane not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return ctx->fail(BLWS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return BLWS_OK;
}

template <int NPAD, int STAGES>
blws_status launch_tc(Ctx* ctx, cudaStream_t s, const TcJobs& jobs, int blocks) {
  auto kern = tc_tf32x3_kernel<NPAD, STAGES>;
  const int bytes = (int)tc_smem_bytes<NPAD, STAGES>();
  static_assert(tc_smem_bytes<NPAD, STAGES>() <= 227 * 1024, "shared memory per CTA");
  BLWS_TRY_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  kern<<<blocks, kTcThreads, bytes, s>>>(jobs);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

}  // namespace

int tc_npad(int b) {
  if (b <= 16) return 16;
  if (b <= 32) return 32;
  if (b <= 64) return 64;
  if (b <= 96) return 96;
  if (b <= 128) return 128;
  if (b <= 192) return 192;
  if (b <= 256) return 256;
  return 0;
}

int tc_ld(int inner) { return ceil_div(inner, 32) * 32; }

blws_status tc_planes_from_cols(Ctx* ctx, cudaStream_t s, const double* A, int lda, int row0, int inner,
                                int rows, const TcPlanes& out) {
  if (rows <= 0) return BLWS_OK;
  const size_t total = (size_t)rows * out.ld;
  tc_planes_cols<<<std::min(ceil_div((long long)total, 256), ctx->sms * 8), 256, 0, s>>>(
      rows, inner, out.ld, A, lda, row0, out.hi, out.lo);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

blws_status tc_planes_from_rows(Ctx* ctx, cudaStream_t s, const double* A, int lda, int m, int n,
                                const TcPlanes& out) {
  if (m <= 0 || n <= 0) return BLWS_OK;
  dim3 grid(ceil_div(m, 32), ceil_div(out.ld, 32));
  tc_planes_rows<<<grid, 256, 0, s>>>(m, n, out.ld, A, lda, out.hi, out.lo);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

blws_status tc_dual_apply(Ctx* ctx, cudaStream_t s, const TcPlanes& Wr, const TcPlanes& Wc, int m,
                          int n, const double* X, int ldx, int b, double* P, int ldp) {
  const int npad = tc_npad(b);
  if (npad == 0) return ctx->fail(BLWS_EINVAL, "tensor-core product: block width %d > 256", b);
  BLWS_TRY(get_encoder(ctx));
  // X_u (rows 0..m) and X_v (rows m..m+n) as planes with b rows
  const int ldu = tc_ld(m), ldv = tc_ld(n);
  float* xp = nullptr;
  BLWS_TRY(ctx->get(BUF_TC_X, (size_t)2 * b * (ldu + ldv), &xp));
  TcPlanes Xu{xp, xp + (size_t)b * ldu, b, m, ldu};
  TcPlanes Xv{xp + (size_t)2 * b * ldu, xp + (size_t)2 * b * ldu + (size_t)b * ldv, b, n, ldv};
  BLWS_TRY(tc_planes_from_cols(ctx, s, X, ldx, 0, m, b, Xu));
  BLWS_TRY(tc_planes_from_cols(ctx, s, X, ldx, m, n, b, Xv));

  // job 0: P_u = W X_v (A = Wr: m rows, K = n); job 1: P_v = W^T X_u (A = Wc: n rows, K = m)
  const int Ms[2] = {m, n}, Ks[2] = {n, m};
  const int tiles0 = ceil_div(m, kTcBM), tiles1 = ceil_div(n, kTcBM);

  TcJobs jobs;
  memset(&jobs, 0, sizeof(jobs));
  size_t part_off[2] = {0, 0}, part_total = 0;
  int splits[2], kchunk[2], tiles[2] = {tiles0, tiles1};
  for (int t = 0; t < 2; ++t) {
    // the tensor core's FP32 accumulation error grows with the number of
    // terms: at most kTcMaxChunk of K per accumulator, then FP64 sums
    const int kblocks = ceil_div(Ks[t], kTcBK);
    const int per = ceil_div(ctx->sms, std::max(1, tiles[t]));  // each product fills about a wave
    int sp = std::max(1, std::min(per, kblocks));
    sp = std::max(sp, ceil_div(Ks[t], kTcMaxChunk));
    kchunk[t] = ceil_div(kblocks, sp) * kTcBK;
    splits[t] = ceil_div(Ks[t], kchunk[t]);
    part_off[t] = part_total;
    part_total += (size_t)splits[t] * npad * tiles[t] * kTcBM;
  }
  float* part = nullptr;
  BLWS_TRY(ctx->get(BUF_TC_PART, part_total, &part));
  const TcPlanes* A[2] = {&Wr, &Wc};
  const TcPlanes* B[2] = {&Xv, &Xu};
  for (int t = 0; t < 2; ++t) {
    TcJob& J = jobs.job[t];
    BLWS_TRY(encode_plane(ctx, &J.a_hi, A[t]->hi, Ms[t], Ks[t], A[t]->ld, kTcBM));
    BLWS_TRY(encode_plane(ctx, &J.a_lo, A[t]->lo, Ms[t], Ks[t], A[t]->ld, kTcBM));
    BLWS_TRY(encode_plane(ctx, &J.b_hi, B[t]->hi, b, Ks[t], B[t]->ld, npad));
    BLWS_TRY(encode_plane(ctx, &J.b_lo, B[t]->lo, b, Ks[t], B[t]->ld, npad));
    J.part = part + part_off[t];
    J.M = Ms[t];
    J.K = Ks[t];
    J.tiles = tiles[t];
    J.splits = splits[t];
    J.kchunk = kchunk[t];
    J.Mpad = tiles[t] * kTcBM;
  }
  double* scal = nullptr;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  jobs.blocks0 = tiles0 * splits[0];
  jobs.N = b;
  jobs.err = reinterpret_cast<int*>(scal + SLOT_TCERR);
  const int blocks = jobs.blocks0 + tiles1 * splits[1];
  BLWS_TRY(ctx->time_begin(s));
  switch (npad) {
    case 16: BLWS_TRY((launch_tc<16, 5>(ctx, s, jobs, blocks))); break;
    case 32: BLWS_TRY((launch_tc<32, 5>(ctx, s, jobs, blocks))); break;
    case 64: BLWS_TRY((launch_tc<64, 4>(ctx, s, jobs, blocks))); break;
    case 96: BLWS_TRY((launch_tc<96, 3>(ctx, s, jobs, blocks))); break;
    case 128: BLWS_TRY((launch_tc<128, 3>(ctx, s, jobs, blocks))); break;
    case 192: BLWS_TRY((launch_tc<192, 2>(ctx, s, jobs, blocks))); break;
    default: BLWS_TRY((launch_tc<256, 2>(ctx, s, jobs, blocks))); break;
  }
  BLWS_TRY(ctx->time_end(s, 2.0 * m * n * b, 1));
  for (int t = 0; t < 2; ++t) {
    const size_t total = (size_t)Ms[t] * b;
    if (total == 0) continue;
    tc_reduce<<<std::min(ceil_div((long long)total, 256), ctx->sms * 8), 256, 0, s>>>(
        Ms[t], b, npad, splits[t], jobs.job[t].Mpad, jobs.job[t].part, P + (t ? m : 0), ldp);
    BLWS_CHECK_LAUNCH(ctx);
  }
  return BLWS_OK;
}

}  // namespace blws

// ------------------------------------------------ bounded-wait self-test --
// One CTA initialises an mbarrier that expects one arrival and waits for its
// first phase through the same bounded wait the tensor-core kernels use;
// nothing arrives, so after `polls` polls the wait gives up and the kernel
// raises the context's tensor-core error word, as a producer/consumer kernel
// does when a copy or an MMA never completes.  No copy, MMA or tensor memory
// is involved, so giving up leaves nothing in flight.
namespace blws {
namespace {

__global__ void wait_probe_kernel(uint32_t polls, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, polls)) atomicExch(err, 1);
}

}  // namespace

blws_status wait_probe(Ctx* ctx, cudaStream_t s, unsigned polls) {
  double* scal = nullptr;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  wait_probe_kernel<<<1, 32, 0, s>>>(polls, reinterpret_cast<int*>(scal + SLOT_TCERR));
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

}  // namespace blws

// ------------------------------------------------------- general products --
namespace blws {

// C = alpha op(A) op(B) + beta C from split TF32 operands (three tcgen05
// products per K step, FP32 sums of at most 256 terms, FP64 beyond), for the
// mixed-precision mode's block products.  The columns of op(B) go through the
// accumulator 256 at a time.
blws_status tc_gemm(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                    const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                    bool sym) {
  if (M <= 0 || N <= 0 || K <= 0) return ctx->fail(BLWS_EINVAL, "tc_gemm: empty product");
  BLWS_TRY(get_encoder(ctx));
  constexpr int kCols = 256;
  const int ldk = tc_ld(K);
  const int nmax = std::min(N, kCols);
  float* base = nullptr;
  BLWS_TRY(ctx->get(BUF_TC_G, (size_t)2 * ((size_t)M + nmax) * ldk, &base));
  const TcPlanes Ap{base, base + (size_t)M * ldk, M, K, ldk};
  float* bbase = base + (size_t)2 * M * ldk;
  // rows of op(A), K-major
  if (ta) BLWS_TRY(tc_planes_from_cols(ctx, s, A, lda, 0, K, M, Ap));
  else BLWS_TRY(tc_planes_from_rows(ctx, s, A, lda, M, K, Ap));
  const int tiles = ceil_div(M, kTcBM);
  const int kblocks = ceil_div(K, kTcBK);
  // about one wave of CTAs, at least two K blocks each
  const int per = ceil_div(ctx->sms, std::max(1, tiles));
  int sp = std::max(1, std::min(per, ceil_div(kblocks, 2)));
  sp = std::max(sp, ceil_div(K, kTcMaxChunk));
  const int kchunk = ceil_div(kblocks, sp) * kTcBK;
  const int splits = ceil_div(K, kchunk);
  double* scal = nullptr;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  for (int j0 = 0; j0 < N; j0 += kCols) {
    const int nc = std::min(kCols, N - j0);
    const int npad = tc_npad(nc);
    const TcPlanes Bp{bbase, bbase + (size_t)nc * ldk, nc, K, ldk};
    // columns j0 .. j0 + nc of op(B) as rows, K-major
    if (tb) BLWS_TRY(tc_planes_from_rows(ctx, s, B + j0, ldb, nc, K, Bp));
    else BLWS_TRY(tc_planes_from_cols(ctx, s, B + (size_t)j0 * ldb, ldb, 0, K, nc, Bp));
    float* part = nullptr;
    BLWS_TRY(ctx->get(BUF_TC_PART, (size_t)splits * npad * tiles * kTcBM, &part));
    TcJobs jobs;
    memset(&jobs, 0, sizeof(jobs));
    TcJob& J = jobs.job[0];
    BLWS_TRY(encode_plane(ctx, &J.a_hi, Ap.hi, M, K, ldk, kTcBM));
    BLWS_TRY(encode_plane(ctx, &J.a_lo, Ap.lo, M, K, ldk, kTcBM));
    BLWS_TRY(encode_plane(ctx, &J.b_hi, Bp.hi, nc, K, ldk, npad));
    BLWS_TRY(encode_plane(ctx, &J.b_lo, Bp.lo, nc, K, ldk, npad));
    J.part = part;
    J.M = M;
    J.K = K;
    J.tiles = tiles;
    J.splits = splits;
    J.kchunk = kchunk;
    J.Mpad = tiles * kTcBM;
    jobs.job[1] = J;  // unused: every block belongs to job 0
    jobs.blocks0 = tiles * splits;
    jobs.N = nc;
    jobs.err = reinterpret_cast<int*>(scal + SLOT_TCERR);
    const int blocks = jobs.blocks0;
    switch (npad) {
      case 16: BLWS_TRY((launch_tc<16, 5>(ctx, s, jobs, blocks))); break;
      case 32: BLWS_TRY((launch_tc<32, 5>(ctx, s, jobs, blocks))); break;
      case 64: BLWS_TRY((launch_tc<64, 4>(ctx, s, jobs, blocks))); break;
      case 96: BLWS_TRY((launch_tc<96, 3>(ctx, s, jobs, blocks))); break;
      case 128: BLWS_TRY((launch_tc<128, 3>(ctx, s, jobs, blocks))); break;
      case 192: BLWS_TRY((launch_tc<192, 2>(ctx, s, jobs, blocks))); break;
      default: BLWS_TRY((launch_tc<256, 2>(ctx, s, jobs, blocks))); break;
    }
    const size_t total = (size_t)M * nc;
    int G = 1;
    while (G < 32 && 2 * G <= splits && total * (size_t)(2 * G) <= (size_t)ctx->sms * 8 * 256) G *= 2;
    const bool symc = sym && N <= kCols && M == N && beta == 0.0;
    tc_reduce_ab<<<(int)std::min<size_t>((total * G + 255) / 256, (size_t)ctx->sms * 8), 256, 0, s>>>(
        M, nc, npad, splits, J.Mpad, part, alpha, beta, C + (size_t)j0 * ldc, ldc, symc ? 1 : 0, G);
    BLWS_CHECK_LAUNCH(ctx);
  }
  return BLWS_OK;
}

}  // namespace blws
