// FP64-equivalent products with the augmented matrix on the tensor cores
// (Ozaki-type splitting): P = [W X_v; W^T X_u] for BLWS_PREC_FP64_TC.
//
// Every row i of an A operand (and every column j of a B operand) is scaled by
// a power of two, 2^E_i >= max |entries|, and written in balanced base-128
// digits: w = 2^E_i sum_{t=1..S} a_t 128^-t with integers |a_1| <= 128 and
// |a_t| <= 64 (t >= 2), each exact in BF16 (S = 7: 49 bits).  Then
//   (W X)_ij = 2^{E_i + F_j} sum_{L} 128^-L acc_L,
//   acc_L = sum_k sum_{t+u=L} a_t(i,k) b_u(k,j),
// and pairs with t + u > S + 1 are dropped (below 2^-47 of the leading
// term).  Each level L = 2..S+1 is one FP32 accumulator in tensor memory,
// filled by tcgen05.mma.kind::f16 on the BF16 digit planes; a level's sum over
// 256 terms stays below 2^24 in magnitude with integer values, so it is exact.
// Every 256 terms the four epilogue warps move the levels out of tensor
// memory into a double-FP32 (hi + lo) accumulator per output (FP64 is slow on
// this GPU; two FP32 words carry 48 bits), and at the end multiply by the
// scales in FP64.  Split-K partials are added in FP64 in a fixed order.
//
// Operands are K-major BF16 planes with 64-byte swizzle (32 elements per
// K block), loaded by 3-D TMA (K, row, digit plane).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ops.cuh"
#include "tc_ptx.cuh"
#include "tune.cuh"

namespace blws {

namespace {

using namespace tc;

constexpr int kOzS = 7;          // digits per value
constexpr int kOzBM = 128;       // rows per CTA (tensor-memory lanes)
constexpr int kOzBN = 64;        // columns per CTA (one accumulator level = 64 columns)
constexpr int kOzBK = 32;        // K block: 32 BF16 = one 64-byte swizzle row
constexpr int kOzChunk = 256;    // exact FP32 sums: at most 256 K terms per level between drains
constexpr int kOzStages = 2;
// drain warps: two per tensor-memory lane quarter, each draining half of the
// 64 columns (eight warps halve the drain that separates a chunk's MMAs from
// the next chunk's; four would need 2 x 64 accumulators per thread)
constexpr int kOzDrainWarps = 8;
constexpr int kOzDrainCols = kOzBN * 4 / kOzDrainWarps;
constexpr int kOzThreads = 128 + 32 * kOzDrainWarps;  // warp 0 TMA, warp 1 MMA, warp 2 TMEM, 4.. drain
constexpr int kOzLevels = kOzS;  // levels L = 2 .. S + 1
constexpr int kOzPairs = kOzS * (kOzS + 1) / 2;  // pairs (t, u) with t + u <= S + 1

struct OzJob {
  CUtensorMap a, b;     // 3-D maps: (K, rows, plane)
  const int* ea;        // row scales of A (rows)
  const int* eb;        // column scales of B (b columns)
  float2* part;         // [splits][npad][Mpad] (hi, lo) partial sums, unscaled
  int M, K, tiles, ngroups, splits, kchunk, Mpad, npad;
};

struct OzJobs {
  OzJob job[2];
  int blocks0;
  int N;
  int* err;
};

// (t, u) digit pairs ordered by level, the first pair of each level first
struct PairTable {
  int t[kOzPairs], u[kOzPairs];
  __host__ __device__ constexpr PairTable() : t{}, u{} {
    int p = 0;
    for (int L = 2; L <= kOzS + 1; ++L)
      for (int tt = 1; tt <= kOzS; ++tt) {
        const int uu = L - tt;
        if (uu >= 1 && uu <= kOzS) {
          t[p] = tt;
          u[p] = uu;
          ++p;
        }
      }
  }
};

// (hi, lo) += (v.x, v.y) for double-FP32 values: Knuth's TwoSum on the high
// words, the low words and the rounding error added to lo
__device__ __forceinline__ void df_add(float& hi, float& lo, float2 v) {
  const float s = hi + v.x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (v.x - bb);
  hi = s;
  lo += err + v.y;
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  // (hi, lo) += v with the rounding error of hi + v kept in lo (Knuth's TwoSum)
  const float s = hi + v;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (v - bb);
  hi = s;
  lo += err;
}

__global__ void __launch_bounds__(kOzThreads, 1) oz_kernel(const __grid_constant__ OzJobs jobs) {
  // the drain warps hold 2 x 64 FP32 accumulators per thread
  constexpr int A_BYTES = kOzBM * kOzBK * 2;  // 8 KB per digit plane
  constexpr int B_BYTES = kOzBN * kOzBK * 2;  // 4 KB
  constexpr int STAGE = kOzS * (A_BYTES + B_BYTES);
  constexpr uint32_t NCOLS = 512;
  constexpr PairTable PT;
  static_assert(kOzLevels * kOzBN <= 512, "levels x columns fit the tensor memory");
  static_assert(STAGE % 1024 == 0, "stage alignment");
  extern __shared__ uint8_t oz_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(oz_smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full_bar[kOzStages];
  __shared__ __align__(8) uint64_t empty_bar[kOzStages];
  __shared__ __align__(8) uint64_t chunk_bar;    // MMA -> drain: a chunk's levels are complete
  // drain -> MMA, one per level: the level's accumulator of the previous chunk
  // has been read and may be overwritten (the next chunk's MMAs start on the
  // levels already drained while the drain works through the rest)
  __shared__ __align__(8) uint64_t level_bar[kOzLevels];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fail_sh;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int jb = (int)blockIdx.x < jobs.blocks0 ? 0 : 1;
  const OzJob& J = jobs.job[jb];
  const int local = jb ? (int)blockIdx.x - jobs.blocks0 : (int)blockIdx.x;
  const int tile = local % J.tiles;
  const int ng = (local / J.tiles) % J.ngroups;
  const int split = local / (J.tiles * J.ngroups);
  const int row0 = tile * kOzBM, col0 = ng * kOzBN;
  const int kbeg = split * J.kchunk;
  const int kend = min(J.K, kbeg + J.kchunk);
  const int nk = (kend - kbeg + kOzBK - 1) / kOzBK;
  constexpr int kPerChunk = kOzChunk / kOzBK;
  const int nchunks = (nk + kPerChunk - 1) / kPerChunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&chunk_bar, 1);
    for (int L = 0; L < kOzLevels; ++L) mbar_init(&level_bar[L], 32 * kOzDrainWarps);  // every drain thread
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
    // producer: S A-planes and S B-planes per K block (two 3-D boxes)
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kOzStages;
      const uint32_t round = (uint32_t)(kb / kOzStages);
      if (kb >= kOzStages && !mbar_wait(&empty_bar[s], (round & 1u) ^ 1u)) {
        fail_sh = 1;
        break;
      }
      uint8_t* st = smem + (size_t)s * STAGE;
      mbar_expect_tx(&full_bar[s], STAGE);
      const int kx = kbeg + kb * kOzBK;
      asm volatile(
          "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(st)),
          "l"(reinterpret_cast<uint64_t>(&J.a)), "r"(kx), "r"(row0), "r"(0), "r"(smem_u32(&full_bar[s]))
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(st + kOzS * A_BYTES)),
          "l"(reinterpret_cast<uint64_t>(&J.b)), "r"(kx), "r"(col0), "r"(0), "r"(smem_u32(&full_bar[s]))
          : "memory");
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = bf16_idesc(kOzBM, kOzBN);
    int kb = 0;
    bool stop = false;
    for (int c = 0; c < nchunks && !stop; ++c) {
      const int kb_end = min(nk, kb + kPerChunk);
      for (int kc = 0; kb < kb_end; ++kb, ++kc) {
        const int s = kb % kOzStages;
        const uint32_t round = (uint32_t)(kb / kOzStages);
        if (!mbar_wait(&full_bar[s], round & 1u)) {
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + (size_t)s * STAGE);
#pragma unroll
        for (int kk = 0; kk < kOzBK / 16; ++kk) {
#pragma unroll
          for (int p = 0; p < kOzPairs; ++p) {
            const int t = PT.t[p], u = PT.u[p], L = t + u;
            const bool first_of_level = (p == 0) || (PT.t[p - 1] + PT.u[p - 1] != L);
            const uint64_t ad = sw64_desc(st + (uint32_t)(t - 1) * A_BYTES + kk * 32);
            const uint64_t bd = sw64_desc(st + kOzS * A_BYTES + (uint32_t)(u - 1) * B_BYTES + kk * 32);
            const uint32_t acc = (kc > 0 || kk > 0 || !first_of_level) ? 1u : 0u;
            if (c > 0 && !acc) {  // the level restarts: its previous chunk must be drained
              if (!mbar_wait(&level_bar[L - 2], (uint32_t)((c - 1) & 1))) stop = true;
              tc_fence_after();
            }
            if (!stop) mma_bf16(tbase + (uint32_t)((L - 2) * kOzBN), ad, bd, idesc, acc);
          }
        }
        mma_commit(&empty_bar[s]);
        if (stop) break;
      }
      if (stop) {
        fail_sh = 1;
        break;
      }
      mma_commit(&chunk_bar);  // this chunk's levels complete once the MMAs above are done
    }
  }
  __syncwarp();

  if (warp < 4) {  // producer, MMA issuer and allocator wait for the drain warps below
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
      tc_fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS)
                   : "memory");
    }
    return;
  }
  // drain (warps 4..: warp w reads tensor-memory lanes 32 ((w - 4) mod 4) ..,
  // columns kOzDrainCols ((w - 4) / 4) ..): every chunk, levels -> double-FP32
  // accumulators, one row per thread
  const int q = (warp - 4) & 3;
  const int cb = ((warp - 4) >> 2) * kOzDrainCols;
  float hi[kOzDrainCols], lo[kOzDrainCols];
#pragma unroll
  for (int j = 0; j < kOzDrainCols; ++j) {
    hi[j] = 0.0f;
    lo[j] = 0.0f;
  }
  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    if (!mbar_wait(&chunk_bar, (uint32_t)(c & 1))) {
      ok = false;
      break;
    }
    tc_fence_after();
#pragma unroll 1
    for (int L = 2; L <= kOzS + 1; ++L) {
      const float scale = __uint_as_float((uint32_t)(127 - 7 * L) << 23);  // 2^(-7 L), exact
      float v[kOzDrainCols];
#pragma unroll
      for (int c0 = 0; c0 < kOzDrainCols; c0 += 16) {
        float w16[16];
        tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)((L - 2) * kOzBN + cb + c0), w16);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[c0 + j] = w16[j];
      }
      // the level is in registers: release it to the next chunk's MMAs
      tc_fence_before();
      mbar_arrive(&level_bar[L - 2]);
#pragma unroll
      for (int j = 0; j < kOzDrainCols; ++j) two_sum_acc(hi[j], lo[j], v[j] * scale);
    }
  }
  if (ok && !fail_sh) {
    // (hi, lo) pairs out; the FP64 combination and the power-of-two scales are
    // applied by the grid-wide reduction (FP64 on one SM would cost more than
    // this CTA's tensor work)
    const int row = row0 + q * 32 + lane;
    if (row < J.M) {
      float2* out = J.part + (size_t)split * J.npad * J.Mpad;
#pragma unroll
      for (int j = 0; j < kOzDrainCols; ++j) {
        const int col = col0 + cb + j;
        if (col < jobs.N) out[(size_t)col * J.Mpad + row] = make_float2(hi[j], lo[j]);
      }
    }
  } else if (threadIdx.x == 128) {
    atomicExch(jobs.err, 1);
  }
  tc_fence_before();
  __syncthreads();  // matches the one above: tensor memory is freed after the last read
}

// ------------------------------------------------------------- splitting --
// exponent E with max |v| < 2^E (0 for an all-zero vector)
__device__ __forceinline__ int scale_exp(double mx) { return mx > 0.0 ? ilogb(mx) + 1 : 0; }

// FP64 runs at 1/64 of the FP32 rate on this GPU, so the splitting and the
// recombination keep FP64 arithmetic out of their per-element work: maxima
// are taken on the bit patterns of |v| (for non-negative doubles the integer
// order is the numeric order), powers of two are built from their bits, and
// sums of (hi, lo) partials are double-FP32.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// scale_exp of the double whose |bits| are b (the largest magnitude of a row)
__device__ __forceinline__ int scale_exp_bits(unsigned long long b) {
  const int be = (int)(b >> 52);
  if (be > 0) return be - 1022;  // normal: ilogb + 1
  return b ? scale_exp(__longlong_as_double((long long)b)) : 0;
}

// 2^e as a double, exactly (normal range), else through ldexp
__device__ __forceinline__ double pow2(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(1023 + e) << 52) : ldexp(1.0, e);
}

// balanced base-128 digits of x = v 2^-E (|x| < 1): M = rint(x 2^(7S)),
// digits from the least significant: d = ((M + 64) mod 128) - 64.  The
// scaling by a power of two is exact (one multiply); M is rounded to nearest,
// ties to even.
__device__ __forceinline__ void digits(double v, int E, int (&a)[kOzS]) {
  const int sh = 7 * kOzS - E;
  const double x = (sh >= -1022 && sh <= 1023) ? v * pow2(sh) : ldexp(v, sh);
  long long M = __double2ll_rn(x);
#pragma unroll
  for (int t = kOzS - 1; t >= 1; --t) {
    const long long d = ((M + 64) & 127) - 64;
    a[t] = (int)d;
    M = (M - d) >> 7;
  }
  a[0] = (int)M;
}

// E[i] for the rows of the column-major m x n block A (ld), from 32 x 32 tiles:
// each tile's row maxima enter by an integer atomic max of their exponents
// (E starts below every exponent; an all-zero row keeps that value, and its
// digits are zero whatever E is)
constexpr int kOzNoExp = -4000;
constexpr int kOzStripMaxN = 1024;  // row planes of blocks with rows up to this long: one launch

__global__ void oz_row_scales(int m, int n, const double* __restrict__ A, int lda, int* E) {
  __shared__ unsigned long long t[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  for (int jj = ty; jj < 32; jj += 8) {
    const int i = i0 + tx, j = j0 + jj;
    t[jj][tx] = (i < m && j < n) ? abs_bits(A[i + (size_t)j * lda]) : 0ull;
  }
  __syncthreads();
  if (ty == 0) {
    unsigned long long mx = 0ull;
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) mx = max(mx, t[jj][tx]);
    if (mx && i0 + tx < m) atomicMax(&E[i0 + tx], scale_exp_bits(mx));
  }
}

__global__ void oz_fill(int n, int v, int* E) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) E[i] = v;
}

// digit planes of `rows` columns of a column-major operand: column r is
// A[row0 + k + r lda], k < inner, split with its own scale E[r]; `chunks` CTAs
// share a column (each finds the column's maximum, then splits its part)
struct ColsJob {
  int rows, plane_rows, inner, ld;
  const double* A;
  int lda, row0, chunks;
  int* E;
  __nv_bfloat16* planes;
};

__device__ __forceinline__ void planes_cols_body(const ColsJob& J, int bid, int nblk) {
  __shared__ unsigned long long red[8];
  __shared__ int e_sh;
  const size_t plane = (size_t)J.plane_rows * J.ld;
  const int span = (J.ld + J.chunks - 1) / J.chunks;
  for (int item = bid; item < J.rows * J.chunks; item += nblk) {
    const int r = item / J.chunks, c = item % J.chunks;
    const double* col = J.A + J.row0 + (size_t)r * J.lda;
    unsigned long long mx = 0ull;
    for (int k = threadIdx.x; k < J.inner; k += blockDim.x) mx = max(mx, abs_bits(col[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m2 = 0ull;
      for (int w = 0; w < (int)blockDim.x / 32; ++w) m2 = max(m2, red[w]);
      e_sh = scale_exp_bits(m2);
      if (c == 0) J.E[r] = e_sh;
    }
    __syncthreads();
    const int er = e_sh;
    const int kend = min(J.ld, (c + 1) * span);
    for (int k = c * span + threadIdx.x; k < kend; k += blockDim.x) {
      int a[kOzS];
      if (k < J.inner) {
        digits(col[k], er, a);
      } else {
#pragma unroll
        for (int t = 0; t < kOzS; ++t) a[t] = 0;
      }
#pragma unroll
      for (int t = 0; t < kOzS; ++t)
        J.planes[t * plane + (size_t)r * J.ld + k] = __float2bfloat16_rn((float)a[t]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) oz_planes_cols(ColsJob J) {
  planes_cols_body(J, blockIdx.x, gridDim.x);
}

// two operands' column planes in one launch: blocks [0, blocks0) for J0, the rest for J1
__global__ void __launch_bounds__(256) oz_planes_cols2(ColsJob J0, ColsJob J1, int blocks0) {
  if ((int)blockIdx.x < blocks0)
    planes_cols_body(J0, blockIdx.x, blocks0);
  else
    planes_cols_body(J1, blockIdx.x - blocks0, gridDim.x - blocks0);
}

// transposed digit planes of the m x n column-major A: plane t, (i, j) = A[i + j lda],
// split with the scale of row i
__global__ void oz_planes_rows(int m, int n, int ld, int plane_rows, const double* __restrict__ A, int lda,
                               const int* __restrict__ E, __nv_bfloat16* planes) {
  __shared__ double tile[32][33];
  const size_t plane = (size_t)plane_rows * ld;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int jj = ty; jj < 32; jj += 8) {
    const int i = i0 + tx, j = j0 + jj;
    tile[jj][tx] = (i < m && j < n) ? A[i + (size_t)j * lda] : 0.0;
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    if (i < m && j < ld) {
      int a[kOzS];
      digits(tile[tx][ii], E[i], a);
#pragma unroll
      for (int t = 0; t < kOzS; ++t)
        planes[t * plane + (size_t)i * ld + j] = __float2bfloat16_rn((float)a[t]);
    }
  }
}

// One launch for the row planes of a column-major m x n block with a short
// row (n up to a thousand or so; plane row i = row i of A, K along A's
// columns): blockIdx.x takes a strip of 32 rows, blockIdx.y one of the
// gridDim.y shares of the planes' columns.  Every CTA of a strip first finds
// the 32 rows' maxima over all n columns (the same exponents in every CTA, no
// atomics, and an all-zero row keeps kOzNoExp, whose digits are zero), then
// splits its share 32 x 32 tiles at a time and writes them transposed; the
// first share records E.
__global__ void __launch_bounds__(256) oz_planes_rows_strip(int m, int n, int ld, int plane_rows,
                                                            const double* __restrict__ A, int lda, int* E,
                                                            __nv_bfloat16* planes) {
  __shared__ double tile[32][33];
  __shared__ unsigned long long red[8][32];
  __shared__ int e_sh[32];
  const size_t plane = (size_t)plane_rows * ld;
  const int i0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  const int i = i0 + tx;
  unsigned long long mx = 0ull;
  if (i < m)
    for (int j = ty; j < n; j += 8) mx = max(mx, abs_bits(A[i + (size_t)j * lda]));
  red[ty][tx] = mx;
  __syncthreads();
  if (ty == 0) {
    unsigned long long m2 = 0ull;
#pragma unroll
    for (int w = 0; w < 8; ++w) m2 = max(m2, red[w][tx]);
    const int e = m2 ? scale_exp_bits(m2) : kOzNoExp;
    e_sh[tx] = e;
    if (blockIdx.y == 0 && i < m) E[i] = e;
  }
  __syncthreads();
  const int tiles = (ld + 31) / 32, per = (tiles + gridDim.y - 1) / gridDim.y;
  const int tb = blockIdx.y * per, te = min(tiles, tb + per);
  for (int tj = tb; tj < te; ++tj) {
    const int j0 = tj * 32;
    for (int jj = ty; jj < 32; jj += 8) {
      const int j = j0 + jj;
      tile[jj][tx] = (i < m && j < n) ? A[i + (size_t)j * lda] : 0.0;
    }
    __syncthreads();
    for (int ii = ty; ii < 32; ii += 8) {
      const int r = i0 + ii, j = j0 + tx;
      if (r < m && j < ld) {
        int a[kOzS];
        digits(tile[tx][ii], e_sh[ii], a);
#pragma unroll
        for (int t = 0; t < kOzS; ++t)
          planes[t * plane + (size_t)r * ld + j] = __float2bfloat16_rn((float)a[t]);
      }
    }
    __syncthreads();
  }
}

// P(r, j) = 2^(E_r + F_j) sum over splits of (hi + lo), in FP64.  Each output
// is summed by a group of G lanes (G a power of two up to 32, so that small
// outputs with many splits still fill the GPU): lane q adds splits q, q + G, ...
// in order, then the group adds its lanes with a fixed shuffle tree -- a fixed
// order for given sizes.  sym (a product known to be symmetric, M = N,
// beta = 0): an element below the diagonal is formed from its mirror's
// partials, so P is exactly symmetric.
__global__ void oz_reduce(int M, int N, int npad, int splits, int Mpad, const float2* __restrict__ part,
                          const int* __restrict__ ea, const int* __restrict__ eb, double* __restrict__ P,
                          int ldp, double alpha, double beta, int sym, int G) {
  const size_t total = (size_t)M * N;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t nth = (size_t)gridDim.x * blockDim.x;
  const int q = (int)(tid % G);
  // every lane of a warp runs the same number of iterations (the shuffles need them all)
  const size_t span = (total * G + nth - 1) / nth * nth;
  for (size_t t = tid; t < span; t += nth) {
    const size_t e = t / G;
    float hi = 0.0f, lo = 0.0f;  // double-FP32 sum of the (hi, lo) partials
    int rr = 0, jj = 0;
    if (e < total) {
      const int r = (int)(e % M), j = (int)(e / M);
      const bool mirror = sym && r > j;
      rr = mirror ? j : r;
      jj = mirror ? r : j;
      const size_t zs = (size_t)npad * Mpad;
      const float2* src = part + (size_t)jj * Mpad + rr;
      int z = q;
      for (; z + 3 * G < splits; z += 4 * G) {  // four independent loads, then the sums in order
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = src[(size_t)(z + u * G) * zs];
#pragma unroll
        for (int u = 0; u < 4; ++u) df_add(hi, lo, v[u]);
      }
      for (; z < splits; z += G) df_add(hi, lo, src[(size_t)z * zs]);
    }
    for (int o = G / 2; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
      df_add(hi, lo, make_float2(oh, ol));
    }
    if (q == 0 && e < total) {
      const int r = (int)(e % M), j = (int)(e / M);
      const int e2 = ea[rr] + eb[jj];
      const double sum = (double)hi + (double)lo;
      const double v = (e2 >= -1022 && e2 <= 1023) ? sum * pow2(e2) : ldexp(sum, e2);
      double* c = P + r + (size_t)j * ldp;
      *c = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *c);
    }
  }
}

// lanes per output of oz_reduce: enough to fill ~8 x 256 threads per SM, at
// most 32 and the split count
int oz_lanes(int sms, size_t total, int splits) {
  int G = 1;
  while (G < 32 && 2 * G <= splits && total * (size_t)(2 * G) <= (size_t)sms * 8 * 256) G *= 2;
  return G;
}

PFN_cuTensorMapEncodeTiled_v12000 g_oz_encode = nullptr;
std::mutex g_oz_mutex;

blws_status oz_encoder(Ctx* ctx) {
  std::lock_guard<std::mutex> lock(g_oz_mutex);
  if (g_oz_encode) return BLWS_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  const cudaError_t e =
      cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return ctx->fail(BLWS_ENOTSUP, "cuTensorMapEncodeTiled is not available from the driver");
  g_oz_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return BLWS_OK;
}

// 3-D map over S digit planes of rows x inner BF16 (ld elements per row, planes
// plane_rows rows apart); rows past `rows` read as zero digits (the copy's
// out-of-bounds fill), so padding rows need not be written
blws_status oz_encode(Ctx* ctx, CUtensorMap* map, const __nv_bfloat16* base, int rows, int plane_rows, int inner,
                      int ld, int box_rows) {
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld % 8) || rows > plane_rows)
    return ctx->fail(BLWS_EINVAL, "digit plane not 16-byte aligned");
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)kOzS};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)plane_rows * ld * 2};
  cuuint32_t box[3] = {(cuuint32_t)kOzBK, (cuuint32_t)box_rows, (cuuint32_t)kOzS};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = g_oz_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(base),
                                 dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return ctx->fail(BLWS_ECUDA, "cuTensorMapEncodeTiled (digits) failed (%d)", (int)r);
  return BLWS_OK;
}

size_t oz_smem_bytes() { return (size_t)kOzStages * kOzS * (kOzBM + kOzBN) * kOzBK * 2 + 1024; }

// Split of K for a product of `units` (row tile, column group) CTAs over
// `kblocks` K blocks with `share` SMs (one CTA per SM): the split count that
// minimises waves x (K blocks per CTA + a fixed CTA overhead), fewest splits on
// ties.  The overhead -- tensor-memory allocation, pipeline fill, the drain
// and the 64 KB store of the partial sums -- was measured at about eight K
// blocks of MMAs (2000 x 2000 product: 4 splits, 256 CTAs, 81 us; 7 splits,
// 448 CTAs, 91 us).  Splits fall on K-block boundaries; each split still sums
// its terms 256 at a time.
constexpr int kOzCtaOverhead = 8;

int oz_pick_splits(int share, int units, int kblocks) {
  share = std::max(share, 1);
  int best = 1;
  long long best_cost = -1;
  for (int sp = 1; sp <= std::min(kblocks, 256); ++sp) {
    const long long waves = ceil_div((long long)units * sp, share);
    const long long cost = waves * (ceil_div(kblocks, sp) + kOzCtaOverhead);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = sp;
    }
  }
  return best;
}

}  // namespace

int oz_ld(int inner) { return ceil_div(inner, 64) * 64; }
int oz_digits() { return kOzS; }

blws_status oz_alloc(Ctx* ctx, int m, int n, OzPlanes* Or, OzPlanes* Oc) {
  const int ldr = oz_ld(n), ldc = oz_ld(m);
  const size_t dr = (size_t)kOzS * m * ldr, dc = (size_t)kOzS * n * ldc;
  uint8_t* p = nullptr;
  const size_t bytes = (dr + dc) * sizeof(__nv_bfloat16) + ((size_t)m + n + 64) * sizeof(int);
  BLWS_TRY(ctx->get(BUF_TC_W, bytes, (void**)&p));
  __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(p);
  int* e = reinterpret_cast<int*>(p + (dr + dc) * sizeof(__nv_bfloat16));
  *Or = OzPlanes{d, e, m, n, ldr};
  *Oc = OzPlanes{d + dr, e + m, n, m, ldc};
  return BLWS_OK;
}

blws_status oz_planes_from_rows(Ctx* ctx, cudaStream_t s, const double* A, int lda, int m, int n,
                                const OzPlanes& out) {
  if (m <= 0 || n <= 0) return BLWS_OK;
  if (n <= kOzStripMaxN) {
    // one launch; a strip's maxima cost 32 n reads per share, so the shares
    // stay few: enough CTAs for about two per SM, at most 8 per strip
    const int strips = ceil_div(m, 32);
    const int shares = std::max(1, std::min(std::min(8, ceil_div(out.ld, 32)), ceil_div(2 * ctx->sms, strips)));
    oz_planes_rows_strip<<<dim3(strips, shares), 256, 0, s>>>(m, n, out.ld, out.rows, A, lda, out.e, out.d);
    BLWS_CHECK_LAUNCH(ctx);
    return BLWS_OK;
  }
  // long rows (the planes of W itself): the maxima by 32 x 32 tiles over the
  // whole grid, then the split
  oz_fill<<<ceil_div(m, 256), 256, 0, s>>>(m, kOzNoExp, out.e);
  BLWS_CHECK_LAUNCH(ctx);
  oz_row_scales<<<dim3(ceil_div(m, 32), ceil_div(n, 32)), 256, 0, s>>>(m, n, A, lda, out.e);
  BLWS_CHECK_LAUNCH(ctx);
  dim3 grid(ceil_div(m, 32), ceil_div(out.ld, 32));
  oz_planes_rows<<<grid, 256, 0, s>>>(m, n, out.ld, out.rows, A, lda, out.e, out.d);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

namespace {
// a few CTAs per column when there are too few columns to fill the GPU (each
// rereads its column for the maximum: cheap next to the digit writes)
ColsJob cols_job(const Ctx* ctx, const double* A, int lda, int row0, int inner, int rows, const OzPlanes& out,
                 int* grid) {
  const int chunks = std::max(1, std::min(8, ceil_div(2 * ctx->sms, rows)));
  *grid = std::min(rows * chunks, ctx->sms * 16);
  return ColsJob{rows, out.rows, inner, out.ld, A, lda, row0, chunks, out.e, out.d};
}

// the column planes of two operands, in one launch when both have columns
blws_status planes_cols_pair(Ctx* ctx, cudaStream_t s, const double* A0, int lda0, int row00, int inner0,
                             int rows0, const OzPlanes& out0, const double* A1, int lda1, int row01,
                             int inner1, int rows1, const OzPlanes& out1) {
  if (rows0 <= 0) return oz_planes_from_cols(ctx, s, A1, lda1, row01, inner1, rows1, out1);
  if (rows1 <= 0) return oz_planes_from_cols(ctx, s, A0, lda0, row00, inner0, rows0, out0);
  int g0 = 0, g1 = 0;
  const ColsJob j0 = cols_job(ctx, A0, lda0, row00, inner0, rows0, out0, &g0);
  const ColsJob j1 = cols_job(ctx, A1, lda1, row01, inner1, rows1, out1, &g1);
  oz_planes_cols2<<<g0 + g1, 256, 0, s>>>(j0, j1, g0);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}
}  // namespace

blws_status oz_planes_from_cols(Ctx* ctx, cudaStream_t s, const double* A, int lda, int row0, int inner,
                                int rows, const OzPlanes& out) {
  if (rows <= 0) return BLWS_OK;
  int grid = 0;
  const ColsJob j = cols_job(ctx, A, lda, row0, inner, rows, out, &grid);
  oz_planes_cols<<<grid, 256, 0, s>>>(j);
  BLWS_CHECK_LAUNCH(ctx);
  return BLWS_OK;
}

blws_status oz_dual_apply(Ctx* ctx, cudaStream_t s, const OzPlanes& Wr, const OzPlanes& Wc, int m, int n,
                          const double* X, int ldx, int b, double* P, int ldp) {
  BLWS_TRY(oz_encoder(ctx));
  const int ngroups = ceil_div(b, kOzBN), npad = ngroups * kOzBN;
  // digit planes of X_u (rows 0..m) and X_v (rows m..m+n): b rows each, scale per column
  const int ldu = oz_ld(m), ldv = oz_ld(n);
  __nv_bfloat16* xp = nullptr;
  int* xe = nullptr;
  BLWS_TRY(ctx->get(BUF_TC_X, (size_t)kOzS * npad * (ldu + ldv) * sizeof(__nv_bfloat16), (void**)&xp));
  BLWS_TRY(ctx->get(BUF_OZ_E, (size_t)2 * npad * sizeof(int), (void**)&xe));
  OzPlanes Xu{xp, xe, npad, m, ldu};
  OzPlanes Xv{xp + (size_t)kOzS * npad * ldu, xe + npad, npad, n, ldv};
  BLWS_TRY(planes_cols_pair(ctx, s, X, ldx, 0, m, b, Xu, X, ldx, m, n, b, Xv));

  const int Ms[2] = {m, n}, Ks[2] = {n, m};
  const int tiles[2] = {ceil_div(m, kOzBM), ceil_div(n, kOzBM)};
  OzJobs jobs;
  memset(&jobs, 0, sizeof(jobs));
  int splits[2], kchunk[2];
  size_t off[2], total = 0;
  // both products run in one launch: with equal K (a square W) one split count
  // for both, against all the SMs; otherwise the SMs are shared in proportion
  // to their work (a tall W gives one product few row tiles and a long K)
  const double work0 = (double)tiles[0] * ceil_div(Ks[0], kOzBK), work1 = (double)tiles[1] * ceil_div(Ks[1], kOzBK);
  for (int t = 0; t < 2; ++t) {
    const int kblocks = ceil_div(Ks[t], kOzBK);
    const int sp = Ks[0] == Ks[1]
                       ? oz_pick_splits(ctx->sms, (tiles[0] + tiles[1]) * ngroups, kblocks)
                       : oz_pick_splits((int)std::lround(ctx->sms * (t ? work1 : work0) / (work0 + work1)),
                                        tiles[t] * ngroups, kblocks);
    kchunk[t] = ceil_div(kblocks, sp) * kOzBK;
    splits[t] = ceil_div(Ks[t], kchunk[t]);
    off[t] = total;
    total += (size_t)splits[t] * npad * tiles[t] * kOzBM;
  }
  float2* part = nullptr;
  BLWS_TRY(ctx->get(BUF_TC_PART, total * sizeof(float2), (void**)&part));
  const OzPlanes* A[2] = {&Wr, &Wc};
  const OzPlanes* B[2] = {&Xv, &Xu};
  for (int t = 0; t < 2; ++t) {
    OzJob& J = jobs.job[t];
    BLWS_TRY(oz_encode(ctx, &J.a, A[t]->d, Ms[t], Ms[t], Ks[t], A[t]->ld, kOzBM));
    BLWS_TRY(oz_encode(ctx, &J.b, B[t]->d, b, npad, Ks[t], B[t]->ld, kOzBN));
    J.ea = A[t]->e;
    J.eb = B[t]->e;
    J.part = part + off[t];
    J.M = Ms[t];
    J.K = Ks[t];
    J.tiles = tiles[t];
    J.ngroups = ngroups;
    J.splits = splits[t];
    J.kchunk = kchunk[t];
    J.Mpad = tiles[t] * kOzBM;
    J.npad = npad;
  }
  double* scal = nullptr;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  jobs.blocks0 = tiles[0] * ngroups * splits[0];
  jobs.N = b;
  jobs.err = reinterpret_cast<int*>(scal + SLOT_TCERR);
  const int blocks = jobs.blocks0 + tiles[1] * ngroups * splits[1];
  const int bytes = (int)oz_smem_bytes();
  BLWS_TRY_CUDA(ctx, cudaFuncSetAttribute(oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  BLWS_TRY(ctx->time_begin(s));
  oz_kernel<<<blocks, kOzThreads, bytes, s>>>(jobs);
  BLWS_CHECK_LAUNCH(ctx);
  BLWS_TRY(ctx->time_end(s, 2.0 * m * n * b, 2));
  for (int t = 0; t < 2; ++t) {
    const size_t tot = (size_t)Ms[t] * b;
    const int G = oz_lanes(ctx->sms, tot, splits[t]);
    oz_reduce<<<(int)std::min<size_t>((tot * G + 255) / 256, (size_t)ctx->sms * 8), 256, 0, s>>>(
        Ms[t], b, npad, splits[t], jobs.job[t].Mpad, jobs.job[t].part, A[t]->e, B[t]->e,
        P + (t ? m : 0), ldp, 1.0, 0.0, 0, G);
    BLWS_CHECK_LAUNCH(ctx);
  }
  return BLWS_OK;
}

// C (M x N, ldc) = alpha op(A) op(B) + beta C with FP64-equivalent digit
// products (op(A) is M x K, op(B) K x N; column-major, op = transpose when
// ta / tb).  The rows of op(A) and the columns of op(B) are scaled and split
// into digit planes (from the contiguous side when the operand is transposed,
// by the tiled transpose otherwise), one job of the digit kernel covers the
// product, split along K to fill the GPU, and the FP64 reduction applies the
// scales, alpha and beta.
blws_status oz_gemm(Ctx* ctx, cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                    const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                    bool sym) {
  BLWS_TRY(oz_encoder(ctx));
  const int ngroups = ceil_div(N, kOzBN), npad = ngroups * kOzBN, ldk = oz_ld(K);
  const size_t pa = (size_t)kOzS * M * ldk, pb = (size_t)kOzS * npad * ldk;
  uint8_t* base = nullptr;
  const size_t bytes = (pa + pb) * sizeof(__nv_bfloat16) + ((size_t)M + npad + 64) * sizeof(int);
  BLWS_TRY(ctx->get(BUF_OZ_G, bytes, (void**)&base));
  __nv_bfloat16* da = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* db = da + pa;
  int* ea = reinterpret_cast<int*>(base + (pa + pb) * sizeof(__nv_bfloat16));
  int* eb = ea + M;
  const OzPlanes Ap{da, ea, M, K, ldk};
  const OzPlanes Bp{db, eb, npad, K, ldk};
  // A^T A (a Gram matrix): op(B)'s planes are op(A)'s, built once
  const bool same = ta && !tb && A == B && lda == ldb && M == N;
  if (same) {
    BLWS_TRY(oz_planes_from_cols(ctx, s, A, lda, 0, K, M, Ap));
  } else if (ta && !tb) {  // both from columns: one launch
    BLWS_TRY(planes_cols_pair(ctx, s, A, lda, 0, K, M, Ap, B, ldb, 0, K, N, Bp));
  } else {
    if (ta) BLWS_TRY(oz_planes_from_cols(ctx, s, A, lda, 0, K, M, Ap));
    else BLWS_TRY(oz_planes_from_rows(ctx, s, A, lda, M, K, Ap));
    if (!tb) BLWS_TRY(oz_planes_from_cols(ctx, s, B, ldb, 0, K, N, Bp));
    else BLWS_TRY(oz_planes_from_rows(ctx, s, B, ldb, N, K, OzPlanes{db, eb, npad, K, ldk}));
  }
  const __nv_bfloat16* bplanes = same ? da : db;
  const int* bexp = same ? ea : eb;
  const int brows = same ? M : npad;  // rows between op(B)'s planes
  const int tiles = ceil_div(M, kOzBM);
  const int kblocks = ceil_div(K, kOzBK);
  double* scal = nullptr;
  BLWS_TRY(ctx->get(BUF_SCAL, SLOT_MAX, &scal));
  const int smem = (int)oz_smem_bytes();
  BLWS_TRY(ctx->smem_limit(Ctx::ATTR_OZ, (const void*)oz_kernel, smem));
  // the digit kernel over `sp` splits of K and the FP64 reduction into C
  auto launch = [&](int sp, double* Cout, int ldo, double bet) -> blws_status {
    const int kchunk = ceil_div(kblocks, sp) * kOzBK;
    const int splits = ceil_div(K, kchunk);
    float2* part = nullptr;
    BLWS_TRY(ctx->get(BUF_TC_PART, (size_t)splits * npad * tiles * kOzBM * sizeof(float2), (void**)&part));
    OzJobs jobs;
    memset(&jobs, 0, sizeof(jobs));
    OzJob& J = jobs.job[0];
    BLWS_TRY(oz_encode(ctx, &J.a, da, M, M, K, ldk, kOzBM));
    // op(B) columns past N: zero digits from the copy's out-of-bounds fill
    BLWS_TRY(oz_encode(ctx, &J.b, bplanes, N, brows, K, ldk, kOzBN));
    J.ea = ea;
    J.eb = bexp;
    J.part = part;
    J.M = M;
    J.K = K;
    J.tiles = tiles;
    J.ngroups = ngroups;
    J.splits = splits;
    J.kchunk = kchunk;
    J.Mpad = tiles * kOzBM;
    J.npad = npad;
    jobs.job[1] = J;  // unused: every block belongs to job 0
    jobs.blocks0 = tiles * ngroups * splits;
    jobs.N = N;
    jobs.err = reinterpret_cast<int*>(scal + SLOT_TCERR);
    oz_kernel<<<jobs.blocks0, kOzThreads, smem, s>>>(jobs);
    BLWS_CHECK_LAUNCH(ctx);
    const size_t tot = (size_t)M * N;
    const int G = oz_lanes(ctx->sms, tot, splits);
    oz_reduce<<<(int)std::min<size_t>((tot * G + 255) / 256, (size_t)ctx->sms * 8), 256, 0, s>>>(
        M, N, npad, splits, J.Mpad, part, ea, bexp, Cout, ldo, alpha, bet,
        sym && M == N && bet == 0.0 ? 1 : 0, G);
    BLWS_CHECK_LAUNCH(ctx);
    return BLWS_OK;
  };
  int sp = oz_pick_splits(ctx->sms, tiles * ngroups, kblocks);
  if (ctx->cfg.tune) {
    // the split count from timing: the wave model above takes a fixed cost per
    // CTA, which the small products (b x b outputs, K in the thousands) miss
    // most; candidates are powers of two up to one K block per split and the
    // model's choice, each timed with its reduction into a scratch C
    const TuneKey key{{ctx->sms, kTuneDigits, ta, tb, sym, tune_bucket(M), tune_bucket(N), tune_bucket(K)}};
    TuneChoice c;
    if (tune_lookup(key, &c)) {
      sp = std::min(c.a, kblocks);
    } else if (ctx->capturing) {
      ctx->capture_broken = true;
      return ctx->fail(BLWS_ECUDA, "untuned digit-plane product shape inside a graph capture");
    } else {
      double* Cs = nullptr;
      BLWS_TRY(ctx->get(BUF_TUNE, (size_t)M * N, &Cs));
      std::vector<int> cand;
      for (int q = 1; q <= kblocks; q *= 2) cand.push_back(q);
      cand.push_back(sp);
      cudaEvent_t e0, e1;
      BLWS_TRY_CUDA(ctx, cudaEventCreate(&e0));
      if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ctx->fail(BLWS_ECUDA, "autotuner events");
      }
      float best_ms = -1.0f, rule_ms = -1.0f;
      int best = sp;
      blws_status st = BLWS_OK;
      for (size_t i = 0; i < cand.size() && st == BLWS_OK; ++i) {
        st = launch(cand[i], Cs, M, 0.0);  // warm-up
        if (st != BLWS_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) st = ctx->fail(BLWS_ECUDA, "autotuner event");
        for (int r = 0; r < 3 && st == BLWS_OK; ++r) st = launch(cand[i], Cs, M, 0.0);
        float ms = 0.0f;
        if (st == BLWS_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          st = ctx->fail(BLWS_ECUDA, "autotuner timing");
        if (st != BLWS_OK) break;
        if (cand[i] == sp) rule_ms = ms;
        if (best_ms < 0.0f || ms < best_ms) {
          best_ms = ms;
          best = cand[i];
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      BLWS_TRY(st);
      if (!(best_ms < 0.95f * rule_ms)) best = sp;  // keep the model's choice unless 5% slower
      tune_store(key, TuneChoice{best, 0});
      sp = best;
    }
  }
  return launch(sp, C, ldc, beta);
}

}  // namespace blws
