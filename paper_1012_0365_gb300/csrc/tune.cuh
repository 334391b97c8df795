// The autotuner's table (blws_config.tune): choices timed once per size
// bucket, kept process-wide and, when the environment variable
// BLWS_TUNE_FILE names a file, read from it at first use and appended to it
// as they are made.  The products that consult it (gemm_f64.cu, tc_ozaki.cu)
// time their own candidates.
#pragma once
#include "common.cuh"

namespace blws {

// v: the device's SM count, the kind of product (kTuneF64 / kTuneF32 for the
// CUDA-core GEMM by its arithmetic type, kTuneDigits for the digit-plane
// product), transposes, symmetry, and the bucketed dimensions
struct TuneKey {
  int v[8];
  bool operator<(const TuneKey& o) const {
    for (int i = 0; i < 8; ++i)
      if (v[i] != o.v[i]) return v[i] < o.v[i];
    return false;
  }
};
// CUDA-core GEMM: a = tile shape (0-4), b = K split (0-3); digit planes:
// a = K splits (>= 1), b unused (0)
struct TuneChoice {
  int a, b;
};
constexpr int kTuneF32 = 4, kTuneF64 = 8, kTuneDigits = 100;

// each dimension rounded up on a ladder of quarter octaves (exact up to 32)
int tune_bucket(int x);
bool tune_lookup(const TuneKey& k, TuneChoice* c);
void tune_store(const TuneKey& k, const TuneChoice& c);

}  // namespace blws
