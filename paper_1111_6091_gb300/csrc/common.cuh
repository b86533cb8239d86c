// Shared definitions for the libcpmg CUDA sources (sm_103a only).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/cpmg.h"

#define CPMG_CUDA_TRY(expr)                                                     \
  do {                                                                          \
    cudaError_t _e = (expr);                                                    \
    if (_e != cudaSuccess) {                                                    \
      cpmg::set_last_error(_e, #expr, __FILE__, __LINE__);                      \
      return CPMG_CUDA_ERROR;                                                   \
    }                                                                           \
  } while (0)

#define CPMG_TRY(expr)                                                          \
  do {                                                                          \
    int _s = (expr);                                                            \
    if (_s != CPMG_OK) return _s;                                               \
  } while (0)

namespace cpmg {

void set_last_error(cudaError_t e, const char* what, const char* file, int line);

// Largest padded rank handled by the register-resident kernels.
constexpr int kMaxRank = CPMG_MAX_RANK;
constexpr int kMaxModes = CPMG_MAX_MODES;

// Padded rank used for register arrays: the smallest supported width >= R.
inline int padded_rank(int R) {
  if (R <= 2) return 2;
  if (R <= 4) return 4;
  if (R <= 6) return 6;
  if (R <= 8) return 8;
  if (R <= 10) return 10;
  if (R <= 12) return 12;
  return 16;
}

// Shape of one tensor level, as seen by the kernels.
struct Shape {
  int N = 0;
  int64_t dims[kMaxModes] = {0};
  int64_t numel() const {
    int64_t p = 1;
    for (int n = 0; n < N; ++n) p *= dims[n];
    return p;
  }
};

// Double-float helpers (a value is hi + lo with |lo| <= ulp(hi)/2).  Error-free
// transformations after Knuth (TwoSum) and the FMA form of Dekker's TwoProduct.
struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float err = __fsub_rn(b, __fsub_rn(s, a));
  return {s, err};
}

// (a.hi + a.lo) + (b.hi + b.lo)
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, lo);
}

// Exact product z*h as a double-float, plus z*l folded into the low part.
__device__ __forceinline__ df df_mul_f(float z, df a) {
  float p = __fmul_rn(z, a.hi);
  float e = __fmaf_rn(z, a.hi, -p);
  e = __fmaf_rn(z, a.lo, e);
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

__host__ __device__ __forceinline__ df df_from_double(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return {h, l};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace cpmg
