// Batched CP-ALS: the relaxation sweep of Section 3 (A^(n) <- Z_(n) Phi^(n) (Gamma^(n))^+ for
// n = 1..N, then Eq. ALSnorm) on many independent, unevenly sized tensors at once, with the
// stopping test of Eq. gradConv per tensor.
//
// One cooperative, persistent kernel runs k whole sweeps of every active tensor followed by one
// g evaluation.  Inside it, phases are separated by a grid barrier (bounded wait):
//   units(n)   warps walk the list of MTTKRP work units of mode n of all tensors; a unit is
//              (tensor, block of 64 rows of the first mode, chunk of columns) and writes its
//              partial sums, in the sweep's arithmetic, to a slot of its own, so each tensor's
//              arithmetic is independent of what else is in the batch
//   rows(n)    one warp per output row: ordered reduction of the row's partials into M^(n)(i,:)
//              and the row of the R x R solve, A^(n)(i,:) = M^(n)(i,:) (Gamma^(n))^+
//   tensor(n)  one block per tensor: the float64 Gram of the new A^(n), Eq. ALSnorm after the
//              last mode (column norms from the Gram diagonals), and (Gamma^(n+1))^+ of the next
//              mode (Gauss-Jordan, or the eigen pseudoinverse when Gamma is singular)
//   eval       MTTKRPs of all modes in float64-accurate arithmetic, ||A Gamma - M||^2 per row
//              and mode, g, the stopping and precision-switch decisions, all on the device
// GB300's float64 pipe is narrow, so the float sweeps do no float64 arithmetic per column or per
// row: they read float-pair copies of the factors and of Gamma^+ that the kernel keeps next to
// the float64 ones, and sum in float (FP32) or float pairs (float64-accurate).  The Grams, the
// inverses and the g evaluation stay float64.  Unit sizes (elements per unit) come from a small
// autotuner that times candidate lists on the batch itself.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ctx.cuh"
#include "linalg.cuh"

namespace cpmg {

constexpr int kBR = 8;          // largest rank of the batched kernels (slots padded to 8)
constexpr int kBModes = 4;      // largest order
constexpr int kBRows = 64;      // first-mode rows per unit (two per lane)
constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kGramStride = kBR * kBR;

// BP_DELTA: float64-accurate sweeps computed as M = M_ref + Z_(n) (KR(A) - KR(A_ref)), with M_ref and
// A_ref from the tensor's last g evaluation (float-pair products) and the correction in FP32
enum { BP_FP32 = 0, BP_FP64 = 1, BP_DF = 3, BP_DELTA = 4 };
enum { BS_RUNNING = -1 };

// One problem of the batch (device copy; the kernel updates the state fields).
struct BTen {
  const void* Z;
  double* A[kBModes];
  float* Ah[kBModes];           // A as float pairs (hi, lo), same layout; kept when shadow != 0
  float* Al[kBModes];
  float* Rh[kBModes];           // A_ref as float pairs: the factors at the last g evaluation
  float* Rl[kBModes];
  double* mref;                 // M_ref^(n) of every mode at A_ref, row r of mode n at kBR (off_n + i)
  double* gram;                 // kBModes x 8 x 8
  double* ginv;                 // 8 x 8: (Gamma^(n))^+ of the next mode to update
  float* gih;                   // ginv as float pairs (8 x 8 each)
  float* gil;
  double* gam;                  // kBModes x 8 x 8: Gamma^(n) of every mode (g evaluation)
  double* rowres;               // per mode and row: ||A Gamma - M||^2, ||M||^2, <M, A> (g evaluation)
  double* part[kBModes];        // partial sums of the MTTKRP of each mode, in the phase's arithmetic
  int64_t dims[kBModes];
  int nk[kBModes];              // partial slots per output row (mode > 0) or column chunks (mode 0)
  int N, R, zf64;
  int prec, gprec;              // sweep / evaluation arithmetic
  int shadow;                   // 1: float sweeps (the float-pair copies are kept)
  int policy;                   // cpmg_precision of the request
  int active;
  int init;                     // 1: ||Z||^2, the Grams and the copies still to be computed
  int status;
  int iters, max_iters;
  int stall;
  int no_delta;                 // 1: delta sweeps stopped helping (g stalled): float pairs to the end
  int check_k;                  // sweeps between this tensor's g evaluations (0: the launch's sweeps)
  int next_check;               // iteration count at which its next evaluation is due
  double g_prev;                // g at its previous evaluation
  double znorm2;
  double tol, mixed_switch;
  double g, g_best, f;
  double res2[kBModes], m2[kBModes], zin;
};

struct BUnit {
  int t, mode, rb, k;
  int64_t c0, c1;               // column range (mode 0) or range of the columns sharing i_n
  int64_t in_idx;               // i_n (mode > 0)
};

// kBRowsPerItem consecutive output rows of one mode of one tensor (one warp per row)
constexpr int kBRowsPerItem = kBThreads / 32;
struct BRow {
  int t, mode;
  int64_t r0;
};

struct BArgs {
  BTen* ten;
  int nten;
  const BUnit* units[kBModes];
  int64_t nunits[kBModes];
  const BRow* rows[kBModes];    // row items per mode
  int64_t nrows[kBModes];
  int maxN;
  int nsweeps;
  int eval;                     // 1: evaluate g and decide; 2: MTTKRP phases only (autotuner)
  unsigned* bar;                // [0] arrivals, [1] generation
  unsigned bar_extra;           // 0; 1 only under the failure-detection test hook
  unsigned long long wait_ns;   // limit of each bounded barrier wait
  int* err;
  int* nactive;
};

// ------------------------------------------------------------------ arithmetic per precision
template <int P> struct BT;
template <> struct BT<BP_FP32> { using V = float; };
template <> struct BT<BP_FP64> { using V = double; };
template <> struct BT<BP_DF> { using V = df; };
template <> struct BT<BP_DELTA> { using V = float; };

template <typename V> __device__ __forceinline__ V bzero();
template <> __device__ __forceinline__ float bzero<float>() { return 0.f; }
template <> __device__ __forceinline__ double bzero<double>() { return 0.0; }
template <> __device__ __forceinline__ df bzero<df>() { return {0.f, 0.f}; }
template <typename V> __device__ __forceinline__ V bone();
template <> __device__ __forceinline__ float bone<float>() { return 1.f; }
template <> __device__ __forceinline__ double bone<double>() { return 1.0; }
template <> __device__ __forceinline__ df bone<df>() { return {1.f, 0.f}; }

__device__ __forceinline__ void bfma(float& acc, float z, float w) { acc = __fmaf_rn(z, w, acc); }
__device__ __forceinline__ void bfma(double& acc, float z, double w) { acc = __fma_rn((double)z, w, acc); }
__device__ __forceinline__ void bfma(double& acc, double z, double w) { acc = __fma_rn(z, w, acc); }
// float pairs: the exact product z * w.hi (rounded part and error) plus z * w.lo; the rounded
// parts are summed error-free into acc.hi (TwoSum) and every error term into acc.lo, which is
// folded back by bnorm after each batch of at most 32 columns
__device__ __forceinline__ void bfma(df& acc, float z, df w) {
  const float p = __fmul_rn(z, w.hi);
  float e = __fmaf_rn(z, w.hi, -p);
  e = __fmaf_rn(z, w.lo, e);
  const df s = df_two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ void bnorm(float&) {}
__device__ __forceinline__ void bnorm(double&) {}
__device__ __forceinline__ void bnorm(df& a) { a = df_two_sum(a.hi, a.lo); }

__device__ __forceinline__ float badd(float a, float b) { return a + b; }
__device__ __forceinline__ double badd(double a, double b) { return a + b; }
__device__ __forceinline__ df badd(df a, df b) { return df_add(a, b); }

__device__ __forceinline__ double bto_d(float x) { return (double)x; }
__device__ __forceinline__ double bto_d(double x) { return x; }
__device__ __forceinline__ double bto_d(df x) { return df_to_double(x); }

__device__ __forceinline__ float bshfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double bshfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df bshfl_xor(df v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ float bshfl(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ double bshfl(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ df bshfl(df v, int l) {
  return {__shfl_sync(0xffffffffu, v.hi, l), __shfl_sync(0xffffffffu, v.lo, l)};
}

// factor entry e of mode m in the arithmetic of V: the float copy (FP32), the float-pair copy
// (float64-accurate), or the float64 array
struct BFac {
  const double* a;
  const float* h;
  const float* l;
};
__device__ __forceinline__ void fac_get(const BFac& f, size_t e, float& v) { v = f.h[e]; }
__device__ __forceinline__ void fac_get(const BFac& f, size_t e, df& v) { v = {f.h[e], f.l[e]}; }
__device__ __forceinline__ void fac_get(const BFac& f, size_t e, double& v) { v = f.a[e]; }
__device__ __forceinline__ float bmul(float a, float b) { return a * b; }
__device__ __forceinline__ double bmul(double a, double b) { return a * b; }
__device__ __forceinline__ df bmul(df a, df b) { return df_mul(a, b); }

// Sum of v[r] over the 32 lanes of the warp, scattered: returns the total of component
// lane / (32 / RB).  log2(RB) halving exchanges, then a butterfly over the lanes holding the
// same component; the order is fixed, so the result is reproducible.
template <int RB, typename V>
__device__ __forceinline__ V warp_rs(V (&v)[RB], int lane) {
#pragma unroll
  for (int h = RB / 2, s = 16; h >= 1; h >>= 1, s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const V keep = up ? v[h + j] : v[j];
      const V give = up ? v[j] : v[h + j];
      v[j] = badd(keep, bshfl_xor(give, s));
    }
  }
  V x = v[0];
#pragma unroll
  for (int s = 16 / RB; s >= 1; s >>= 1) x = badd(x, bshfl_xor(x, s));
  return x;
}

// A^(m)(e) <- x, with the float-pair copy when the tensor keeps one
__device__ __forceinline__ void put_a(const BTen& T, int m, int64_t e, double x) {
  T.A[m][e] = x;
  if (T.shadow) {
    const df d = df_from_double(x);
    T.Ah[m][e] = d.hi;
    T.Al[m][e] = d.lo;
  }
}

// ------------------------------------------------------------------ grid barrier (bounded)
__device__ __forceinline__ uint64_t bclock() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Every CTA arrives once; the last of gridDim.x + extra arrivals releases the others.  extra is 0
// except under the failure-detection test hook, where 1 makes the barrier unreachable and every
// wait run out after wait_ns (the kernel then reports error bit 2 and returns).
__device__ bool grid_sync(unsigned* bar, int* err, unsigned extra, unsigned long long wait_ns) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x + extra - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = bclock();
      while (*gen == g) {
        if (bclock() - t0 > wait_ns) {
          atomicOr(err, 2);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// ------------------------------------------------------------------ MTTKRP unit (one warp)
// Rows r0..r0+63 of the first mode (two per lane) against 32 columns at a time: each lane forms
// the Khatri-Rao row of one column (components r < RB) into shared memory, then every lane
// accumulates its two tensor rows against the 32 rows, four columns' loads in flight at once.
// Index arithmetic is 32-bit (batched tensors hold fewer than 2^32 elements).
template <int P, typename TZ, int RB>
__device__ void unit_run(const BTen& T, const BUnit& u, int lane, void* wsv, uint32_t* wc) {
  using V = typename BT<P>::V;
  V* ws = reinterpret_cast<V*>(wsv);
  const int N = T.N, R = T.R, n = u.mode;
  uint32_t dims[kBModes];
  BFac fac[kBModes];
#pragma unroll
  for (int m = 0; m < kBModes; ++m) {
    dims[m] = (uint32_t)T.dims[m];
    fac[m] = {T.A[m], T.Ah[m], T.Al[m]};
  }
  const uint32_t I0 = dims[0];
  const TZ* Z = reinterpret_cast<const TZ*>(T.Z);
  uint32_t Lp = 1;
#pragma unroll
  for (int m = 1; m < kBModes; ++m)
    if (m < n) Lp *= dims[m];
  const uint32_t In = dims[n < kBModes ? n : 0];
  const uint32_t r0 = (uint32_t)u.rb * kBRows;
  const uint32_t rend = (r0 + kBRows < I0) ? r0 + kBRows : I0;
  const uint32_t c1 = (uint32_t)u.c1, inx = (uint32_t)u.in_idx;
  V acc[2][RB];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[q][r] = bzero<V>();
  const uint32_t i1a = r0 + lane, i1b = r0 + lane + 32;
  const bool va = i1a < rend, vb = i1b < rend;
  for (uint32_t jb = (uint32_t)u.c0; jb < c1; jb += 32) {
    const int cnt = (int)(c1 - jb < 32 ? c1 - jb : 32);
    if (lane < cnt) {
      const uint32_t j = jb + lane;
      const uint32_t col = (n == 0) ? j : (j % Lp) + Lp * (inx + In * (j / Lp));
      wc[lane] = col;
      V w[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) w[r] = bone<V>();
      uint32_t rem = col;
#pragma unroll
      for (int m = 1; m < kBModes; ++m) {
        if (m < N) {
          const uint32_t Im = dims[m];
          const uint32_t im = rem % Im;
          rem /= Im;
          if (m != n) {
#pragma unroll
            for (int r = 0; r < RB; ++r)
              if (r < R) {
                V a;
                fac_get(fac[m], im + (size_t)Im * r, a);
                w[r] = bmul(w[r], a);
              }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) ws[lane * RB + r] = (r < R) ? w[r] : bzero<V>();
    }
    __syncwarp();
    int jj = 0;
    if constexpr (sizeof(V) == 4 && sizeof(TZ) == 4) {
      // FP32 sweeps are latency-bound: 16 loads in flight per lane (8 columns) per group
      for (; jj + 8 <= cnt; jj += 8) {
        float za[8], zb[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const size_t base = (size_t)I0 * wc[jj + c];
          za[c] = va ? (float)Z[base + i1a] : 0.f;
          zb[c] = vb ? (float)Z[base + i1b] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            const V wr = ws[(jj + c) * RB + r];
            bfma(acc[0][r], za[c], wr);
            bfma(acc[1][r], zb[c], wr);
          }
        }
      }
    }
    for (; jj + 4 <= cnt; jj += 4) {
      TZ za[4], zb[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const size_t base = (size_t)I0 * wc[jj + c];
        za[c] = va ? Z[base + i1a] : TZ(0);
        zb[c] = vb ? Z[base + i1b] : TZ(0);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const V wr = ws[(jj + c) * RB + r];
          bfma(acc[0][r], za[c], wr);
          bfma(acc[1][r], zb[c], wr);
        }
      }
    }
    for (; jj < cnt; ++jj) {
      const size_t base = (size_t)I0 * wc[jj];
      const TZ za = va ? Z[base + i1a] : TZ(0);
      const TZ zb = vb ? Z[base + i1b] : TZ(0);
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const V wr = ws[jj * RB + r];
        bfma(acc[0][r], za, wr);
        bfma(acc[1][r], zb, wr);
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < RB; ++r) bnorm(acc[q][r]);
    __syncwarp();
  }
  if (n == 0) {
    V* Pp = reinterpret_cast<V*>(T.part[0]) + (size_t)u.k * I0 * kBR;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint32_t i1 = q ? i1b : i1a;
      if (q ? vb : va)
#pragma unroll
        for (int r = 0; r < RB; ++r) Pp[(size_t)i1 * kBR + r] = acc[q][r];
    }
  } else {
    // contract the rows with A^(1): t[r] = sum_i1 A^(1)(i1, r) acc(i1, r), then over the warp
    V t[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      V s = bzero<V>();
      if (r < R) {
        V a;
        if (va) {
          fac_get(fac[0], i1a + (size_t)I0 * r, a);
          s = bmul(a, acc[0][r]);
        }
        if (vb) {
          fac_get(fac[0], i1b + (size_t)I0 * r, a);
          s = badd(s, bmul(a, acc[1][r]));
        }
      }
      t[r] = s;
    }
    const V tot = warp_rs<RB>(t, lane);
    constexpr int G = 32 / RB;
    if (lane % G == 0) {
      V* Pp = reinterpret_cast<V*>(T.part[n]) + ((size_t)u.in_idx * T.nk[n] + u.k) * kBR;
      Pp[lane / G] = tot;
    }
  }
}

// MTTKRP unit of a delta sweep (BP_DELTA, float tensors): the Khatri-Rao rows of the current factors
// and of A_ref are formed in float pairs and their difference is rounded to float; the products with
// Z accumulate in FP32.  Their rounding scales with the factor change since A_ref, not with M.  For
// mode n > 0 the unit also carries mode 1: A1 W - A1ref Wref = A1 (W - Wref) + (A1 - A1ref) Wref, so
// each FP32 sum is multiplied by a small factor or is small itself.
template <int RB>
__device__ void unit_run_delta(const BTen& T, const BUnit& u, int lane, void* wsv, uint32_t* wc) {
  float2* ws = reinterpret_cast<float2*>(wsv);  // (W - Wref, Wref) per column and rank
  const int N = T.N, R = T.R, n = u.mode;
  uint32_t dims[kBModes];
#pragma unroll
  for (int m = 0; m < kBModes; ++m) dims[m] = (uint32_t)T.dims[m];
  const uint32_t I0 = dims[0];
  const float* Z = reinterpret_cast<const float*>(T.Z);
  uint32_t Lp = 1;
#pragma unroll
  for (int m = 1; m < kBModes; ++m)
    if (m < n) Lp *= dims[m];
  const uint32_t In = dims[n < kBModes ? n : 0];
  const uint32_t r0 = (uint32_t)u.rb * kBRows;
  const uint32_t rend = (r0 + kBRows < I0) ? r0 + kBRows : I0;
  const uint32_t c1 = (uint32_t)u.c1, inx = (uint32_t)u.in_idx;
  float acc1[2][RB], acc2[2][RB];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int r = 0; r < RB; ++r) acc1[q][r] = acc2[q][r] = 0.f;
  const uint32_t i1a = r0 + lane, i1b = r0 + lane + 32;
  const bool va = i1a < rend, vb = i1b < rend;
  for (uint32_t jb = (uint32_t)u.c0; jb < c1; jb += 32) {
    const int cnt = (int)(c1 - jb < 32 ? c1 - jb : 32);
    if (lane < cnt) {
      const uint32_t j = jb + lane;
      const uint32_t col = (n == 0) ? j : (j % Lp) + Lp * (inx + In * (j / Lp));
      wc[lane] = col;
      df w[RB], wr[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) w[r] = wr[r] = df{1.f, 0.f};
      uint32_t rem = col;
#pragma unroll
      for (int m = 1; m < kBModes; ++m) {
        if (m < N) {
          const uint32_t Im = dims[m];
          const uint32_t im = rem % Im;
          rem /= Im;
          if (m != n) {
#pragma unroll
            for (int r = 0; r < RB; ++r)
              if (r < R) {
                const size_t e = im + (size_t)Im * r;
                w[r] = df_mul(w[r], df{T.Ah[m][e], T.Al[m][e]});
                wr[r] = df_mul(wr[r], df{T.Rh[m][e], T.Rl[m][e]});
              }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const df d = df_add(w[r], df{-wr[r].hi, -wr[r].lo});
        ws[lane * RB + r] = r < R ? make_float2(__fadd_rn(d.hi, d.lo), __fadd_rn(wr[r].hi, wr[r].lo))
                                  : make_float2(0.f, 0.f);
      }
    }
    __syncwarp();
    int jj = 0;
    for (; jj + 8 <= cnt; jj += 8) {  // 16 loads in flight per lane, as the FP32 sweep
      float za[8], zb[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const size_t base = (size_t)I0 * wc[jj + c];
        za[c] = va ? Z[base + i1a] : 0.f;
        zb[c] = vb ? Z[base + i1b] : 0.f;
      }
#pragma unroll
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const float2 wv = ws[(jj + c) * RB + r];
          acc1[0][r] = __fmaf_rn(za[c], wv.x, acc1[0][r]);
          acc1[1][r] = __fmaf_rn(zb[c], wv.x, acc1[1][r]);
          if (n != 0) {
            acc2[0][r] = __fmaf_rn(za[c], wv.y, acc2[0][r]);
            acc2[1][r] = __fmaf_rn(zb[c], wv.y, acc2[1][r]);
          }
        }
    }
    for (; jj < cnt; ++jj) {
      const size_t base = (size_t)I0 * wc[jj];
      const float za = va ? Z[base + i1a] : 0.f;
      const float zb = vb ? Z[base + i1b] : 0.f;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const float2 wv = ws[jj * RB + r];
        acc1[0][r] = __fmaf_rn(za, wv.x, acc1[0][r]);
        acc1[1][r] = __fmaf_rn(zb, wv.x, acc1[1][r]);
        if (n != 0) {
          acc2[0][r] = __fmaf_rn(za, wv.y, acc2[0][r]);
          acc2[1][r] = __fmaf_rn(zb, wv.y, acc2[1][r]);
        }
      }
    }
    __syncwarp();
  }
  if (n == 0) {
    float* Pp = reinterpret_cast<float*>(T.part[0]) + (size_t)u.k * I0 * kBR;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint32_t i1 = q ? i1b : i1a;
      if (q ? vb : va)
#pragma unroll
        for (int r = 0; r < RB; ++r) Pp[(size_t)i1 * kBR + r] = acc1[q][r];
    }
  } else {
    float t[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      float sum = 0.f;
      if (r < R) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (!(q ? vb : va)) continue;
          const size_t e = (q ? i1b : i1a) + (size_t)I0 * r;
          const float ah = T.Ah[0][e], al = T.Al[0][e];
          const float da = __fadd_rn(__fsub_rn(ah, T.Rh[0][e]), __fsub_rn(al, T.Rl[0][e]));
          sum = __fmaf_rn(__fadd_rn(ah, al), acc1[q][r], sum);
          sum = __fmaf_rn(da, acc2[q][r], sum);
        }
      }
      t[r] = sum;
    }
    const float tot = warp_rs<RB>(t, lane);
    constexpr int G = 32 / RB;
    if (lane % G == 0) {
      float* Pp = reinterpret_cast<float*>(T.part[n]) + ((size_t)u.in_idx * T.nk[n] + u.k) * kBR;
      Pp[lane / G] = tot;
    }
  }
}

struct BSmem {
  double ws[kBWarps][32 * kBR];   // Khatri-Rao rows of 32 columns (float / double / float pairs)
  uint32_t wc[kBWarps][32];
  double G[kBR * kBR], Pi[kBR * kBR], V[kBR * kBR], w[kBR];
  double red[3][kBThreads];
  double sc[kBModes][kBR];
  int fail;
};

template <int P, typename TZ>
__device__ __forceinline__ void unit_dispatch(const BTen& T, const BUnit& u, int lane, void* ws, uint32_t* wc) {
  if (T.R <= 4) unit_run<P, TZ, 4>(T, u, lane, ws, wc);
  else unit_run<P, TZ, 8>(T, u, lane, ws, wc);
}

// The g evaluation of a launch covers the active tensors whose own check is due (or that reached
// their sweep cap); the others only sweep.
__device__ __forceinline__ bool eval_due(const BTen& T) {
  return T.active && (T.iters >= T.next_check || (T.max_iters > 0 && T.iters >= T.max_iters));
}

__device__ void phase_units(const BArgs& a, int n, bool eval, BSmem& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kBWarps + warp, nw = (int64_t)gridDim.x * kBWarps;
  for (int64_t ui = gw; ui < a.nunits[n]; ui += nw) {
    const BUnit u = a.units[n][ui];
    const BTen& T = a.ten[u.t];
    if (!T.active || (eval && !eval_due(T))) continue;
    const int p = eval ? T.gprec : T.prec;
    if (T.zf64) unit_dispatch<BP_FP64, double>(T, u, lane, sm.ws[warp], sm.wc[warp]);
    else if (p == BP_FP32) unit_dispatch<BP_FP32, float>(T, u, lane, sm.ws[warp], sm.wc[warp]);
    else if (p == BP_DELTA) {
      if (T.R <= 4) unit_run_delta<4>(T, u, lane, sm.ws[warp], sm.wc[warp]);
      else unit_run_delta<8>(T, u, lane, sm.ws[warp], sm.wc[warp]);
    }
    else if (p == BP_DF) unit_dispatch<BP_DF, float>(T, u, lane, sm.ws[warp], sm.wc[warp]);
    else unit_dispatch<BP_FP64, float>(T, u, lane, sm.ws[warp], sm.wc[warp]);
  }
}

// deterministic block sum of one value per thread: a fixed butterfly inside each warp, then the
// warp sums in warp order (13 dependent float64 adds at 256 threads instead of 256; GB300's float64
// add latency is tens of cycles)
__device__ double bblock_sum(double v, double* buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) buf[warp] = v;
  __syncthreads();
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double s = buf[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) s += buf[k];
    tot = s;
  }
  __syncthreads();
  const double r = tot;
  __syncthreads();
  return r;
}

// stripe-parallel Gram of A (I x R, column-major) into gram (row stride kBR), fixed order:
// rows are split into stripes summed in parallel, then the stripes in order (GB300's float64
// units have long dependent latencies, so the chains stay short)
__device__ void gram_rows(const double* A, int64_t I, int R, double* gram, double* buf) {
  const int npairs = R * (R + 1) / 2;
  const int stripes = (int)blockDim.x / npairs > 0 ? (int)blockDim.x / npairs : 1;
  const int t = threadIdx.x;
  if (t < stripes * npairs) {
    const int p = t % npairs, sidx = t / npairs;
    int r = 0, q = p;
    while (q >= R - r) {
      q -= R - r;
      ++r;
    }
    const int c = r + q;
    double acc = 0.0;
    for (int64_t i = sidx; i < I; i += stripes) acc = __fma_rn(A[i + I * r], A[i + I * c], acc);
    buf[t] = acc;
  }
  __syncthreads();
  for (int p = t; p < npairs; p += blockDim.x) {
    int r = 0, q = p;
    while (q >= R - r) {
      q -= R - r;
      ++r;
    }
    const int c = r + q;
    double acc = 0.0;
    for (int k = 0; k < stripes; ++k) acc += buf[k * npairs + p];
    gram[r * kBR + c] = acc;
    gram[c * kBR + r] = acc;
  }
  __syncthreads();
}

// singular Gamma (thread 0): Pi = Gamma^+ from a symmetric eigendecomposition
__device__ __noinline__ void bpinv(const double* G, double* Pi, double* V, double* w, int R) {
  const double eps = 2.220446049250313e-16;
  double Gc[kBR * kBR];
  for (int i = 0; i < R * R; ++i) Gc[i] = G[i];
  jacobi_eig_dev(Gc, V, w, R);
  double wmax = 0.0;
  for (int i = 0; i < R; ++i) wmax = fmax(wmax, fabs(w[i]));
  const double cut = R * eps * wmax;
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < R; ++j) {
      double s = 0.0;
      for (int k = 0; k < R; ++k)
        if (fabs(w[k]) > cut) s += V[i * R + k] * V[j * R + k] / w[k];
      Pi[i * R + j] = s;
    }
}

// T.ginv = (Gamma^(n))^+ with Gamma^(n) the Hadamard product of the other Grams (block-wide),
// plus its float-pair copy for the float sweeps
__device__ void gamma_inverse(BTen& T, int n, BSmem& sm) {
  const int R = T.R, N = T.N;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) v *= T.gram[m * kGramStride + (e / R) * kBR + (e % R)];
    sm.G[e] = v;
    sm.Pi[e] = v;
  }
  __syncthreads();
  double dmax = 0.0;
  for (int i = 0; i < R; ++i) dmax = fmax(dmax, sm.G[i * R + i]);
  const double thresh = R * 2.220446049250313e-16 * (dmax > 0 ? dmax : 1.0);
  if (!gj_inverse(sm.Pi, R, thresh, &sm.fail) && threadIdx.x == 0) bpinv(sm.G, sm.Pi, sm.V, sm.w, R);
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int o = (e / R) * kBR + (e % R);
    T.ginv[o] = sm.Pi[e];
    if (T.shadow) {
      const df d = df_from_double(sm.Pi[e]);
      T.gih[o] = d.hi;
      T.gil[o] = d.lo;
    }
  }
  __syncthreads();
}

// Gamma^(n) of every mode (for the residuals of the g evaluation; block-wide)
__device__ void gamma_all(BTen& T) {
  const int R = T.R, N = T.N;
  for (int e = threadIdx.x; e < N * R * R; e += blockDim.x) {
    const int n = e / (R * R), rc = e % (R * R), r = rc / R, c = rc % R;
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) v *= T.gram[m * kGramStride + r * kBR + c];
    T.gam[n * kGramStride + r * kBR + c] = v;
  }
}

// Eq. ALSnorm with the column norms taken from the Gram diagonals (block-wide)
__device__ void normalize_tensor(BTen& T, BSmem& sm) {
  const int R = T.R, N = T.N, tid = threadIdx.x;
  for (int e = tid; e < N * R; e += blockDim.x) {
    const int m = e / R, r = e % R;
    sm.V[e] = sqrt(T.gram[m * kGramStride + r * kBR + r]);
  }
  __syncthreads();
  if (tid < R) {
    double prod = 1.0;
    for (int m = 0; m < N; ++m) prod *= sm.V[m * R + tid];
    const double lam = nth_root(prod, N);
    for (int m = 0; m < N; ++m) {
      const double nr = sm.V[m * R + tid];
      sm.sc[m][tid] = nr > 0 ? lam / nr : 1.0;
    }
  }
  __syncthreads();
  for (int m = 0; m < N; ++m) {
    const int Im = (int)T.dims[m];
    for (int e = tid; e < Im * R; e += blockDim.x) put_a(T, m, e, T.A[m][e] * sm.sc[m][e / Im]);
    for (int e = tid; e < R * R; e += blockDim.x) {
      const int r = e / R, c = e % R;
      T.gram[m * kGramStride + r * kBR + c] *= sm.sc[m][r] * sm.sc[m][c];
    }
  }
  __syncthreads();
  if (tid == 0) T.iters += 1;
  __syncthreads();
}

// gi(k, r) times m_k: float-pair products for the float sweeps
__device__ __forceinline__ df gi_mul(float m, const BTen& T, int o) { return df_mul_f(m, df{T.gih[o], T.gil[o]}); }
__device__ __forceinline__ df gi_mul(df m, const BTen& T, int o) { return df_mul(m, df{T.gih[o], T.gil[o]}); }

// Row i of mode n (one warp).  The lanes sum the row's partial slots lane, lane + 32, ... in
// the phase's arithmetic and scatter-reduce them (lane holds component lane / (32 / RB)).
// update: the ALS row A(i,:) = M(i,:) Gamma^+, lane r forming component r (float pairs for the
// float sweeps, float64 for FP64).  !update: the row's contributions to ||A Gamma - M||^2,
// ||M||^2 and <M, A> in float64, stored per row for an ordered sum.
template <int P, int RB>
__device__ void row_one(const BTen& T, int n, int64_t i, int lane, bool update) {
  using V = typename BT<P>::V;
  constexpr int G = 32 / RB;
  const int R = T.R, N = T.N;
  const int64_t In = T.dims[n];
  const int nk = T.nk[n];
  const V* base;
  size_t stride;
  if (n == 0) {
    base = reinterpret_cast<const V*>(T.part[0]) + (size_t)i * kBR;
    stride = (size_t)In * kBR;
  } else {
    base = reinterpret_cast<const V*>(T.part[n]) + (size_t)i * nk * kBR;
    stride = kBR;
  }
  V m[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) m[r] = bzero<V>();
  for (int k = lane; k < nk; k += 32) {
    const V* p = base + (size_t)k * stride;
#pragma unroll
    for (int r = 0; r < RB; ++r) m[r] = badd(m[r], p[r]);
  }
  const V mine = warp_rs<RB>(m, lane);
  if (update) {
    V mk[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) mk[k] = bshfl(mine, k * G);
    if (lane < R) {
      const int64_t e = i + In * lane;
      if constexpr (P == BP_FP64) {
        double x = 0.0;
#pragma unroll
        for (int k = 0; k < RB; ++k)
          if (k < R) x = __fma_rn(mk[k], T.ginv[k * kBR + lane], x);
        T.A[n][e] = x;
      } else if constexpr (P == BP_DELTA) {
        // M = M_ref + the FP32 correction, then A(i,:) = M Gamma^+ in float pairs
        int64_t off = 0;
        for (int q = 0; q < n; ++q) off += T.dims[q];
        const double* mr = T.mref + (size_t)kBR * (off + i);
        df x = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < RB; ++k)
          if (k < R) x = df_add(x, gi_mul(df_add(df_from_double(mr[k]), df{mk[k], 0.f}), T, k * kBR + lane));
        T.A[n][e] = df_to_double(x);
        T.Ah[n][e] = x.hi;
        T.Al[n][e] = x.lo;
      } else {
        df x = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < RB; ++k)
          if (k < R) x = df_add(x, gi_mul(mk[k], T, k * kBR + lane));
        T.A[n][e] = df_to_double(x);
        T.Ah[n][e] = x.hi;
        T.Al[n][e] = x.lo;
      }
    }
  } else {
    const V mv = bshfl(mine, (lane < RB ? lane : 0) * G);
    double res = 0.0, mm = 0.0, zi = 0.0;
    if (lane < R) {
      const double* A = T.A[n];
      const double* gm = T.gam + n * kGramStride;
      double ag = 0.0;
      for (int k = 0; k < R; ++k) ag = __fma_rn(A[i + In * k], gm[k * kBR + lane], ag);
      const double mr = bto_d(mv);
      const double d = ag - mr;
      res = d * d;
      mm = mr * mr;
      zi = mr * A[i + In * lane];
      if (T.policy == CPMG_PREC_MIXED && T.shadow && (T.prec == BP_DF || T.prec == BP_DELTA) && !T.no_delta) {
        // this evaluation's products become the reference of the delta sweeps that follow
        int64_t off = 0;
        for (int q = 0; q < n; ++q) off += T.dims[q];
        T.mref[(size_t)kBR * (off + i) + lane] = mr;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      res += __shfl_xor_sync(0xffffffffu, res, o);
      mm += __shfl_xor_sync(0xffffffffu, mm, o);
      zi += __shfl_xor_sync(0xffffffffu, zi, o);
    }
    if (lane == 0) {
      int64_t off = 0;
      for (int q = 0; q < n; ++q) off += T.dims[q];
      double* rr = T.rowres + 3 * (off + i);
      rr[0] = res;
      rr[1] = mm;
      rr[2] = zi;
    }
  }
  (void)N;
}

template <int P>
__device__ __forceinline__ void row_dispatch(const BTen& T, int n, int64_t i, int lane, bool update) {
  if (T.R <= 4) row_one<P, 4>(T, n, i, lane, update);
  else row_one<P, 8>(T, n, i, lane, update);
}

// row items of mode n (or of every mode for the g evaluation): one warp per row
__device__ void phase_rows(const BArgs& a, const BRow* items, int64_t nitems, bool update) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BRow rw = items[it];
    const BTen& T = a.ten[rw.t];
    if (!T.active || (!update && !eval_due(T))) continue;
    const int n = rw.mode;
    const int64_t i = rw.r0 + warp;
    if (i >= T.dims[n]) continue;
    const int p = update ? T.prec : T.gprec;
    if (T.zf64 || p == BP_FP64) row_dispatch<BP_FP64>(T, n, i, lane, update);
    else if (p == BP_DF) row_dispatch<BP_DF>(T, n, i, lane, update);
    else if (p == BP_DELTA) row_dispatch<BP_DELTA>(T, n, i, lane, update);
    else row_dispatch<BP_FP32>(T, n, i, lane, update);
  }
}

__device__ void check_tensor(BTen& T, int* nactive, int launch_k, BSmem& sm) {
  const bool take_ref =
      T.policy == CPMG_PREC_MIXED && T.shadow && (T.prec == BP_DF || T.prec == BP_DELTA) && !T.no_delta;
  if (take_ref)  // A_ref: the factors this evaluation's products (M_ref, stored by the rows) belong to
    for (int m = 0; m < T.N; ++m)
      for (int64_t e = threadIdx.x; e < T.dims[m] * T.R; e += blockDim.x) {
        T.Rh[m][e] = T.Ah[m][e];
        T.Rl[m][e] = T.Al[m][e];
      }
  // sum over (r, c) of prod_n Upsilon^(n)_{rc} = ||[[A]]||^2, spread over threads
  double part = 0.0;
  for (int e = threadIdx.x; e < T.R * T.R; e += blockDim.x) {
    const int r = e / T.R, c = e % T.R;
    double p = 1.0;
    for (int n = 0; n < T.N; ++n) p *= T.gram[n * kGramStride + r * kBR + c];
    part += p;
  }
  const double cross = bblock_sum(part, sm.red[0]);
  // per-mode sums of the row contributions, in row order within stripes
  int64_t off = 0;
  for (int n = 0; n < T.N; ++n) {
    const int64_t In = T.dims[n];
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
    for (int64_t i = threadIdx.x; i < In; i += blockDim.x) {
      const double* rr = T.rowres + 3 * (off + i);
      r0 += rr[0];
      r1 += rr[1];
      r2 += rr[2];
    }
    const double s0 = bblock_sum(r0, sm.red[0]);
    const double s1 = bblock_sum(r1, sm.red[1]);
    const double s2 = bblock_sum(r2, sm.red[2]);
    if (threadIdx.x == 0) {
      T.res2[n] = s0;
      T.m2[n] = s1;
      if (n == T.N - 1) T.zin = s2;
    }
    off += In;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double g2 = 0.0, m2 = 0.0;
  for (int n = 0; n < T.N; ++n) {
    g2 += T.res2[n];
    m2 += T.m2[n];
  }
  const double zn = sqrt(T.znorm2);
  const double g = sqrt(g2) / zn;
  T.f = 0.5 * (T.znorm2 - 2.0 * T.zin + cross);
  T.g = g;
  if (!isfinite(g)) {
    T.status = CPMG_NUMERIC;
    T.active = 0;
  } else if (g < T.tol) {
    T.status = CPMG_OK;
    T.active = 0;
  } else if (T.max_iters > 0 && T.iters >= T.max_iters) {
    T.status = CPMG_NOT_CONVERGED;
    T.active = 0;
  } else if (T.policy == CPMG_PREC_MIXED && T.prec == BP_FP32) {
    // float sweeps stop helping once g nears their rounding floor, or stop improving
    const double floor_g = T.mixed_switch * 5.960464477539063e-08 * sqrt(m2) / zn;
    if (T.g_best < 0 || g < T.g_best) {
      T.g_best = g;
      T.stall = 0;
    } else {
      T.stall += 1;
    }
    if (g < floor_g || T.stall >= 20) {
      T.prec = BP_DF;
      T.g_best = -1.0;
      T.stall = 0;
    }
  } else if (take_ref) {
    // refined: delta sweeps from the reference just taken, as long as they keep lowering g
    if (T.g_best < 0 || g < T.g_best) {
      T.g_best = g;
      T.stall = 0;
    } else {
      T.stall += 1;
    }
    if (T.stall >= 3) {
      T.no_delta = 1;
      T.prec = BP_DF;
    } else {
      T.prec = BP_DELTA;
    }
  }
  if (T.active && T.policy == CPMG_PREC_MIXED) {
    // the next check's g: FP32 products while the tensor sweeps in FP32 and g is more than 64 times
    // its FP32 floor (the rounding is then a few percent of g at most); float-pair accurate from
    // there on, so the switch and the stopping test always see an accurate g
    const double floor_g = T.mixed_switch * 5.960464477539063e-08 * sqrt(m2) / zn;
    T.gprec = (T.prec == BP_FP32 && g > 64.0 * floor_g) ? BP_FP32 : BP_DF;
  }
  if (T.active) {
    // next interval: about half the sweeps the observed rate predicts are left, a power-of-two
    // multiple of the launch's sweeps, at most 32 (and the launch's sweeps while g is not falling)
    int k = launch_k;
    if (T.g_prev > 0.0 && g < T.g_prev && T.tol > 0.0 && g > T.tol) {
      const int kp = T.check_k > 0 ? T.check_k : launch_k;
      const double left = kp * log(T.tol / g) / log(g / T.g_prev);
      while (2 * k <= 32 && 2 * k <= 0.5 * left) k *= 2;
    }
    T.check_k = k;
    T.next_check = T.iters + k;
    T.g_prev = g;
    atomicAdd(nactive, 1);
  }
}

__global__ void __launch_bounds__(kBThreads, 2) k_batch(BArgs a) {
  __shared__ BSmem sm;
  bool ok = true;
  for (int sw = 0; sw < a.nsweeps && ok; ++sw) {
    for (int n = 0; n < a.maxN && ok; ++n) {
      if (n == 0) phase_units(a, 0, false, sm);  // later modes' units ran after the previous tensor phase
      ok = grid_sync(a.bar, a.err, a.bar_extra, a.wait_ns);
      if (ok) phase_rows(a, a.rows[n], a.nrows[n], true);
      ok = ok && grid_sync(a.bar, a.err, a.bar_extra, a.wait_ns);
      // per tensor: the Gram of the new A^(n); after the last mode Eq. ALSnorm; then Gamma^+
      // of the next mode to update
      for (int t = blockIdx.x; t < a.nten && ok; t += gridDim.x) {
        BTen& T = a.ten[t];
        if (!T.active || n >= T.N) continue;
        gram_rows(T.A[n], T.dims[n], T.R, T.gram + n * kGramStride, sm.red[0]);
        const bool last_mode = n == T.N - 1;
        if (last_mode) normalize_tensor(T, sm);
        gamma_inverse(T, last_mode ? 0 : n + 1, sm);
      }
      // Mode n+1's MTTKRP units need the factors as the rows phase left them; a tensor's tensor
      // phase changes its factors only after its last mode (Eq. ALSnorm), and such a tensor has
      // no units of mode n+1.  So each CTA goes on to its share of those units without a grid
      // barrier; Gamma^+ of mode n+1 is read only by the rows phase, after the next barrier.  The
      // sweep boundary keeps its barrier: every normalization precedes the next sweep's units.
      if (ok && n + 1 < a.maxN) phase_units(a, n + 1, false, sm);
      else ok = ok && grid_sync(a.bar, a.err, a.bar_extra, a.wait_ns);
    }
  }
  if (a.eval && ok) {
    for (int n = 0; n < a.maxN; ++n) phase_units(a, n, a.eval == 1, sm);
    if (a.eval == 1)
      for (int t = blockIdx.x; t < a.nten; t += gridDim.x)
        if (eval_due(a.ten[t])) gamma_all(a.ten[t]);
    ok = grid_sync(a.bar, a.err, a.bar_extra, a.wait_ns);
    if (a.eval == 1 && ok) {
      for (int n = 0; n < a.maxN; ++n) phase_rows(a, a.rows[n], a.nrows[n], false);
      ok = grid_sync(a.bar, a.err, a.bar_extra, a.wait_ns);
      for (int t = blockIdx.x; t < a.nten && ok; t += gridDim.x) {
        BTen& T = a.ten[t];
        if (!T.active) continue;
        if (!eval_due(T)) {  // still running, evaluated at a later launch
          if (threadIdx.x == 0) atomicAdd(a.nactive, 1);
          continue;
        }
        check_tensor(T, a.nactive, a.nsweeps, sm);
        __syncthreads();
      }
    }
  }
}

// ------------------------------------------------------------------ setup / final kernels
// ||Z||^2, the Grams, the float-pair copies and Gamma^(1)^+ of every tensor still to initialize
// (block per tensor)
__global__ void __launch_bounds__(kBThreads) k_batch_init(BTen* ten, int nten) {
  __shared__ BSmem sm;
  __shared__ double buf[kBThreads];
  for (int t = blockIdx.x; t < nten; t += gridDim.x) {
    BTen& T = ten[t];
    if (!T.init) continue;
    int64_t P = 1;
    for (int m = 0; m < T.N; ++m) P *= T.dims[m];
    // ||Z||^2: float tensors square and sum in float pairs (exact products, error-free sums),
    // four loads in flight per thread
    double s = 0.0;
    if (T.zf64) {
      const double* Zd = reinterpret_cast<const double*>(T.Z);
      for (int64_t e = threadIdx.x; e < P; e += blockDim.x) s += Zd[e] * Zd[e];
    } else {
      const float* Zf = reinterpret_cast<const float*>(T.Z);
      df acc = {0.f, 0.f};
      for (int64_t e0 = threadIdx.x; e0 < P; e0 += 4 * (int64_t)blockDim.x) {
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int64_t e = e0 + (int64_t)k * blockDim.x;
          v[k] = e < P ? Zf[e] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc = df_add(acc, df_mul_f(v[k], {v[k], 0.f}));
      }
      s = df_to_double(acc);
    }
    const double zz = bblock_sum(s, buf);
    for (int m = 0; m < T.N; ++m) {
      gram_rows(T.A[m], T.dims[m], T.R, T.gram + m * kGramStride, buf);
      if (T.shadow)
        for (int64_t e = threadIdx.x; e < T.dims[m] * T.R; e += blockDim.x) put_a(T, m, e, T.A[m][e]);
    }
    gamma_inverse(T, 0, sm);
    if (threadIdx.x == 0) {
      T.znorm2 = zz;
      T.init = 0;
    }
    __syncthreads();
  }
}

// sort the rank-one terms by decreasing lambda (ties keep their order), end of Section 3
__global__ void __launch_bounds__(kBThreads) k_batch_sort(BTen* ten, const int* idx, int count) {
  __shared__ int perm[kBR];
  __shared__ double tmp[kBThreads];
  for (int q = blockIdx.x; q < count; q += gridDim.x) {
    BTen& T = ten[idx[q]];
    const int R = T.R, N = T.N;
    if (threadIdx.x == 0) {
      double lam[kBR];
      for (int r = 0; r < R; ++r) {
        double p = 1.0;
        for (int m = 0; m < N; ++m) {
          const int64_t Im = T.dims[m];
          double s = 0.0;
          for (int64_t i = 0; i < Im; ++i) s += T.A[m][i + Im * r] * T.A[m][i + Im * r];
          p *= sqrt(s);
        }
        lam[r] = nth_root(p, N);
        perm[r] = r;
      }
      for (int i = 1; i < R; ++i) {  // stable insertion sort, decreasing
        const int pi = perm[i];
        int j = i - 1;
        while (j >= 0 && lam[perm[j]] < lam[pi]) {
          perm[j + 1] = perm[j];
          --j;
        }
        perm[j + 1] = pi;
      }
    }
    __syncthreads();
    for (int m = 0; m < N; ++m) {
      const int64_t Im = T.dims[m];
      for (int64_t i0 = 0; i0 < Im; i0 += blockDim.x / kBR) {
        const int64_t i = i0 + threadIdx.x / kBR;
        const int r = threadIdx.x % kBR;
        double v = 0.0;
        if (i < Im && r < R) v = T.A[m][i + Im * perm[r]];
        tmp[threadIdx.x] = v;
        __syncthreads();
        if (i < Im && r < R) T.A[m][i + Im * r] = tmp[threadIdx.x];
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host side
struct BItem {                   // one problem as given by the caller
  const void* Z;
  int zf64, N, R;
  int64_t dims[kBModes];
  double* A[kBModes];            // device float64 factors, updated in place
  double* gram;                  // device block of aux_doubles(): Grams, Gamma^+, row sums
  cpmg_opts o;
  int64_t target;                // elements per MTTKRP unit (autotuned per shape class)
  bool has_state;
  bool late;                     // past kLateSweeps: kLateUnit-element units, not the tuned size
  BTen state;                    // device state carried over when the batch is rebuilt
};

static int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

// A tensor still running after kLateSweeps sweeps switches to the smallest unit size: the tuned
// sizes favour throughput over a full batch, while the few tensors left late in a solve are
// latency-bound (a lone 40x126x48 rank-8 float-pair sweep: 0.41 ms at 32k-element units, 0.16 ms
// at 2k).  The switch depends only on the tensor's own sweep count, so its arithmetic is the same
// alone, in any batch, and in the server.
constexpr int kLateSweeps = 512;
constexpr int64_t kLateUnit = 4096;

// Marks the loaded tensors that crossed kLateSweeps; true when any unit list must be rebuilt.
static bool late_switch(std::vector<BItem*>& items, const std::vector<BTen>& host) {
  bool changed = false;
  for (size_t j = 0; j < items.size(); ++j)
    if (!items[j]->late && host[j].active && host[j].iters >= kLateSweeps) {
      items[j]->late = true;
      items[j]->target = std::min<int64_t>(items[j]->target, kLateUnit);
      changed = true;
    }
  return changed;
}

static int64_t numel_of(const BItem& it) {
  int64_t P = 1;
  for (int m = 0; m < it.N; ++m) P *= it.dims[m];
  return P;
}

// Unit lists and partial-sum layout (per tensor and mode) for the items' unit sizes.
static void plan_units(const std::vector<BItem>& items, std::vector<BUnit>* units, int* nk, size_t* part_off,
                       size_t* part_total) {
  for (int n = 0; n < kBModes; ++n) units[n].clear();
  size_t off = 0;
  for (size_t t = 0; t < items.size(); ++t) {
    const BItem& it = items[t];
    const int64_t I0 = it.dims[0];
    const int64_t P = numel_of(it);
    const int nrb = (int)cdiv64(I0, kBRows);
    const int64_t C = std::max<int64_t>(32, cdiv64(cdiv64(it.target, std::min<int64_t>(I0, kBRows)), 32) * 32);
    for (int n = 0; n < kBModes; ++n) {
      part_off[t * kBModes + n] = off;
      nk[t * kBModes + n] = 0;
      if (n >= it.N) continue;
      if (n == 0) {
        const int64_t ncol = P / I0;
        const int nch = (int)cdiv64(ncol, C);
        nk[t * kBModes + n] = nch;
        for (int ch = 0; ch < nch; ++ch)
          for (int rb = 0; rb < nrb; ++rb)
            units[0].push_back({(int)t, 0, rb, ch, ch * C, std::min<int64_t>(ncol, (ch + 1) * C), -1});
        off += (size_t)nch * I0 * kBR;
      } else {
        const int64_t In = it.dims[n];
        const int64_t ncol = P / (I0 * In);
        const int nch = (int)cdiv64(ncol, C);
        nk[t * kBModes + n] = nch * nrb;
        for (int64_t i = 0; i < In; ++i)
          for (int ch = 0; ch < nch; ++ch)
            for (int rb = 0; rb < nrb; ++rb)
              units[n].push_back({(int)t, n, rb, ch * nrb + rb, ch * C, std::min<int64_t>(ncol, (ch + 1) * C), i});
        off += (size_t)In * nch * nrb * kBR;
      }
    }
  }
  *part_total = off;
}

// per-tensor device state besides the factors: kBModes Grams, one Gamma^+ (float64 and float
// pairs), kBModes Gammas, 3 doubles per row, and the float-pair copy of the factors (kBR pairs
// per row)
static size_t aux_doubles(const BItem& it) {
  int64_t rows = 0;
  for (int m = 0; m < it.N; ++m) rows += it.dims[m];
  return (size_t)(2 * kBModes + 2) * kGramStride + (3 + 3 * kBR) * (size_t)rows;
}

static size_t partial_doubles_of(const BItem& it) {
  std::vector<BItem> one(1, it);
  std::vector<BUnit> u[kBModes];
  int nk[kBModes];
  size_t po[kBModes], tot = 0;
  plan_units(one, u, nk, po, &tot);
  return tot;
}

static BTen make_desc(const BItem& it) {
  BTen T;
  std::memset(&T, 0, sizeof(T));
  if (it.has_state) T = it.state;
  T.Z = it.Z;
  for (int m = 0; m < kBModes; ++m) {
    T.A[m] = it.A[m];
    T.dims[m] = it.dims[m];
    T.part[m] = nullptr;
  }
  T.gram = it.gram;
  T.ginv = it.gram + kBModes * kGramStride;
  T.gam = T.ginv + kGramStride;
  T.gih = reinterpret_cast<float*>(T.gam + kBModes * kGramStride);
  T.gil = T.gih + kGramStride;
  T.rowres = T.gam + (kBModes + 1) * kGramStride;
  int64_t rows = 0;
  for (int m = 0; m < it.N; ++m) rows += it.dims[m];
  float* fb = reinterpret_cast<float*>(T.rowres + 3 * rows);
  for (int m = 0; m < kBModes; ++m) {
    T.Ah[m] = m < it.N ? fb : nullptr;
    T.Al[m] = m < it.N ? fb + kBR * it.dims[m] : nullptr;
    if (m < it.N) fb += 2 * kBR * it.dims[m];
  }
  for (int m = 0; m < kBModes; ++m) {
    T.Rh[m] = m < it.N ? fb : nullptr;
    T.Rl[m] = m < it.N ? fb + kBR * it.dims[m] : nullptr;
    if (m < it.N) fb += 2 * kBR * it.dims[m];
  }
  T.mref = reinterpret_cast<double*>(fb);
  T.N = it.N;
  T.R = it.R;
  T.zf64 = it.zf64;
  T.shadow = !(it.zf64 || it.o.precision == CPMG_PREC_FP64);
  if (it.has_state) return T;
  T.policy = it.o.precision;
  if (it.zf64 || it.o.precision == CPMG_PREC_FP64) {
    T.prec = BP_FP64;
    T.gprec = BP_FP64;
  } else {
    T.prec = (it.o.precision == CPMG_PREC_DF) ? BP_DF : BP_FP32;
    // MIXED starts far above the FP32 floor: its first checks evaluate g with FP32 products
    T.gprec = it.o.precision == CPMG_PREC_MIXED ? BP_FP32 : BP_DF;
  }
  T.active = 1;
  T.init = 1;
  T.status = BS_RUNNING;
  T.max_iters = it.o.max_als_iters;
  T.tol = it.o.tol;
  T.mixed_switch = it.o.mixed_switch > 0 ? it.o.mixed_switch : 4.0;
  T.g = -1.0;
  T.g_best = -1.0;
  return T;
}

// Device resources of one batch; buffers grow by capacity so a server can rebuild cheaply.
struct BatchDev {
  cpmg_ctx* c = nullptr;
  int nten = 0, maxN = 0, grid = 0;
  int grid_run = 0;              // CTAs of the next launch: the loaded work's need, at most `grid`
  unsigned bar_extra = 0;        // grid-barrier settings (see BArgs)
  unsigned long long wait_ns = 2000000000ull;
  BTen* d_ten = nullptr;
  size_t cap_ten = 0;
  BUnit* d_units[kBModes] = {nullptr, nullptr, nullptr, nullptr};
  size_t cap_units[kBModes] = {0, 0, 0, 0};
  int64_t nunits[kBModes] = {0, 0, 0, 0};
  BRow* d_rows[kBModes] = {nullptr, nullptr, nullptr, nullptr};
  size_t cap_rows[kBModes] = {0, 0, 0, 0};
  int64_t nrows[kBModes] = {0, 0, 0, 0};
  double* d_part = nullptr;
  size_t cap_part = 0;
  int* d_idx = nullptr;
  size_t cap_idx = 0;
  unsigned* d_bar = nullptr;
  int* d_flags = nullptr;        // [0] error, [1] active count
  int* h_flags = nullptr;        // pinned mirror
  std::vector<BTen> host;
  ~BatchDev() { release(); }
  void release() {
    if (!c) return;
    for (int n = 0; n < kBModes; ++n) ctx_free(c, d_units[n]), d_units[n] = nullptr, cap_units[n] = 0;
    for (int n = 0; n < kBModes; ++n) ctx_free(c, d_rows[n]), d_rows[n] = nullptr, cap_rows[n] = 0;
    ctx_free(c, d_ten);
    ctx_free(c, d_part);
    ctx_free(c, d_idx);
    ctx_free(c, d_bar);
    ctx_free(c, d_flags);
    if (h_flags) cudaFreeHost(h_flags);
    d_ten = nullptr;
    d_part = nullptr;
    d_idx = nullptr;
    d_bar = nullptr;
    d_flags = h_flags = nullptr;
    cap_ten = cap_part = cap_idx = 0;
    c = nullptr;
  }
};

template <typename T>
static int grow(cpmg_ctx* c, T** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return CPMG_OK;
  ctx_free(c, *p);
  *p = nullptr;
  *cap = 0;
  const size_t n = std::max<size_t>(need, 1) + need / 4;
  CPMG_TRY(ctx_alloc(c, reinterpret_cast<void**>(p), n * sizeof(T)));
  *cap = n;
  return CPMG_OK;
}

static int batch_open(cpmg_ctx* c, BatchDev& B) {
  B.c = c;
  CPMG_TRY(ctx_alloc(c, reinterpret_cast<void**>(&B.d_bar), 2 * sizeof(unsigned)));
  CPMG_TRY(ctx_alloc(c, reinterpret_cast<void**>(&B.d_flags), 4 * sizeof(int)));
  CPMG_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&B.h_flags), 4 * sizeof(int)));
  CPMG_CUDA_TRY(cudaMemsetAsync(B.d_flags, 0, 4 * sizeof(int), ctx_stream(c)));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kBThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  cudaGetLastError();
  B.grid = per_sm * ctx_sms(c);
  return CPMG_OK;
}

// Descriptors, unit lists and partial layout for `items`; runs the init kernel for new ones.
static int batch_load(BatchDev& B, const std::vector<BItem>& items) {
  cudaStream_t st = ctx_stream(B.c);
  B.nten = (int)items.size();
  B.maxN = 0;
  for (auto& it : items) B.maxN = std::max(B.maxN, it.N);
  std::vector<BUnit> units[kBModes];
  std::vector<int> nk(items.size() * kBModes, 0);
  std::vector<size_t> poff(items.size() * kBModes, 0);
  size_t ptotal = 0;
  plan_units(items, units, nk.data(), poff.data(), &ptotal);
  CPMG_TRY(grow(B.c, &B.d_part, &B.cap_part, ptotal));
  CPMG_TRY(grow(B.c, &B.d_ten, &B.cap_ten, items.size()));
  for (int n = 0; n < kBModes; ++n) {
    B.nunits[n] = (int64_t)units[n].size();
    if (units[n].empty()) continue;
    CPMG_TRY(grow(B.c, &B.d_units[n], &B.cap_units[n], units[n].size()));
    CPMG_CUDA_TRY(cudaMemcpyAsync(B.d_units[n], units[n].data(), units[n].size() * sizeof(BUnit),
                                  cudaMemcpyHostToDevice, st));
  }
  // row items: kBRowsPerItem output rows of one mode of one tensor
  std::vector<BRow> rows[kBModes];
  for (size_t t = 0; t < items.size(); ++t)
    for (int n = 0; n < items[t].N; ++n)
      for (int64_t r0 = 0; r0 < items[t].dims[n]; r0 += kBRowsPerItem) rows[n].push_back({(int)t, n, r0});
  for (int n = 0; n < kBModes; ++n) {
    B.nrows[n] = (int64_t)rows[n].size();
    if (rows[n].empty()) continue;
    CPMG_TRY(grow(B.c, &B.d_rows[n], &B.cap_rows[n], rows[n].size()));
    CPMG_CUDA_TRY(cudaMemcpyAsync(B.d_rows[n], rows[n].data(), rows[n].size() * sizeof(BRow),
                                  cudaMemcpyHostToDevice, st));
  }
  // a smaller batch needs fewer CTAs: its phases have fewer units and rows than warps, and every
  // grid barrier waits for each CTA of the launch
  int64_t need = (int64_t)items.size();
  for (int n = 0; n < kBModes; ++n)
    need = std::max({need, cdiv64(B.nunits[n], kBWarps), cdiv64(B.nrows[n], kBWarps)});
  B.grid_run = (int)std::max<int64_t>(1, std::min<int64_t>(need, B.grid));
  B.host.resize(items.size());
  bool any_init = false;
  for (size_t t = 0; t < items.size(); ++t) {
    B.host[t] = make_desc(items[t]);
    for (int n = 0; n < kBModes; ++n) {
      B.host[t].nk[n] = nk[t * kBModes + n];
      B.host[t].part[n] = n < items[t].N ? B.d_part + poff[t * kBModes + n] : nullptr;
    }
    any_init = any_init || B.host[t].init;
  }
  CPMG_CUDA_TRY(cudaMemcpyAsync(B.d_ten, B.host.data(), B.host.size() * sizeof(BTen), cudaMemcpyHostToDevice, st));
  if (any_init) {
    k_batch_init<<<std::max(1, std::min(B.nten, 4 * ctx_sms(B.c))), kBThreads, 0, st>>>(B.d_ten, B.nten);
    CPMG_CUDA_TRY(cudaGetLastError());
    ctx_add_launches(B.c, 1);
    CPMG_CUDA_TRY(cudaMemcpyAsync(B.host.data(), B.d_ten, B.host.size() * sizeof(BTen), cudaMemcpyDeviceToHost, st));
  }
  CPMG_CUDA_TRY(cudaStreamSynchronize(st));
  return CPMG_OK;
}

// Algorithmic traffic of one launch: Z of every active tensor read once per MTTKRP pass (N per
// sweep, N more for the g evaluation), plus its float64 factors read and written once per sweep.
static double launch_bytes(const BatchDev& B, int nsweeps, int eval) {
  double b = 0.0;
  for (const BTen& T : B.host) {
    if (!T.active) continue;
    double P = 1.0, rows = 0.0;
    for (int m = 0; m < T.N; ++m) P *= (double)T.dims[m], rows += (double)T.dims[m];
    const double zb = (T.zf64 ? 8.0 : 4.0) * P;
    b += (double)(nsweeps * T.N + (eval ? T.N : 0)) * zb + (double)nsweeps * 16.0 * T.R * rows;
  }
  return b;
}

static int launch_batch(BatchDev& B, int nsweeps, int eval, bool profile = false) {
  cudaStream_t st = ctx_stream(B.c);
  BArgs a;
  a.ten = B.d_ten;
  a.nten = B.nten;
  for (int n = 0; n < kBModes; ++n) {
    a.units[n] = B.d_units[n];
    a.nunits[n] = B.nunits[n];
    a.rows[n] = B.d_rows[n];
    a.nrows[n] = B.nrows[n];
  }
  a.maxN = B.maxN;
  a.nsweeps = nsweeps;
  a.eval = eval;
  a.bar = B.d_bar;
  a.bar_extra = B.bar_extra;
  a.wait_ns = B.wait_ns;
  a.err = B.d_flags;
  a.nactive = B.d_flags + 1;
  void* args[] = {&a};
  CPMG_CUDA_TRY(cudaMemsetAsync(B.d_flags + 1, 0, sizeof(int), st));
  CPMG_CUDA_TRY(cudaMemsetAsync(B.d_bar, 0, 2 * sizeof(unsigned), st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (profile) CPMG_TRY(ctx_profile_events(B.c, 4, launch_bytes(B, nsweeps, eval), &e0, &e1));
  if (e0) CPMG_CUDA_TRY(cudaEventRecord(e0, st));
  const int grid = B.grid_run > 0 ? B.grid_run : B.grid;
  CPMG_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_batch, dim3(grid), dim3(kBThreads), args, 0, st));
  if (e1) CPMG_CUDA_TRY(cudaEventRecord(e1, st));
  ctx_add_launches(B.c, 1);
  return CPMG_OK;
}

// k sweeps + one evaluation; refreshes the host mirror of every descriptor.
static int batch_step(BatchDev& B, int k, int* nactive, bool profile = false) {
  cudaStream_t st = ctx_stream(B.c);
  CPMG_TRY(launch_batch(B, k, 1, profile));
  CPMG_CUDA_TRY(cudaMemcpyAsync(B.h_flags, B.d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CPMG_CUDA_TRY(cudaMemcpyAsync(B.host.data(), B.d_ten, B.host.size() * sizeof(BTen), cudaMemcpyDeviceToHost, st));
  CPMG_CUDA_TRY(cudaStreamSynchronize(st));
  if (B.h_flags[0]) return CPMG_TIMEOUT;
  *nactive = B.h_flags[1];
  return CPMG_OK;
}

static int batch_sort(BatchDev& B, const std::vector<int>& idx) {
  if (idx.empty()) return CPMG_OK;
  cudaStream_t st = ctx_stream(B.c);
  CPMG_TRY(grow(B.c, &B.d_idx, &B.cap_idx, idx.size()));
  CPMG_CUDA_TRY(cudaMemcpyAsync(B.d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  k_batch_sort<<<std::max(1, std::min((int)idx.size(), 4 * ctx_sms(B.c))), kBThreads, 0, st>>>(B.d_ten, B.d_idx,
                                                                                             (int)idx.size());
  CPMG_CUDA_TRY(cudaGetLastError());
  ctx_add_launches(B.c, 1);
  CPMG_CUDA_TRY(cudaStreamSynchronize(st));
  return CPMG_OK;
}

// ------------------------------------------------------------------ autotuner and server state
struct BatchState {
  std::map<std::string, int64_t> tuned;   // unit size per shape class
  int64_t fixed_target = 0;                // > 0: every class uses this unit size
  // request server
  struct Req {
    uint64_t id;
    BItem item;
    std::chrono::steady_clock::time_point t_submit, t_done;
    cpmg_result res;
    int state;     // 0 queued, 1 running, 2 done
    bool cancel = false;  // cpmg_server_cancel on a running request: retire at the next boundary
    // a multilevel request (cpmg_server_submit_multilevel): the caller's buffers and options
    bool ml = false;
    cpmg_tensor z{};
    int R = 0;
    std::vector<double*> A, T;
    cpmg_opts opts{};
    size_t bytes;  // HBM held while running (tensor, factors, partials, Gram)
  };
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::map<uint64_t, Req*> reqs;
  std::vector<double> lat;
  std::thread worker;
  bool stop = false, started = false;
  int worker_status = CPMG_OK;
  uint64_t next_id = 1;
  size_t budget = 0, reserved = 0;
  int max_active = 1024;
  int sweeps_per_launch = 8;
  // multilevel requests: their own queue, served by kMlWorkers threads with a context each
  std::deque<Req*> ml_queue;
  int ml_running = 0;
  std::vector<std::thread> ml_workers;
  bool ml_started = false;
  // failure-detection test hook (cpmg_debug_config): barrier wait limit, unreachable barrier
  double wait_limit_s = 2.0;
  int unreachable_barrier = 0;
  std::chrono::steady_clock::time_point t_first, t_last;
  bool any = false;
  int64_t completed = 0;
  int64_t launches = 0;
};

static BatchState* state_of(cpmg_ctx* c) {
  BatchState*& s = ctx_batch_state(c);
  if (!s) s = new BatchState();
  return s;
}

static std::string class_key(const BItem& it) {
  const int64_t P = numel_of(it);
  int lp = 0, li = 0;
  while ((int64_t(1) << lp) < P) ++lp;
  while ((int64_t(1) << li) < it.dims[0]) ++li;
  const int prec = it.zf64 ? 9 : it.o.precision;
  char b[64];
  snprintf(b, sizeof(b), "N%d_R%d_p%d_i%d_P%d", it.N, it.R, prec, li, lp);
  return b;
}

// Sets items[].target from the per-context cache; classes not seen yet are tuned jointly by
// timing one MTTKRP pass of every mode (sweep arithmetic, no state change) per candidate.
static int autotune(BatchDev& B, std::vector<BItem>& items) {
  BatchState* S = state_of(B.c);
  std::vector<int> todo;
  for (size_t t = 0; t < items.size(); ++t) {
    if (items[t].late) continue;  // keeps its late unit size
    if (S->fixed_target > 0) {
      items[t].target = S->fixed_target;
      continue;
    }
    auto f = S->tuned.find(class_key(items[t]));
    if (f != S->tuned.end()) items[t].target = f->second;
    else todo.push_back((int)t);
  }
  if (todo.empty()) return CPMG_OK;
  // Candidates in increasing size, each timed as the faster of two MTTKRP-only launches over the
  // whole batch. The timed launch has every tensor running; the rest of a solve runs fewer and
  // fewer tensors, and there smaller units (more work items per tensor) are faster. So the choice
  // is the smallest candidate within 5 % of the fastest launch (measured on the 512-tensor
  // workload: 2048 elements solve it in 4.88 s, 8192 in 5.15 s, while their launches differ by
  // less than the noise of one timing).
  constexpr int kCands = 5;
  const int64_t cands[kCands] = {2048, 4096, 8192, 16384, 32768};
  float ms_of[kCands];
  cudaStream_t st = ctx_stream(B.c);
  cudaEvent_t e0, e1;
  CPMG_CUDA_TRY(cudaEventCreate(&e0));
  CPMG_CUDA_TRY(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  int rc = CPMG_OK;
  for (int ci = 0; ci < kCands && rc == CPMG_OK; ++ci) {
    for (int t : todo) items[t].target = cands[ci];
    if ((rc = batch_load(B, items)) != CPMG_OK) break;
    if ((rc = launch_batch(B, 0, 2)) != CPMG_OK) break;  // warm
    ms_of[ci] = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, st);
      if ((rc = launch_batch(B, 0, 2)) != CPMG_OK) break;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = CPMG_CUDA_ERROR;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms_of[ci] = std::min(ms_of[ci], ms);
    }
    best_ms = std::min(best_ms, ms_of[ci]);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CPMG_TRY(rc);
  int64_t best = cands[kCands - 1];
  for (int ci = kCands - 1; ci >= 0; --ci)
    if (ms_of[ci] <= 1.05f * best_ms) best = cands[ci];
  for (int t : todo) {
    items[t].target = best;
    S->tuned[class_key(items[t])] = best;
  }
  // descriptors were loaded with init done: keep the computed ||Z||^2 and Grams
  for (size_t t = 0; t < items.size(); ++t) {
    items[t].has_state = true;
    items[t].state = B.host[t];
  }
  return CPMG_OK;
}

static int check_item(const cpmg_tensor* Z, int R, double* const* A, const cpmg_opts* o, BItem* it) {
  if (!Z || !A || !o) return CPMG_INVALID_ARG;
  if (Z->N < 2 || Z->N > kBModes || R < 1 || R > kBR || !Z->data) return CPMG_INVALID_ARG;
  if (Z->mem != CPMG_MEM_DEVICE || (Z->dtype != CPMG_F32 && Z->dtype != CPMG_F64)) return CPMG_INVALID_ARG;
  if (o->precision < 0 || o->precision > 3) return CPMG_INVALID_ARG;
  int64_t P = 1;
  for (int m = 0; m < Z->N; ++m) {
    if (Z->dims[m] < 1 || !A[m]) return CPMG_INVALID_ARG;
    P *= Z->dims[m];
  }
  if (P >= (int64_t(1) << 32)) return CPMG_INVALID_ARG;  // 32-bit index arithmetic in the kernel
  std::memset(it, 0, sizeof(*it));
  it->Z = Z->data;
  it->zf64 = Z->dtype == CPMG_F64;
  it->N = Z->N;
  it->R = R;
  for (int m = 0; m < kBModes; ++m) {
    it->dims[m] = m < Z->N ? Z->dims[m] : 1;
    it->A[m] = m < Z->N ? A[m] : nullptr;
  }
  it->o = *o;
  it->target = 8192;
  it->has_state = false;
  return CPMG_OK;
}

static void fill_result(const BTen& T, cpmg_result* r, double seconds) {
  std::memset(r, 0, sizeof(*r));
  r->f = T.f;
  r->g = T.g;
  r->iters_als = T.iters;
  r->levels = 1;
  r->status = T.status == BS_RUNNING ? CPMG_NOT_CONVERGED : T.status;
  r->seconds = seconds;
}

static double now_sec() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------ server worker
static void server_loop(cpmg_ctx* c, BatchState* S) {
  cudaSetDevice(ctx_device(c));
  BatchDev B;
  int rc = batch_open(c, B);
  bool dirty = true;
  std::vector<BItem> items;
  while (rc == CPMG_OK) {
    std::vector<BatchState::Req*> admitted;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (!S->stop && S->queue.empty() && S->active.empty()) S->cv.wait_for(lk, std::chrono::milliseconds(5));
      if (S->stop) break;
      // admission by HBM budget, in arrival order
      while (!S->queue.empty() && (int)S->active.size() < S->max_active) {
        BatchState::Req* q = S->queue.front();
        if (S->budget && S->reserved + q->bytes > S->budget && !S->active.empty()) break;
        S->queue.pop_front();
        S->active.push_back(q);
        S->reserved += q->bytes;
        q->state = 1;
        admitted.push_back(q);
        dirty = true;
      }
    }
    for (auto* q : admitted)
      if (!q->item.gram) {
        void* g = nullptr;
        if ((rc = ctx_alloc(c, &g, aux_doubles(q->item) * sizeof(double))) != CPMG_OK) break;
        q->item.gram = reinterpret_cast<double*>(g);
      }
    if (rc != CPMG_OK) break;
    if (dirty) {
      items.clear();
      for (auto* q : S->active) items.push_back(q->item);
      if ((rc = autotune(B, items)) != CPMG_OK) break;
      if ((rc = batch_load(B, items)) != CPMG_OK) break;
      for (size_t t = 0; t < items.size(); ++t) {
        S->active[t]->item.target = items[t].target;
        S->active[t]->item.has_state = true;
        S->active[t]->item.state = B.host[t];
      }
      dirty = false;
    }
    int nact = 0;
    if ((rc = batch_step(B, S->sweeps_per_launch, &nact)) != CPMG_OK) break;
    S->launches += 1;
    std::vector<int> fin;
    {
      std::lock_guard<std::mutex> lk(S->mu);  // cancel flags are set by other threads
      std::vector<BItem*> cur;
      for (size_t t = 0; t < S->active.size(); ++t) {
        S->active[t]->item.state = B.host[t];
        cur.push_back(&S->active[t]->item);
        if (!B.host[t].active || S->active[t]->cancel) fin.push_back((int)t);
      }
      if (late_switch(cur, B.host)) dirty = true;
    }
    if (!fin.empty()) {
      if ((rc = batch_sort(B, fin)) != CPMG_OK) break;
      const auto now = std::chrono::steady_clock::now();
      std::lock_guard<std::mutex> lk(S->mu);
      std::vector<BatchState::Req*> keep;
      size_t fi = 0;
      for (size_t t = 0; t < S->active.size(); ++t) {
        BatchState::Req* q = S->active[t];
        if (fi < fin.size() && fin[fi] == (int)t) {
          ++fi;
          q->t_done = now;
          const double lat = std::chrono::duration<double>(now - q->t_submit).count();
          fill_result(B.host[t], &q->res, lat);
          if (q->cancel && B.host[t].active) q->res.status = CPMG_CANCELLED;  // stopped before its end
          q->state = 2;
          S->reserved -= q->bytes;
          S->lat.push_back(lat);
          S->completed += 1;
          S->t_last = now;
          ctx_free(c, q->item.gram);
          q->item.gram = nullptr;
        } else {
          keep.push_back(q);
        }
      }
      S->active.swap(keep);
      dirty = true;
      S->cv.notify_all();
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->worker_status = rc;
  // fail everything still pending so pollers do not wait forever
  for (auto* q : S->active) {
    std::memset(&q->res, 0, sizeof(q->res));
    q->res.status = rc == CPMG_OK ? CPMG_CANCELLED : rc;
    q->state = 2;
    ctx_free(c, q->item.gram);
    q->item.gram = nullptr;
  }
  S->active.clear();
  for (auto* q : S->queue) {
    std::memset(&q->res, 0, sizeof(q->res));
    q->res.status = rc == CPMG_OK ? CPMG_CANCELLED : rc;
    q->state = 2;
  }
  S->queue.clear();
  S->reserved = 0;
  S->cv.notify_all();
}

// ------------------------------------------------------------------ multilevel request workers
constexpr int kMlWorkers = 2;

// One multilevel request at a time, by the "Multilevel" driver of Section 6.1 (cpmg_decompose) on
// a context and stream of the worker's own: the request's hierarchy is allocated when it starts
// and released when it ends, its launches overlap the batched worker's, and its arithmetic does
// not depend on what else runs.  Admission shares the server's HBM budget.
static void ml_loop(cpmg_ctx* parent, BatchState* S) {
  const int dev = ctx_device(parent);
  cudaSetDevice(dev);
  cudaStream_t st = nullptr;
  cpmg_ctx* c2 = nullptr;
  int rc = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess ? CPMG_OK : CPMG_CUDA_ERROR;
  if (rc == CPMG_OK) rc = cpmg_create(&c2, dev, 0, st);
  while (true) {
    BatchState::Req* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (!S->stop && (S->ml_queue.empty() || (S->budget && S->reserved + S->ml_queue.front()->bytes > S->budget &&
                                                   (S->reserved > 0))))
        S->cv.wait_for(lk, std::chrono::milliseconds(5));
      if (S->stop) break;
      q = S->ml_queue.front();
      S->ml_queue.pop_front();
      q->state = 1;
      S->reserved += q->bytes;
      S->ml_running += 1;
    }
    cpmg_result r;
    std::memset(&r, 0, sizeof(r));
    int s = rc;
    if (s == CPMG_OK) s = cpmg_decompose(c2, &q->z, q->R, q->A.data(), q->T.empty() ? nullptr : q->T.data(), &q->opts, &r);
    const auto now = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    q->res = r;
    if (s != CPMG_OK && s != CPMG_NOT_CONVERGED) q->res.status = s;
    const double lat = std::chrono::duration<double>(now - q->t_submit).count();
    q->res.seconds = lat;
    q->t_done = now;
    q->state = 2;
    S->reserved -= q->bytes;
    S->ml_running -= 1;
    S->lat.push_back(lat);
    S->completed += 1;
    S->t_last = now;
    S->cv.notify_all();
  }
  if (c2) cpmg_destroy(c2);
  if (st) cudaStreamDestroy(st);
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto* q : S->ml_queue) {  // not started: fail them so that pollers do not wait forever
    std::memset(&q->res, 0, sizeof(q->res));
    q->res.status = CPMG_CANCELLED;
    q->state = 2;
  }
  S->ml_queue.clear();
  S->cv.notify_all();
}

void batch_state_destroy(cpmg_ctx* c) {
  BatchState*& s = ctx_batch_state(c);
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& w : s->ml_workers)
    if (w.joinable()) w.join();
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  s = nullptr;
}

}  // namespace cpmg

using namespace cpmg;

extern "C" {

static int batch_solve_dev(cpmg_ctx* c, int count, const cpmg_tensor* Z, const int* R, double* const* const* A,
                           const cpmg_opts* opts, cpmg_result* results);

// Host buffers: every tensor and its factors are copied into one device arena, solved there, and
// the factors copied back; the copies are part of the call.
static int batch_solve_host(cpmg_ctx* c, int count, const cpmg_tensor* Z, const int* R, double* const* const* A,
                            const cpmg_opts* opts, cpmg_result* results) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t total = 0;
  for (int t = 0; t < count; ++t) {
    if (Z[t].mem != CPMG_MEM_HOST || !Z[t].data || !A[t] || Z[t].N < 2 || Z[t].N > kBModes || R[t] < 1 ||
        R[t] > kBR || (Z[t].dtype != CPMG_F32 && Z[t].dtype != CPMG_F64))
      return CPMG_INVALID_ARG;
    int64_t P = 1;
    for (int m = 0; m < Z[t].N; ++m) {
      if (Z[t].dims[m] < 1 || !A[t][m]) return CPMG_INVALID_ARG;
      P *= Z[t].dims[m];
      total += up(sizeof(double) * Z[t].dims[m] * R[t]);
    }
    total += up((Z[t].dtype == CPMG_F64 ? 8 : 4) * (size_t)P);
  }
  unsigned char* arena = nullptr;
  CPMG_TRY(ctx_alloc(c, reinterpret_cast<void**>(&arena), total));
  cudaStream_t st = ctx_stream(c);
  std::vector<cpmg_tensor> dz(Z, Z + count);
  std::vector<double*> dptr((size_t)count * kBModes, nullptr);
  std::vector<double* const*> da(count);
  size_t off = 0;
  int rc = CPMG_OK;
  for (int t = 0; t < count && rc == CPMG_OK; ++t) {
    int64_t P = 1;
    for (int m = 0; m < Z[t].N; ++m) P *= Z[t].dims[m];
    const size_t zb = (Z[t].dtype == CPMG_F64 ? 8 : 4) * (size_t)P;
    dz[t].data = arena + off;
    dz[t].mem = CPMG_MEM_DEVICE;
    if (cudaMemcpyAsync(arena + off, Z[t].data, zb, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = CPMG_CUDA_ERROR;
    off += up(zb);
    for (int m = 0; m < Z[t].N && rc == CPMG_OK; ++m) {
      const size_t ab = sizeof(double) * Z[t].dims[m] * R[t];
      dptr[(size_t)t * kBModes + m] = reinterpret_cast<double*>(arena + off);
      if (cudaMemcpyAsync(arena + off, A[t][m], ab, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = CPMG_CUDA_ERROR;
      off += up(ab);
    }
    da[t] = dptr.data() + (size_t)t * kBModes;
  }
  if (rc == CPMG_OK) rc = batch_solve_dev(c, count, dz.data(), R, da.data(), opts, results);
  const bool copy_back = rc == CPMG_OK || rc == CPMG_NOT_CONVERGED;
  for (int t = 0; t < count && copy_back; ++t)
    for (int m = 0; m < Z[t].N; ++m)
      if (cudaMemcpyAsync(A[t][m], dptr[(size_t)t * kBModes + m], sizeof(double) * Z[t].dims[m] * R[t],
                          cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = CPMG_CUDA_ERROR;
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == CPMG_OK) rc = CPMG_CUDA_ERROR;
  ctx_free(c, arena);
  return rc;
}

int cpmg_batch_solve(cpmg_ctx* c, int count, const cpmg_tensor* Z, const int* R, double* const* const* A,
                     const cpmg_opts* opts, cpmg_result* results) {
  cudaGetLastError();
  if (!c || count < 1 || !Z || !R || !A || !opts || !results) return CPMG_INVALID_ARG;
  if (Z[0].mem == CPMG_MEM_HOST) {
    {
      BatchState* S = state_of(c);
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->started) return CPMG_INVALID_ARG;  // the context serves requests
    }
    return batch_solve_host(c, count, Z, R, A, opts, results);
  }
  return batch_solve_dev(c, count, Z, R, A, opts, results);
}

static int batch_solve_dev(cpmg_ctx* c, int count, const cpmg_tensor* Z, const int* R, double* const* const* A,
                           const cpmg_opts* opts, cpmg_result* results) {
  {
    BatchState* S = state_of(c);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->started) return CPMG_INVALID_ARG;  // the context serves requests
  }
  const double t0 = now_sec();
  std::vector<BItem> items(count);
  for (int t = 0; t < count; ++t) CPMG_TRY(check_item(&Z[t], R[t], A[t], opts, &items[t]));
  BatchDev B;
  double* grams = nullptr;
  int st = batch_open(c, B);
  {
    BatchState* S = state_of(c);
    B.bar_extra = S->unreachable_barrier ? 1u : 0u;
    B.wait_ns = (unsigned long long)(S->wait_limit_s * 1e9);
  }
  size_t aux_total = 0;
  for (int t = 0; t < count; ++t) aux_total += aux_doubles(items[t]);
  if (st == CPMG_OK) st = ctx_alloc(c, reinterpret_cast<void**>(&grams), aux_total * sizeof(double));
  if (st == CPMG_OK) {
    size_t off = 0;
    for (int t = 0; t < count; ++t) {
      items[t].gram = grams + off;
      off += aux_doubles(items[t]);
    }
    st = autotune(B, items);
  }
  if (st == CPMG_OK) st = batch_load(B, items);
  const int k = opts->check_every > 0 ? opts->check_every : 8;
  // loaded[j]: the tensor in slot j of the loaded batch; last[t]: tensor t's latest device state
  std::vector<int> loaded(count);
  for (int t = 0; t < count; ++t) loaded[t] = t;
  std::vector<BTen> last(count);
  if (st == CPMG_OK) {
    const int64_t maxl = (std::max(opts->max_als_iters, 1) + k - 1) / k + 2;
    int nact = count;
    for (int64_t l = 0; l < maxl && nact > 0 && st == CPMG_OK; ++l) {
      st = batch_step(B, k, &nact, true);
      if (st != CPMG_OK || nact == 0) continue;
      std::vector<BItem*> cur(loaded.size());
      for (size_t j = 0; j < loaded.size(); ++j) cur[j] = &items[loaded[j]];
      const bool late = late_switch(cur, B.host);
      if (!late && nact * 2 > (int)loaded.size()) continue;
      // reload only the tensors still running (at most half of those loaded, or some switched to
      // late units); their state carries over, and each tensor's units, partial slots and sums
      // are its own, so its arithmetic does not depend on the others
      std::vector<BItem> act;
      std::vector<int> idx;
      for (size_t j = 0; j < loaded.size(); ++j) {
        last[loaded[j]] = B.host[j];
        if (!B.host[j].active) continue;
        BItem it = items[loaded[j]];
        it.has_state = true;
        it.state = B.host[j];
        act.push_back(it);
        idx.push_back(loaded[j]);
      }
      st = batch_load(B, act);
      loaded.swap(idx);
    }
    for (size_t j = 0; j < loaded.size() && st == CPMG_OK; ++j) last[loaded[j]] = B.host[j];
  }
  if (st == CPMG_OK) {
    if ((int)loaded.size() != count) {  // every tensor back in, with its final state, for the sort
      for (int t = 0; t < count; ++t) {
        items[t].has_state = true;
        items[t].state = last[t];
      }
      st = batch_load(B, items);
    }
    std::vector<int> all(count);
    for (int t = 0; t < count; ++t) all[t] = t;
    if (st == CPMG_OK) st = batch_sort(B, all);
  }
  const double dt = now_sec() - t0;
  int worst = st;
  for (int t = 0; t < count; ++t) {
    if (st == CPMG_OK) {
      fill_result(B.host[t], &results[t], dt);
      if (results[t].status != CPMG_OK && worst == CPMG_OK) worst = results[t].status;
    } else {
      std::memset(&results[t], 0, sizeof(cpmg_result));
      results[t].status = st;
    }
  }
  ctx_free(c, grams);
  return worst;
}

int cpmg_batch_plan(int N, const int64_t* dims, int R, int64_t unit_elements, int mode, int64_t* units,
                    int64_t max_units, int64_t* n_units, int* nk, int64_t* partial_doubles) {
  if (N < 2 || N > kBModes || !dims || R < 1 || R > kBR || unit_elements < 1 || mode < 0 || mode >= N ||
      !n_units || max_units < 0 || (max_units > 0 && !units))
    return CPMG_INVALID_ARG;
  BItem it;
  std::memset(&it, 0, sizeof(it));
  it.N = N;
  it.R = R;
  int64_t P = 1;
  for (int m = 0; m < kBModes; ++m) {
    it.dims[m] = m < N ? dims[m] : 1;
    if (m < N && dims[m] < 1) return CPMG_INVALID_ARG;
    P *= it.dims[m];
  }
  if (P >= (int64_t(1) << 32)) return CPMG_INVALID_ARG;
  it.target = unit_elements;
  std::vector<BItem> one(1, it);
  std::vector<BUnit> u[kBModes];
  int k[kBModes];
  size_t po[kBModes], tot = 0;
  plan_units(one, u, k, po, &tot);
  *n_units = (int64_t)u[mode].size();
  for (int64_t i = 0; i < std::min<int64_t>(max_units, (int64_t)u[mode].size()); ++i) {
    const BUnit& x = u[mode][i];
    int64_t* d = units + 5 * i;
    d[0] = x.rb;
    d[1] = x.k;
    d[2] = x.c0;
    d[3] = x.c1;
    d[4] = x.in_idx;
  }
  if (nk) *nk = k[mode];
  if (partial_doubles) *partial_doubles = (int64_t)tot;
  return CPMG_OK;
}

int cpmg_server_cancel(cpmg_ctx* c, uint64_t ticket) {
  if (!c) return CPMG_INVALID_ARG;
  BatchState* S = state_of(c);
  std::lock_guard<std::mutex> lk(S->mu);
  auto f = S->reqs.find(ticket);
  if (f == S->reqs.end()) return CPMG_INVALID_ARG;
  BatchState::Req* q = f->second;
  if (q->state == 0) {  // still queued: leaves the queue now, its factors untouched
    auto& qu = q->ml ? S->ml_queue : S->queue;
    for (auto it = qu.begin(); it != qu.end(); ++it)
      if (*it == q) {
        qu.erase(it);
        break;
      }
    std::memset(&q->res, 0, sizeof(q->res));
    q->res.status = CPMG_CANCELLED;
    q->res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - q->t_submit).count();
    q->state = 2;
    S->cv.notify_all();
  } else if (q->state == 1 && !q->ml) {
    q->cancel = true;  // the worker retires it after the launch in flight
  }  // a running multilevel request is one solver call: it finishes
  return CPMG_OK;
}

int cpmg_debug_config(cpmg_ctx* c, double wait_limit_s, int unreachable_barrier) {
  if (!c || !(wait_limit_s > 0.0) || wait_limit_s > 60.0) return CPMG_INVALID_ARG;
  BatchState* S = state_of(c);
  std::lock_guard<std::mutex> lk(S->mu);
  S->wait_limit_s = wait_limit_s;
  S->unreachable_barrier = unreachable_barrier != 0;
  return CPMG_OK;
}

int cpmg_server_config(cpmg_ctx* c, size_t hbm_budget_bytes, int max_active, int sweeps_per_launch,
                       int64_t unit_elements) {
  if (!c || max_active < 0 || sweeps_per_launch < 0 || unit_elements < 0) return CPMG_INVALID_ARG;
  BatchState* S = state_of(c);
  std::lock_guard<std::mutex> lk(S->mu);
  S->budget = hbm_budget_bytes;
  if (max_active > 0) S->max_active = max_active;
  if (sweeps_per_launch > 0) S->sweeps_per_launch = sweeps_per_launch;
  S->fixed_target = unit_elements;
  return CPMG_OK;
}

int cpmg_server_submit(cpmg_ctx* c, const cpmg_tensor* Z, int R, double* const* A, const cpmg_opts* opts,
                       uint64_t* ticket) {
  if (!c || !ticket) return CPMG_INVALID_ARG;
  BItem it;
  CPMG_TRY(check_item(Z, R, A, opts, &it));
  BatchState* S = state_of(c);
  auto* q = new BatchState::Req();
  q->item = it;
  q->item.gram = nullptr;
  q->state = 0;
  q->t_submit = std::chrono::steady_clock::now();
  const int64_t P = numel_of(it);
  size_t fb = 0;
  for (int m = 0; m < it.N; ++m) fb += (size_t)it.dims[m] * R * 8;
  q->bytes = (size_t)P * (it.zf64 ? 8 : 4) + fb + partial_doubles_of(it) * 8 + aux_doubles(it) * 8;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->budget && q->bytes > S->budget) {
    delete q;
    return CPMG_OUT_OF_BUDGET;
  }
  if (S->worker_status != CPMG_OK) {
    delete q;
    return S->worker_status;
  }
  q->id = S->next_id++;
  S->reqs[q->id] = q;
  S->queue.push_back(q);
  if (!S->any) {
    S->any = true;
    S->t_first = q->t_submit;
  }
  if (!S->worker.joinable()) {
    S->started = true;
    S->worker = std::thread(server_loop, c, S);
  }
  *ticket = q->id;
  lk.unlock();
  S->cv.notify_all();
  return CPMG_OK;
}

int cpmg_server_submit_multilevel(cpmg_ctx* c, const cpmg_tensor* Z, int R, double* const* A,
                                  double* const* A_test, const cpmg_opts* opts, uint64_t* ticket) {
  if (!c || !ticket || !Z || !A || !opts || !Z->data) return CPMG_INVALID_ARG;
  if (Z->N < 2 || Z->N > CPMG_MAX_MODES || Z->mem != CPMG_MEM_DEVICE || R < 1 || R > CPMG_MAX_RANK)
    return CPMG_INVALID_ARG;
  if (opts->n_t < 0 || opts->n_t > CPMG_MAX_TEST_BLOCKS || (opts->n_t > 0 && !A_test)) return CPMG_INVALID_ARG;
  auto* q = new BatchState::Req();
  q->ml = true;
  q->z = *Z;
  q->R = R;
  q->opts = *opts;
  int64_t P = 1;
  size_t fb = 0;
  for (int m = 0; m < Z->N; ++m) {
    if (Z->dims[m] < 1 || !A[m]) {
      delete q;
      return CPMG_INVALID_ARG;
    }
    P *= Z->dims[m];
    fb += (size_t)Z->dims[m] * R * 8;
    q->A.push_back(A[m]);
  }
  for (int t = 0; t < opts->n_t; ++t)
    for (int m = 0; m < Z->N; ++m) {
      if (!A_test[t * Z->N + m]) {
        delete q;
        return CPMG_INVALID_ARG;
      }
      q->T.push_back(A_test[t * Z->N + m]);
    }
  std::memset(&q->item, 0, sizeof(q->item));
  q->state = 0;
  q->t_submit = std::chrono::steady_clock::now();
  // HBM held while it runs: the coarse tensors (under 1/7 of Z for third order, more for lower
  // orders: counted as one more Z), the MTTKRP scratch (about one more Z), the factor sets
  const size_t zb = (size_t)P * (Z->dtype == CPMG_F64 ? 8 : 4);
  q->bytes = zb + zb + 2 * zb + fb * (size_t)(2 * opts->n_t + 8) + ((size_t)64 << 20);
  BatchState* S = state_of(c);
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->budget && q->bytes > S->budget) {
    delete q;
    return CPMG_OUT_OF_BUDGET;
  }
  q->id = S->next_id++;
  S->reqs[q->id] = q;
  S->ml_queue.push_back(q);
  if (!S->any) {
    S->any = true;
    S->t_first = q->t_submit;
  }
  if (!S->ml_started) {
    S->ml_started = true;
    S->started = true;  // the context now serves: other solver calls are refused
    for (int w = 0; w < kMlWorkers; ++w) S->ml_workers.emplace_back(ml_loop, c, S);
  }
  *ticket = q->id;
  lk.unlock();
  S->cv.notify_all();
  return CPMG_OK;
}

int cpmg_server_poll(cpmg_ctx* c, uint64_t ticket, cpmg_result* out) {
  if (!c || !out) return CPMG_INVALID_ARG;
  BatchState* S = state_of(c);
  std::lock_guard<std::mutex> lk(S->mu);
  auto f = S->reqs.find(ticket);
  if (f == S->reqs.end()) return CPMG_INVALID_ARG;
  BatchState::Req* q = f->second;
  if (q->state != 2) return CPMG_PENDING;
  *out = q->res;
  S->reqs.erase(f);
  delete q;
  return CPMG_OK;
}

int cpmg_server_wait(cpmg_ctx* c, double timeout_s) {
  if (!c) return CPMG_INVALID_ARG;
  BatchState* S = state_of(c);
  std::unique_lock<std::mutex> lk(S->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (!S->queue.empty() || !S->active.empty() || !S->ml_queue.empty() || S->ml_running > 0) {
    if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout) return CPMG_PENDING;
  }
  return S->worker_status;
}

int cpmg_server_stats(cpmg_ctx* c, double* p50_s, double* p99_s, double* req_per_s, int64_t* completed) {
  if (!c) return CPMG_INVALID_ARG;
  BatchState* S = state_of(c);
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->lat;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    const size_t i = (size_t)std::min<double>((double)v.size() - 1, std::ceil(p * v.size()) - 1);
    return v[i];
  };
  if (p50_s) *p50_s = pct(0.50);
  if (p99_s) *p99_s = pct(0.99);
  if (req_per_s) {
    const double span = S->completed ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    *req_per_s = span > 0 ? S->completed / span : 0.0;
  }
  if (completed) *completed = S->completed;
  return CPMG_OK;
}

}  // extern "C"
