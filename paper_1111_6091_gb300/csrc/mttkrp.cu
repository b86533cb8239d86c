// MTTKRP M = Z_(n) Phi^(n) (Eq. fineeq1 with Phi^(n) of Eq. Phi) on sm_103a CUDA cores.
//
// Layout: Z is column-major, so with I_1 the first (contiguous) mode every "column"
// (fixed i_2..i_N) is I_1 consecutive elements.  For mode n the columns are indexed
// by col = o_lo + Lp * (i_n + I_n * o_hi), where o_lo runs over the modes strictly
// between the first mode and n (Lp values) and o_hi over the modes after n (G values).
// The Khatri-Rao row for the non-first, non-n modes factorizes as
//     W(col, r) = Kin(o_lo, r) * Kout(o_hi, r),
// with Kin / Kout the Khatri-Rao products of those mode groups (small tables built
// from the float64 factors before the main kernel).  Then
//     mode 1:  M(i_1, r)   = sum_col Z(i_1, col) W(col, r)
//     mode n:  M(i_n, r)   = sum_col [ sum_{i_1} Z(i_1, col) A^(1)(i_1, r) ] W(col, r).
// Each thread owns VW consecutive rows i_1 (one 16-byte load per column when VW = 4),
// keeps A^(1) for those rows in registers (mode n > 1), and walks columns; Z is read
// exactly once.  Per-CTA partials are combined by a second kernel in a fixed order,
// so results are bitwise reproducible.
//
// Arithmetic: P_FP32 float products and sums; P_FP64 double; P_DF pairs of floats
// (exact products via FMA, error-free sums), about 2^-48 relative per operation.
#include "mttkrp.cuh"

#include <algorithm>
#include <cmath>

namespace cpmg {

template <int PREC> struct Tr;
template <> struct Tr<P_FP32> { using V = float;  using Tab = float;  using Part = float;  };
template <> struct Tr<P_FP64> { using V = double; using Tab = double; using Part = double; };
template <> struct Tr<P_DF>   { using V = df;     using Tab = float2; using Part = double; };

static size_t tab_size(int prec) { return prec == P_FP32 ? 4 : 8; }
static size_t part_size(int prec) { return prec == P_FP32 ? 4 : 8; }

size_t MttkrpPlan::partial_bytes() const {
  size_t per = (mode == 0) ? (size_t)SEG * RP : (size_t)RP * nw;
  return (size_t)nunits * per * part_elem;
}
size_t MttkrpPlan::tables_bytes() const {
  size_t rows = use_tma ? (size_t)Lp * G : (size_t)(has_in ? Lp : 0) + (size_t)(has_out ? G : 0);
  return ((rows * TS * table_bytes + 255) / 256) * 256 + 256;
}

// ------------------------------------------------------------------ generic helpers
template <typename V> struct Ops;
template <> struct Ops<float> {
  __device__ static float zero() { return 0.f; }
  __device__ static float mul(float a, float b) { return a * b; }
  __device__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  __device__ static float mulz(float z, float a) { return z * a; }
  __device__ static float fmaz(float z, float a, float c) { return __fmaf_rn(z, a, c); }
  __device__ static void acc(float& c, float z, float a) { c = __fmaf_rn(z, a, c); }
  __device__ static void acc(float& c, float u, float w, int) { c = __fmaf_rn(u, w, c); }
  __device__ static void norm(float&) {}
  __device__ static double to_d(float a) { return (double)a; }
};
template <> struct Ops<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  __device__ static double mulz(double z, double a) { return z * a; }
  __device__ static double fmaz(double z, double a, double c) { return __fma_rn(z, a, c); }
  __device__ static void acc(double& c, double z, double a) { c = __fma_rn(z, a, c); }
  __device__ static void acc(double& c, double u, double w, int) { c = __fma_rn(u, w, c); }
  __device__ static void norm(double&) {}
  __device__ static double to_d(double a) { return a; }
};
template <> struct Ops<df> {
  __device__ static df zero() { return {0.f, 0.f}; }
  __device__ static df mul(df a, df b) { return df_mul(a, b); }
  __device__ static df fma(df a, df b, df c) { return df_add(c, df_mul(a, b)); }
  __device__ static df fmaz(float z, df a, df c) { return df_add(c, df_mul_f(z, a)); }
  // Accumulation in the hot loops: the rounded product goes into c.hi by TwoSum, the product's
  // rounding error and the TwoSum error into c.lo; norm folds c.lo back and runs after every
  // few columns (a stage or an unrolled group), so c.lo never sums more than a handful of terms.
  __device__ static void acc(df& c, float z, df a) {
    const float p = __fmul_rn(z, a.hi);
    float e = __fmaf_rn(z, a.hi, -p);
    e = __fmaf_rn(z, a.lo, e);
    const df s = df_two_sum(c.hi, p);
    c.hi = s.hi;
    c.lo = __fadd_rn(c.lo, __fadd_rn(s.lo, e));
  }
  __device__ static void acc(df& c, df u, df w, int) {
    const float p = __fmul_rn(u.hi, w.hi);
    float e = __fmaf_rn(u.hi, w.hi, -p);
    e = __fmaf_rn(u.hi, w.lo, e);
    e = __fmaf_rn(u.lo, w.hi, e);
    const df s = df_two_sum(c.hi, p);
    c.hi = s.hi;
    c.lo = __fadd_rn(c.lo, __fadd_rn(s.lo, e));
  }
  __device__ static void norm(df& c) { c = df_two_sum(c.hi, c.lo); }
  __device__ static double to_d(df a) { return df_to_double(a); }
};

template <typename Tab, typename V> __device__ __forceinline__ V tab_get(const Tab* p);
template <> __device__ __forceinline__ float tab_get<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ double tab_get<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ df tab_get<float2, df>(const float2* p) {
  float2 v = __ldg(p);
  return {v.x, v.y};
}

// Load RP table entries of one row (RP is a multiple of 4, rows 16-byte aligned).
template <int PREC, int RP>
__device__ __forceinline__ void load_row(const typename Tr<PREC>::Tab* row, typename Tr<PREC>::V* out) {
  if constexpr (PREC == P_FP32) {
    const float4* p = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int k = 0; k < RP / 4; ++k) {
      float4 v = __ldg(p + k);
      out[4 * k] = v.x; out[4 * k + 1] = v.y; out[4 * k + 2] = v.z; out[4 * k + 3] = v.w;
    }
  } else if constexpr (PREC == P_FP64) {
    const double2* p = reinterpret_cast<const double2*>(row);
#pragma unroll
    for (int k = 0; k < RP / 2; ++k) {
      double2 v = __ldg(p + k);
      out[2 * k] = v.x; out[2 * k + 1] = v.y;
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int k = 0; k < RP / 2; ++k) {
      float4 v = __ldg(p + k);
      out[2 * k] = {v.x, v.y}; out[2 * k + 1] = {v.z, v.w};
    }
  }
}

// Vector of VW tensor elements as the compute scalar (float for FP32/DF, double for FP64).
template <typename TZ, int PREC> struct ZS { using T = float; };
template <typename TZ> struct ZS<TZ, P_FP64> { using T = double; };

template <typename TZ, int VW, typename S>
__device__ __forceinline__ void load_z(const TZ* p, S* z) {
  if constexpr (sizeof(TZ) == 4 && VW == 4) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    z[0] = (S)v.x; z[1] = (S)v.y; z[2] = (S)v.z; z[3] = (S)v.w;
  } else if constexpr (sizeof(TZ) == 4 && VW == 2) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    z[0] = (S)v.x; z[1] = (S)v.y;
  } else if constexpr (sizeof(TZ) == 8 && VW == 2) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    z[0] = (S)v.x; z[1] = (S)v.y;
  } else {
#pragma unroll
    for (int q = 0; q < VW; ++q) z[q] = (S)__ldg(p + q);
  }
}

// ------------------------------------------------------------------ tables kernel
struct FactorPtrs {
  const double* p[kMaxModes];
  int64_t I[kMaxModes];
};

struct TabArgs {
  FactorPtrs f;
  int R, TS;
  int n_in, in_modes[kMaxModes];
  int n_out, out_modes[kMaxModes];
  int n_all, all_modes[kMaxModes];  // in_modes then out_modes
  int64_t Lp, G;
  void* kin;
  void* kout;
  void* wfull;                      // W(f) = Kin(f mod Lp) * Kout(f div Lp), f < Lp G
};

template <int PREC>
__global__ void k_tables(TabArgs a) {
  using Tab = typename Tr<PREC>::Tab;
  const int which = blockIdx.y;  // 0: Kin, 1: Kout, 2: full row table W
  const int nm = which == 0 ? a.n_in : (which == 1 ? a.n_out : a.n_all);
  const int* modes = which == 0 ? a.in_modes : (which == 1 ? a.out_modes : a.all_modes);
  const int64_t rows = which == 0 ? a.Lp : (which == 1 ? a.G : a.Lp * a.G);
  Tab* out = reinterpret_cast<Tab*>(which == 0 ? a.kin : (which == 1 ? a.kout : a.wfull));
  if (out == nullptr || (nm == 0 && which != 2)) return;
  const int64_t total = rows * a.TS;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / a.TS;
    const int r = (int)(e % a.TS);
    double prod = 0.0;
    if (r < a.R) {
      prod = 1.0;
      int64_t rem = row;
      for (int k = 0; k < nm; ++k) {
        const int m = modes[k];
        const int64_t I = a.f.I[m];
        const int64_t i = rem % I;
        rem /= I;
        prod *= a.f.p[m][i + I * r];
      }
    }
    if constexpr (PREC == P_FP32) out[e] = (float)prod;
    else if constexpr (PREC == P_FP64) out[e] = prod;
    else { df d = df_from_double(prod); out[e] = make_float2(d.hi, d.lo); }
  }
}

// ------------------------------------------------------------------ main kernel
struct MainArgs {
  const void* Z;
  const double* A1;  // float64 factor of the first mode (mode > 0 only)
  int64_t I1, SEG, In, Lp, G, F;
  int TX, TY, nseg, C, R;
  int has_in, has_out, first;
  const void* kin;
  const void* kout;
  void* partial;
};

constexpr int kUnroll = 4;
constexpr int kMaxCps = 4;  // columns per thread per stage held in registers by the TMA kernel

// FP32 kernels with up to 12 padded ranks fit 128 registers at 448 threads; everything
// else runs 256-thread CTAs.
constexpr int max_threads(int prec, int RP) { return (prec == P_FP32 && RP <= 12) ? 448 : 256; }

template <typename TZ, int PREC, int VW, int RP, bool FIRST>
__global__ void __launch_bounds__(max_threads(PREC, RP), 1) k_mttkrp_main(MainArgs a) {
  using V = typename Tr<PREC>::V;
  using Tab = typename Tr<PREC>::Tab;
  using Part = typename Tr<PREC>::Part;
  using S = typename ZS<TZ, PREC>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const int t = threadIdx.x;
  const int tx = t % a.TX, ty = t / a.TX;
  int64_t u = blockIdx.x;
  const int chunk = (int)(u % a.C);
  u /= a.C;
  const int seg = (int)(u % a.nseg);
  const int64_t in = u / a.nseg;
  const int64_t row0 = (int64_t)seg * a.SEG + (int64_t)tx * VW;
  const bool active = (ty < a.TY) && (row0 < a.I1);
  const int64_t f0 = (a.F * chunk) / a.C, f1 = (a.F * (chunk + 1)) / a.C;

  const TZ* Z = reinterpret_cast<const TZ*>(a.Z);
  const Tab* kin = reinterpret_cast<const Tab*>(a.kin);
  const Tab* kout = reinterpret_cast<const Tab*>(a.kout);

  constexpr int QA = FIRST ? VW : 1;   // accumulator rows
  constexpr int QW = FIRST ? 1 : VW;   // A^(1) rows held in registers
  V accm[QA][RP];   // mode 1: per-row accumulators;  mode n>1: one accumulator row
  V a1[QW][RP];     // mode n>1: A^(1) rows of this thread
#pragma unroll
  for (int q = 0; q < QA; ++q)
#pragma unroll
    for (int r = 0; r < RP; ++r) accm[q][r] = Ops<V>::zero();
#pragma unroll
  for (int q = 0; q < QW; ++q)
#pragma unroll
    for (int r = 0; r < RP; ++r) a1[q][r] = Ops<V>::zero();

  if (!FIRST && active) {
#pragma unroll
    for (int q = 0; q < QW; ++q)
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        if (r < a.R) {
          const double v = a.A1[row0 + q + a.I1 * r];
          if constexpr (PREC == P_FP32) a1[q][r] = (float)v;
          else if constexpr (PREC == P_FP64) a1[q][r] = v;
          else a1[q][r] = df_from_double(v);
        }
      }
  }

  if (active) {
    // column iterator: f = f0 + ty, f0 + ty + TY, ...
    int64_t f = f0 + ty;
    int64_t o_lo = f % a.Lp, o_hi = f / a.Lp;
    const int64_t dq = a.TY / a.Lp, dr = a.TY % a.Lp;
    const int64_t colstride = a.Lp * a.In;  // o_hi step in columns
    while (f < f1) {
      S zb[kUnroll][VW];
      int64_t lo[kUnroll], hi[kUnroll];
      bool ok[kUnroll];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        ok[k] = f < f1;
        lo[k] = o_lo;
        hi[k] = o_hi;
        if (ok[k]) {
          const int64_t col = o_lo + a.Lp * in + colstride * o_hi;
          load_z<TZ, VW, S>(Z + col * a.I1 + row0, zb[k]);
        }
        f += a.TY;
        o_lo += dr;
        o_hi += dq;
        if (o_lo >= a.Lp) { o_lo -= a.Lp; ++o_hi; }
      }
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        if (!ok[k]) continue;
        V w[RP];
        if (a.has_in) {
          load_row<PREC, RP>(kin + lo[k] * RP, w);
          if (a.has_out) {
            V w2[RP];
            load_row<PREC, RP>(kout + hi[k] * RP, w2);
#pragma unroll
            for (int r = 0; r < RP; ++r) w[r] = Ops<V>::mul(w[r], w2[r]);
          }
        } else if (a.has_out) {
          load_row<PREC, RP>(kout + hi[k] * RP, w);
        } else {
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            if constexpr (PREC == P_DF) w[r] = {1.f, 0.f};
            else w[r] = (V)1;
          }
        }
        if constexpr (FIRST) {
#pragma unroll
          for (int q = 0; q < VW; ++q)
#pragma unroll
            for (int r = 0; r < RP; ++r) Ops<V>::acc(accm[q][r], zb[k][q], w[r]);
        } else {
          V uu[RP];
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            if constexpr (PREC == P_DF) uu[r] = df_mul_f(zb[k][0], a1[0][r]);
            else uu[r] = Ops<V>::mulz(zb[k][0], a1[0][r]);
          }
#pragma unroll
          for (int q = 1; q < QW; ++q)
#pragma unroll
            for (int r = 0; r < RP; ++r) Ops<V>::acc(uu[r], zb[k][q], a1[q][r]);
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            Ops<V>::norm(uu[r]);
            Ops<V>::acc(accm[0][r], uu[r], w[r], 0);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < QA; ++q)
#pragma unroll
        for (int r = 0; r < RP; ++r) Ops<V>::norm(accm[q][r]);
    }
  }

  // ---------------------------------------------------------------- reductions
  if constexpr (!FIRST) {
    Part* red = reinterpret_cast<Part*>(smem_raw);
    const int lane = t & 31, warp = t >> 5, nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      Part v;
      if constexpr (PREC == P_FP32) v = accm[0][r];
      else v = (Part)Ops<V>::to_d(accm[0][r]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp * RP + r] = v;
    }
    __syncthreads();
    if (t < RP) {
      Part s = 0;
      for (int w = 0; w < nwarps; ++w) s += red[w * RP + t];
      reinterpret_cast<Part*>(a.partial)[blockIdx.x * (int64_t)RP + t] = s;
    }
  } else {
    // reduce the TY column groups of the same rows: [ty][row_in_seg][r] in smem, then sum over ty
    Part* red = reinterpret_cast<Part*>(smem_raw);
    const int64_t segrows = (int64_t)a.TX * VW;
    if (ty < a.TY) {
#pragma unroll
      for (int q = 0; q < QA; ++q)
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          Part v;
          if constexpr (PREC == P_FP32) v = accm[q][r];
          else v = (Part)Ops<V>::to_d(accm[q][r]);
          red[((int64_t)ty * segrows + (int64_t)tx * VW + q) * RP + r] = v;
        }
    }
    __syncthreads();
    Part* out = reinterpret_cast<Part*>(a.partial) + (int64_t)blockIdx.x * segrows * RP;
    for (int64_t e = t; e < segrows * RP; e += blockDim.x) {
      Part s = 0;
      for (int g = 0; g < a.TY; ++g) s += red[(int64_t)g * segrows * RP + e];
      out[e] = s;
    }
  }
}

// ------------------------------------------------------------------ TMA-pipelined kernel
// Same arithmetic and partial-sum layout as k_mttkrp_main, but the tensor is streamed into a
// ring of shared-memory stages by cp.async.bulk (TMA bulk copies completing on mbarriers),
// issued by one producer warp that also forms the Khatri-Rao rows W of each stage.  The
// consumer threads read their VW elements and the W rows from shared memory.  Every wait
// is bounded (~2 s of %globaltimer); on expiry the kernel sets bit 0 of *err and stops.
struct TmaArgs {
  MainArgs m;
  int64_t nunits;          // work units; each CTA takes a contiguous range of them
  const void* wfull;       // full Khatri-Rao row table W(f), F x RP
  int tab_smem;            // Kin/Kout copied to shared memory at tab_off
  uint32_t tab_off;
  int CPS, S, NC, contiguous;
  int64_t ROWS;            // rows of one segment held per column in shared memory
  uint32_t stage_off;      // byte offset of stage 0
  uint32_t red_off;        // byte offset of the mode-1 reduction area (after the mbarriers)
  uint32_t stage_stride;   // bytes between stages
  uint32_t w_off;          // byte offset of the W-row ring (WS = 2 S slots of w_stride bytes)
  uint32_t w_stride;
  uint32_t bar_off;        // byte offset of the mbarriers
  uint32_t col_off;        // byte offset of the producer's column list
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// try_wait suspends the thread until the phase completes or the hinted time (1 ms) passes.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: true when the phase with this parity completed, false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (gtimer() - t0 > 2000000000ull) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Packed pairs of floats for the FP32 path: fma.rn.f32x2 performs two FMAs per instruction.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ float2 up2(unsigned long long v) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(v));
  return f;
}

template <int PREC, int RP>
__device__ __forceinline__ void load_row_s(const typename Tr<PREC>::Tab* row, typename Tr<PREC>::V* out) {
  if constexpr (PREC == P_FP32) {
    const float4* p = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int k = 0; k < RP / 4; ++k) {
      float4 v = p[k];
      out[4 * k] = v.x; out[4 * k + 1] = v.y; out[4 * k + 2] = v.z; out[4 * k + 3] = v.w;
    }
  } else if constexpr (PREC == P_FP64) {
    const double2* p = reinterpret_cast<const double2*>(row);
#pragma unroll
    for (int k = 0; k < RP / 2; ++k) {
      double2 v = p[k];
      out[2 * k] = v.x; out[2 * k + 1] = v.y;
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int k = 0; k < RP / 2; ++k) {
      float4 v = p[k];
      out[2 * k] = {v.x, v.y}; out[2 * k + 1] = {v.z, v.w};
    }
  }
}

template <typename TZ, int VW, typename S>
__device__ __forceinline__ void load_z_s(const TZ* p, S* z) {
  if constexpr (sizeof(TZ) == 4 && VW == 4) {
    float4 v = *reinterpret_cast<const float4*>(p);
    z[0] = (S)v.x; z[1] = (S)v.y; z[2] = (S)v.z; z[3] = (S)v.w;
  } else if constexpr (sizeof(TZ) == 4 && VW == 2) {
    float2 v = *reinterpret_cast<const float2*>(p);
    z[0] = (S)v.x; z[1] = (S)v.y;
  } else if constexpr (sizeof(TZ) == 8 && VW == 2) {
    double2 v = *reinterpret_cast<const double2*>(p);
    z[0] = (S)v.x; z[1] = (S)v.y;
  } else {
#pragma unroll
    for (int q = 0; q < VW; ++q) z[q] = (S)p[q];
  }
}

// Consumers (up to 448 FP32 threads at <= 12 padded ranks, 256 otherwise) plus one producer warp.
// At most four warps land on each SM sub-partition, so 128 (FP32) / 168 registers stay available.
constexpr int tma_threads(int prec, int RP) { return (prec == P_FP32 && RP <= 12) ? 480 : 288; }

// HP: float pairs actually computed (FP32: ceil(R / 2), so R = 10 runs 5 pairs, not the 6 of the
// padded table row); other precisions compute all RP.
template <typename TZ, int PREC, int VW, int RP, bool FIRST, int HP = RP / 2>
__global__ void __launch_bounds__(tma_threads(PREC, RP), 1) k_mttkrp_tma(TmaArgs ta) {
  using V = typename Tr<PREC>::V;
  using Tab = typename Tr<PREC>::Tab;
  using Part = typename Tr<PREC>::Part;
  using S = typename ZS<TZ, PREC>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const MainArgs& a = ta.m;
  const int t = threadIdx.x;
  const int ncpad = (ta.NC + 31) & ~31;
  const int nwc = ncpad / 32;  // consumer warps
  const int SF = a.TY * ta.CPS;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + ta.bar_off);
  uint64_t* empty = full + ta.S;
  int64_t* colbuf = reinterpret_cast<int64_t*>(smem_raw + ta.col_off);
  const Tab* wfull = reinterpret_cast<const Tab*>(ta.wfull);
  // this CTA's contiguous range of work units
  const int64_t ub = (ta.nunits * (int64_t)blockIdx.x) / gridDim.x;
  const int64_t ue = (ta.nunits * (int64_t)(blockIdx.x + 1)) / gridDim.x;
  if (t == 0) {
    for (int s = 0; s < ta.S; ++s) {
      mbar_init(&full[s], ta.contiguous ? 1 : 32);
      mbar_init(&empty[s], nwc);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // FP32 keeps one accumulator per row in every mode (mode n > 1 applies A^(1) once per unit)
  constexpr int QA = (PREC == P_FP32 || FIRST) ? VW : 1;
  constexpr int QW = FIRST ? 1 : VW;
  bool failed = false;

  if (t >= ncpad && ta.contiguous) {
    // ------------------------------------------------ producer, contiguous stages: one thread
    // issues one copy of whole columns and one of the matching table rows per stage
    if (t == ncpad) {
      const TZ* Z = reinterpret_cast<const TZ*>(a.Z);
      int s = 0;
      uint32_t ph = 0;      // parity of the ring's current pass
      int64_t issued = 0;
      for (int64_t u = ub; u < ue && !failed; ++u) {
        const int chunk = (int)(u % a.C);
        const int64_t in = u / ((int64_t)a.C * a.nseg);
        const int64_t rows = a.I1 < ta.ROWS ? a.I1 : ta.ROWS;
        const uint32_t colbytes = (uint32_t)(rows * sizeof(TZ));
        const int64_t f0 = (a.F * chunk) / a.C, f1 = (a.F * (chunk + 1)) / a.C;
        // contiguous: mode 1 (f is the column) or the last mode (column f + F * in)
        const int64_t colbase = (a.In == 1) ? 0 : a.F * in;
        for (int64_t fs = f0; fs < f1; fs += SF) {
          if (issued >= ta.S && !mbar_wait(&empty[s], ph ^ 1u)) { failed = true; break; }
          const int nf = (int)((f1 - fs) < SF ? (f1 - fs) : SF);
          unsigned char* stage = smem_raw + ta.stage_off + (size_t)s * ta.stage_stride;
          const uint32_t wbytes = (uint32_t)(nf * RP * sizeof(Tab));
          mbar_arrive_tx(&full[s], colbytes * (uint32_t)nf + wbytes);
          bulk_g2s(stage + ta.w_off, wfull + fs * RP, wbytes, &full[s]);
          bulk_g2s(stage, Z + (colbase + fs) * a.I1, colbytes * (uint32_t)nf, &full[s]);
          ++issued;
          if (++s == ta.S) { s = 0; ph ^= 1u; }
        }
      }
      // no copy may still be in flight when shared memory is reused or released
      for (int64_t j = (issued > ta.S ? issued - ta.S : 0); j < issued; ++j)
        if (!mbar_wait(&full[j % ta.S], (uint32_t)((j / ta.S) & 1))) failed = true;
    }
  } else if (t >= ncpad) {
    // ------------------------------------------------ producer warp: bulk copies only
    const int lane = t - ncpad;
    const TZ* Z = reinterpret_cast<const TZ*>(a.Z);
    int64_t it = 0, issued = 0;
    for (int64_t u = ub; u < ue && !failed; ++u) {
      const int chunk = (int)(u % a.C);
      const int seg = (int)((u / a.C) % a.nseg);
      const int64_t in = u / ((int64_t)a.C * a.nseg);
      const int64_t segrow0 = (int64_t)seg * a.SEG;
      const int64_t rows = (a.I1 - segrow0) < ta.ROWS ? (a.I1 - segrow0) : ta.ROWS;
      const uint32_t colbytes = (uint32_t)(rows * sizeof(TZ));
      const int64_t f0 = (a.F * chunk) / a.C, f1 = (a.F * (chunk + 1)) / a.C;
      // column of f = fs + lane (+32 ...), advanced without divisions
      int64_t o_lo = (f0 + lane) % a.Lp, o_hi = (f0 + lane) / a.Lp;
      const int64_t dq = SF / a.Lp, dr = SF % a.Lp;
      const int64_t q32 = 32 / a.Lp, r32 = 32 % a.Lp;
      for (int64_t fs = f0; fs < f1; fs += SF, ++it) {
        const int s = (int)(it % ta.S);
        if (it >= ta.S && !mbar_wait(&empty[s], (uint32_t)(((it / ta.S) - 1) & 1))) { failed = true; break; }
        const int nf = (int)((f1 - fs) < SF ? (f1 - fs) : SF);
        unsigned char* stage = smem_raw + ta.stage_off + (size_t)s * ta.stage_stride;
        const uint32_t wbytes = (uint32_t)(nf * RP * sizeof(Tab));
        if (!ta.contiguous) {
          int64_t lo = o_lo, hi = o_hi;
          for (int k = lane; k < nf; k += 32) {
            colbuf[k] = lo + a.Lp * in + a.Lp * a.In * hi;
            lo += r32;
            hi += q32;
            if (lo >= a.Lp) { lo -= a.Lp; ++hi; }
          }
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive_tx(&full[s], colbytes * (uint32_t)nf + wbytes);
          bulk_g2s(stage + ta.w_off, wfull + fs * RP, wbytes, &full[s]);
          if (ta.contiguous) {
            const int64_t col0 = o_lo + a.Lp * in + a.Lp * a.In * o_hi;
            bulk_g2s(stage, Z + col0 * a.I1 + segrow0, colbytes * (uint32_t)nf, &full[s]);
          }
        }
        __syncwarp();
        if (!ta.contiguous)
          for (int k = lane; k < nf; k += 32)
            bulk_g2s(stage + (size_t)k * colbytes, Z + colbuf[k] * a.I1 + segrow0, colbytes, &full[s]);
        if (lane != 0) mbar_arrive(&full[s]);
        __syncwarp();
        issued = it + 1;
        o_lo += dr;
        o_hi += dq;
        if (o_lo >= a.Lp) { o_lo -= a.Lp; ++o_hi; }
      }
    }
    if (lane == 0) {  // no copy may still be in flight when shared memory is reused or released
      for (int64_t j = (issued > ta.S ? issued - ta.S : 0); j < issued; ++j)
        if (!mbar_wait(&full[j % ta.S], (uint32_t)((j / ta.S) & 1))) failed = true;
    }
  } else {
    // ------------------------------------------------ consumers
    const int tx = t % a.TX, ty = t / a.TX;
    const int warp = t >> 5, lane = t & 31;
    V accm[QA][RP];
    V a1[QW][RP];
    // FP32: packed pairs (the V arrays then only carry the values into the reductions)
    constexpr int H = (PREC == P_FP32) ? HP : 1;
    unsigned long long acc2[QA][H];
    unsigned long long a1p[QW][H];
#pragma unroll
    for (int q = 0; q < QA; ++q)
#pragma unroll
      for (int h = 0; h < H; ++h) acc2[q][h] = 0ull;
#pragma unroll
    for (int q = 0; q < QW; ++q)
#pragma unroll
      for (int h = 0; h < H; ++h) a1p[q][h] = 0ull;
#pragma unroll
    for (int q = 0; q < QA; ++q)
#pragma unroll
      for (int r = 0; r < RP; ++r) accm[q][r] = Ops<V>::zero();
#pragma unroll
    for (int q = 0; q < QW; ++q)
#pragma unroll
      for (int r = 0; r < RP; ++r) a1[q][r] = Ops<V>::zero();
    int64_t it = 0;
    int cur_seg = -1;
    for (int64_t u = ub; u < ue && !failed; ++u) {
      const int chunk = (int)(u % a.C);
      const int seg = (int)((u / a.C) % a.nseg);
      const int64_t segrow0 = (int64_t)seg * a.SEG;
      const int64_t rows = (a.I1 - segrow0) < ta.ROWS ? (a.I1 - segrow0) : ta.ROWS;
      const uint32_t colbytes = (uint32_t)(rows * sizeof(TZ));
      const int64_t f0 = (a.F * chunk) / a.C, f1 = (a.F * (chunk + 1)) / a.C;
      const bool active = t < ta.NC && (int64_t)tx * VW < rows;
      if (!FIRST && seg != cur_seg) {
        cur_seg = seg;
        const int64_t row0 = segrow0 + (int64_t)tx * VW;
#pragma unroll
        for (int q = 0; q < QW; ++q)
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            double v = 0.0;
            if (active && r < a.R) v = a.A1[row0 + q + a.I1 * r];
            if constexpr (PREC == P_FP32) a1[q][r] = (float)v;
            else if constexpr (PREC == P_FP64) a1[q][r] = v;
            else a1[q][r] = df_from_double(v);
          }
        if constexpr (PREC == P_FP32) {
#pragma unroll
          for (int q = 0; q < QW; ++q)
#pragma unroll
            for (int h = 0; h < H; ++h) a1p[q][h] = pk2(a1[q][2 * h], a1[q][2 * h + 1]);
        }
      }
      for (int64_t fs = f0; fs < f1; fs += SF, ++it) {
        const int s = (int)(it % ta.S);
        if (!mbar_wait(&full[s], (uint32_t)((it / ta.S) & 1))) { failed = true; break; }
        const int nf = (int)((f1 - fs) < SF ? (f1 - fs) : SF);
        const unsigned char* stage = smem_raw + ta.stage_off + (size_t)s * ta.stage_stride;
        const Tab* W = reinterpret_cast<const Tab*>(stage + ta.w_off);
        if (active) {
#pragma unroll 2
          for (int j = 0; j < ta.CPS; ++j) {
            const int k = ty + a.TY * j;
            if (k >= nf) break;
            S zb[VW];
            load_z_s<TZ, VW, S>(reinterpret_cast<const TZ*>(stage + (size_t)k * colbytes) + (int64_t)tx * VW, zb);
            if constexpr (PREC == P_FP32) {
              // row of the Khatri-Rao table: the HP pairs that are computed
              const ulonglong2* wp = reinterpret_cast<const ulonglong2*>(W + k * RP);
              unsigned long long w2[2 * ((HP + 1) / 2)];
#pragma unroll
              for (int h = 0; h < (HP + 1) / 2; ++h) {
                const ulonglong2 v = wp[h];
                w2[2 * h] = v.x;
                w2[2 * h + 1] = v.y;
              }
#pragma unroll
              for (int q = 0; q < VW; ++q) {
                const unsigned long long zz = pk2(zb[q], zb[q]);
#pragma unroll
                for (int h = 0; h < HP; ++h) fma2(acc2[q][h], zz, w2[h]);
              }
            } else {
              V w[RP];
              load_row_s<PREC, RP>(W + k * RP, w);
              if constexpr (FIRST) {
#pragma unroll
                for (int q = 0; q < VW; ++q)
#pragma unroll
                  for (int r = 0; r < RP; ++r) Ops<V>::acc(accm[q][r], zb[q], w[r]);
              } else {
                V uu[RP];
#pragma unroll
                for (int r = 0; r < RP; ++r) {
                  if constexpr (PREC == P_DF) uu[r] = df_mul_f(zb[0], a1[0][r]);
                  else uu[r] = Ops<V>::mulz(zb[0], a1[0][r]);
                }
#pragma unroll
                for (int q = 1; q < QW; ++q)
#pragma unroll
                  for (int r = 0; r < RP; ++r) Ops<V>::acc(uu[r], zb[q], a1[q][r]);
#pragma unroll
                for (int r = 0; r < RP; ++r) {
                  Ops<V>::norm(uu[r]);
                  Ops<V>::acc(accm[0][r], uu[r], w[r], 0);
                }
              }
            }
          }
          if constexpr (PREC == P_DF) {
#pragma unroll
            for (int q = 0; q < QA; ++q)
#pragma unroll
              for (int r = 0; r < RP; ++r) Ops<V>::norm(accm[q][r]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      // consecutive units of the same output row and row segment accumulate in registers; the
      // run's total is written to the slot of its last unit, the other slots get zeros
      const bool run_end = (u + 1 >= ue) || ((u + 1) % a.C == 0);
      if constexpr (!FIRST) {
       if (!run_end) {
        Part* zout = reinterpret_cast<Part*>(a.partial) + (u * nwc + warp) * (int64_t)RP;
        if (lane < RP) zout[lane] = (Part)0;
       } else {
        if constexpr (PREC == P_FP32) {
          // sum over this thread's rows of A^(1)(i_1, r) * (sum over columns of z * w)
#pragma unroll
          for (int h = 0; h < H; ++h) {
            unsigned long long r2 = mul2(acc2[0][h], a1p[0][h]);
#pragma unroll
            for (int q = 1; q < VW; ++q) fma2(r2, acc2[q][h], a1p[q][h]);
            const float2 f = up2(r2);
            accm[0][2 * h] = f.x;
            accm[0][2 * h + 1] = f.y;
#pragma unroll
            for (int q = 0; q < VW; ++q) acc2[q][h] = 0ull;
          }
        }
        // per-warp partial of this unit: partial[(u * nwc + warp) * RP + r]
        Part* out = reinterpret_cast<Part*>(a.partial) + (u * nwc + warp) * (int64_t)RP;
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          Part v;
          if constexpr (PREC == P_FP32) v = accm[0][r];
          else v = (Part)Ops<V>::to_d(accm[0][r]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) out[r] = v;
          accm[0][r] = Ops<V>::zero();
        }
       }
      }
    }
    if constexpr (FIRST) {
      if constexpr (PREC == P_FP32) {
#pragma unroll
        for (int q = 0; q < QA; ++q)
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const float2 f = up2(acc2[q][h]);
            accm[q][2 * h] = f.x;
            accm[q][2 * h + 1] = f.y;
          }
      }
      // one unit per CTA: reduce the TY column groups of the same rows.  Only consumer warps
      // take part (named barrier 1); the reduction area starts after the mbarriers.
      asm volatile("bar.sync 1, %0;" ::"r"(ncpad) : "memory");
      Part* red = reinterpret_cast<Part*>(smem_raw + ta.red_off);
      const int64_t segrows = (int64_t)a.TX * VW;
      if (t < ta.NC) {
#pragma unroll
        for (int q = 0; q < QA; ++q)
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            Part v;
            if constexpr (PREC == P_FP32) v = accm[q][r];
            else v = (Part)Ops<V>::to_d(accm[q][r]);
            red[((int64_t)ty * segrows + (int64_t)tx * VW + q) * RP + r] = v;
          }
      }
      asm volatile("bar.sync 1, %0;" ::"r"(ncpad) : "memory");
      Part* out = reinterpret_cast<Part*>(a.partial) + ub * segrows * RP;
      for (int64_t e = t; e < segrows * RP; e += ncpad) {
        Part sum = 0;
        for (int g = 0; g < a.TY; ++g) sum += red[(int64_t)g * segrows * RP + e];
        out[e] = sum;
      }
    }
  }
  if (failed && ta.err) atomicOr(ta.err, 1);
  __syncthreads();
}

// ------------------------------------------------------------------ finish kernel
struct FinishArgs {
  const void* partial;
  int64_t rows;  // I_1 (mode 1) or I_n
  int64_t SEG;
  int nseg, C, R, RP, first, part8;
  int nw;        // per-unit partials per output (warps of the TMA kernel; 1 otherwise)
  double* M;
};

// One warp per output entry: lane l sums terms l, l+32, ... in order, then a fixed
// shuffle tree; the result does not depend on the launch geometry.
__global__ void k_mttkrp_finish(FinishArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t total = a.rows * a.R;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = wid; e < total; e += nwarps) {
    const int64_t i = e % a.rows;
    const int r = (int)(e / a.rows);
    double s = 0.0;
    if (a.first) {
      const int64_t seg = i / a.SEG, ii = i % a.SEG;
      for (int c = lane; c < a.C; c += 32) {
        const int64_t u = seg * a.C + c;
        const int64_t idx = (u * a.SEG + ii) * a.RP + r;
        s += a.part8 ? reinterpret_cast<const double*>(a.partial)[idx]
                     : (double)reinterpret_cast<const float*>(a.partial)[idx];
      }
    } else {
      const int64_t nterm = (int64_t)a.nseg * a.C * a.nw;
      for (int64_t q = lane; q < nterm; q += 32) {
        const int64_t u = i * a.nseg * a.C + q / a.nw;
        const int64_t idx = (u * a.nw + q % a.nw) * a.RP + r;
        s += a.part8 ? reinterpret_cast<const double*>(a.partial)[idx]
                     : (double)reinterpret_cast<const float*>(a.partial)[idx];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) a.M[i + a.rows * r] = s;
  }
}

// ------------------------------------------------------------------ dispatch
using MainFn = void (*)(MainArgs);

template <typename TZ, int PREC, int VW, bool FIRST>
static MainFn pick_rp1(int RP) {
  switch (RP) {
    case 4: return k_mttkrp_main<TZ, PREC, VW, 4, FIRST>;
    case 8: return k_mttkrp_main<TZ, PREC, VW, 8, FIRST>;
    case 12: return k_mttkrp_main<TZ, PREC, VW, 12, FIRST>;
    default: return k_mttkrp_main<TZ, PREC, VW, 16, FIRST>;
  }
}

static thread_local bool g_pick_first = false;

template <typename TZ, int PREC, int VW>
static MainFn pick_rp(int RP) {
  return g_pick_first ? pick_rp1<TZ, PREC, VW, true>(RP) : pick_rp1<TZ, PREC, VW, false>(RP);
}

static MainFn pick_kernel(const MttkrpPlan& p) {
  g_pick_first = p.mode == 0;
  if (p.prec == P_FP32) {
    if (p.zdtype == CPMG_F32) return p.VW == 4 ? pick_rp<float, P_FP32, 4>(p.RP) : pick_rp<float, P_FP32, 1>(p.RP);
    return p.VW == 2 ? pick_rp<double, P_FP32, 2>(p.RP) : pick_rp<double, P_FP32, 1>(p.RP);
  }
  if (p.prec == P_FP64) {
    if (p.zdtype == CPMG_F32) return p.VW == 2 ? pick_rp<float, P_FP64, 2>(p.RP) : pick_rp<float, P_FP64, 1>(p.RP);
    return p.VW == 2 ? pick_rp<double, P_FP64, 2>(p.RP) : pick_rp<double, P_FP64, 1>(p.RP);
  }
  // P_DF reads float tensors only
  return p.VW == 2 ? pick_rp<float, P_DF, 2>(p.RP) : pick_rp<float, P_DF, 1>(p.RP);
}

using TmaFn = void (*)(TmaArgs);

// The dynamic shared-memory cap is a property of the kernel function, shared by every plan
// that launches it, so it is raised once to the device's opt-in maximum (never lowered).
static int smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || x <= 0)
      x = 227 * 1024;
    v = x;
  }
  return v;
}

template <typename Fn>
static void raise_smem_cap(Fn fn) {
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
  cudaGetLastError();
}

template <typename TZ, int PREC, int VW, bool FIRST>
static TmaFn tma_rp1(int RP, int R) {
  if constexpr (PREC == P_FP32) {
    // odd ranks run one pair fewer than the padded row holds
    const bool odd_less = (R + 1) / 2 < RP / 2;
    switch (RP) {
      case 4: return odd_less ? k_mttkrp_tma<TZ, PREC, VW, 4, FIRST, 1> : k_mttkrp_tma<TZ, PREC, VW, 4, FIRST, 2>;
      case 8: return odd_less ? k_mttkrp_tma<TZ, PREC, VW, 8, FIRST, 3> : k_mttkrp_tma<TZ, PREC, VW, 8, FIRST, 4>;
      case 12: return odd_less ? k_mttkrp_tma<TZ, PREC, VW, 12, FIRST, 5> : k_mttkrp_tma<TZ, PREC, VW, 12, FIRST, 6>;
      default: return odd_less ? k_mttkrp_tma<TZ, PREC, VW, 16, FIRST, 7> : k_mttkrp_tma<TZ, PREC, VW, 16, FIRST, 8>;
    }
  }
  switch (RP) {
    case 4: return k_mttkrp_tma<TZ, PREC, VW, 4, FIRST>;
    case 8: return k_mttkrp_tma<TZ, PREC, VW, 8, FIRST>;
    case 12: return k_mttkrp_tma<TZ, PREC, VW, 12, FIRST>;
    default: return k_mttkrp_tma<TZ, PREC, VW, 16, FIRST>;
  }
}

template <typename TZ, int PREC, int VW>
static TmaFn tma_rp(const MttkrpPlan& p) {
  return p.mode == 0 ? tma_rp1<TZ, PREC, VW, true>(p.RP, p.R) : tma_rp1<TZ, PREC, VW, false>(p.RP, p.R);
}

static TmaFn pick_tma(const MttkrpPlan& p) {
  if (p.prec == P_FP32) {
    if (p.zdtype == CPMG_F32) return tma_rp<float, P_FP32, 4>(p);
    return tma_rp<double, P_FP32, 2>(p);
  }
  if (p.prec == P_FP64) {
    if (p.zdtype == CPMG_F32) return tma_rp<float, P_FP64, 2>(p);
    return tma_rp<double, P_FP64, 2>(p);
  }
  return tma_rp<float, P_DF, 2>(p);
}

static size_t main_smem(const MttkrpPlan& p, int block) {
  if (p.mode != 0) return (size_t)((block + 31) / 32) * p.RP * p.part_elem;
  return (size_t)p.TY * p.SEG * p.RP * p.part_elem;
}

int mttkrp_plan(const Shape& s, int mode, int R, int prec, int zdtype, const void* Z, int num_sms,
                MttkrpPlan* out, bool allow_tma, const MttkrpLimits* lim) {
  if (s.N < 2 || s.N > kMaxModes || mode < 0 || mode >= s.N || R < 1 || R > kMaxRank)
    return CPMG_INVALID_ARG;
  if (prec == P_DF && zdtype != CPMG_F32) prec = P_FP64;  // float64 tensors: native FP64
  MttkrpPlan p;
  p.mode = mode;
  p.prec = prec;
  p.zdtype = zdtype;
  p.R = R;
  p.RP = (R + 3) / 4 * 4;
  p.TS = p.RP;
  p.table_bytes = tab_size(prec);
  p.part_elem = part_size(prec);
  p.I1 = s.dims[0];
  const uintptr_t zp = reinterpret_cast<uintptr_t>(Z);
  if (prec == P_FP32 && zdtype == CPMG_F32) p.VW = (p.I1 % 4 == 0 && zp % 16 == 0) ? 4 : 1;
  else if (zdtype == CPMG_F64) p.VW = (p.I1 % 2 == 0 && zp % 16 == 0) ? 2 : 1;
  else p.VW = (p.I1 % 2 == 0 && zp % 8 == 0) ? 2 : 1;
  const int maxthreads = max_threads(prec, p.RP);
  const int64_t nvec = (p.I1 + p.VW - 1) / p.VW;
  p.TX = (int)std::min<int64_t>(nvec, maxthreads);
  p.SEG = (int64_t)p.TX * p.VW;
  p.nseg = (int)((p.I1 + p.SEG - 1) / p.SEG);
  // mode groups
  p.n_in = p.n_out = 0;
  if (mode == 0) {
    for (int m = 1; m < s.N - 1; ++m) p.in_modes[p.n_in++] = m;
    p.out_modes[p.n_out++] = s.N - 1;
  } else {
    for (int m = 1; m < mode; ++m) p.in_modes[p.n_in++] = m;
    for (int m = mode + 1; m < s.N; ++m) p.out_modes[p.n_out++] = m;
  }
  p.Lp = 1;
  for (int k = 0; k < p.n_in; ++k) p.Lp *= s.dims[p.in_modes[k]];
  p.G = 1;
  for (int k = 0; k < p.n_out; ++k) p.G *= s.dims[p.out_modes[k]];
  p.has_in = p.n_in > 0;
  p.has_out = p.n_out > 0;
  p.In = (mode == 0) ? 1 : s.dims[mode];
  const int64_t F = p.Lp * p.G;
  p.TY = (int)std::max<int64_t>(1, std::min<int64_t>(maxthreads / p.TX, F));
  if (lim && lim->ty > 0) p.TY = std::min(p.TY, lim->ty);
  // TMA staging: columns of whole 16-byte multiples, 16-byte aligned tensor
  const size_t esz = zdtype == CPMG_F64 ? 8 : 4;
  p.use_tma = allow_tma && ((size_t)p.I1 * esz) % 16 == 0 && zp % 16 == 0 &&
              (p.nseg == 1 || ((size_t)p.SEG * esz) % 16 == 0);
  if (p.use_tma) {
    p.ROWS = std::min<int64_t>(p.SEG, p.I1);
    const size_t colbytes = (size_t)p.ROWS * esz;
    // stages of ~48-64 KB: the per-stage hand-off, not the copy engine, limits small stages
    p.CPS = (int)std::max<size_t>(1, std::min<size_t>(8, 65536 / ((size_t)p.TY * colbytes)));
    if (lim && lim->cps > 0) p.CPS = std::min(p.CPS, lim->cps);
    const size_t SF = (size_t)p.TY * p.CPS;
    p.w_off = (uint32_t)((SF * colbytes + 127) / 128 * 128);
    p.stage_stride = (uint32_t)((p.w_off + SF * p.RP * p.table_bytes + 127) / 128 * 128);
    const size_t red = (mode == 0) ? (size_t)p.TY * p.SEG * p.RP * p.part_elem : 0;
    p.tab_smem = false;
    p.bar_off = 0;
    p.col_off = 256;
    p.stage_off = (uint32_t)((256 + SF * 8 + 127) / 128 * 128);
    const size_t budget = (size_t)smem_optin() - p.stage_off;
    p.S = (int)std::min<size_t>(8, budget / (size_t)p.stage_stride);
    if (p.S < 2) {
      p.use_tma = false;
    } else {
      p.red_off = p.stage_off;
      p.smem_tma = std::max<size_t>(p.stage_off + (size_t)p.S * p.stage_stride, p.stage_off + red);
      p.contiguous = p.nseg == 1 && (mode == 0 || mode == s.N - 1);
      p.nw = (mode == 0) ? 1 : ((p.TX * p.TY + 31) / 32);
      if (p.smem_tma > (size_t)smem_optin()) p.use_tma = false;
    }
    if (!p.use_tma) p.nw = 1;
  }
  // chunking: enough CTAs to fill the GPU a few times over with little tail waste
  const int block = p.use_tma ? (((p.TX * p.TY + 31) & ~31) + 32) : p.TX * p.TY;
  int per_sm = 1;
  if (p.use_tma) {
    TmaFn fn = pick_tma(p);
    raise_smem_cap(fn);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, p.smem_tma) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  } else {
    MainFn fn = pick_kernel(p);
    const size_t smem = main_smem(p, block);
    if (smem > 48 * 1024) raise_smem_cap(fn);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
  }
  cudaGetLastError();
  const int64_t slots = (int64_t)num_sms * per_sm;
  const int64_t base = p.In * p.nseg;
  const int64_t minper = p.use_tma ? (int64_t)p.TY * p.CPS : (int64_t)p.TY * 2;
  const int64_t cmax = std::max<int64_t>(1, std::min<int64_t>(F / std::max<int64_t>(minper, 1), 1024));
  int bestC = 1;
  if (p.use_tma && mode != 0) {
    // persistent CTAs over contiguous unit ranges: about 16 units per CTA balances the ranges
    const int64_t want = (16 * slots + base - 1) / base;
    bestC = (int)std::max<int64_t>(1, std::min<int64_t>(want, cmax));
  } else {
    double best = -1.0;
    for (int64_t c = 1; c <= cmax; ++c) {
      const int64_t units = base * c;
      const double waves = (double)units / (double)slots;
      // fraction of the SM-time the last wave keeps busy; below one wave, the share of SMs used
      const double eff = units < slots ? waves : waves / std::ceil(waves);
      if (eff > best + 1e-3) { best = eff; bestC = (int)c; }
      if (units > 16 * slots || best > 0.995) break;
    }
  }
  p.C = bestC;
  p.nunits = base * p.C;
  p.grid = (p.use_tma && mode != 0) ? std::min<int64_t>(p.nunits, slots) : p.nunits;
  *out = p;
  return CPMG_OK;
}

int mttkrp_run(const MttkrpPlan& p, const Shape& s, const void* Z, const double* const* A,
               const MttkrpScratch& w, double* M, cudaStream_t st, cudaEvent_t ev0,
               cudaEvent_t ev1, int* err, bool finish, bool ev_external) {
  // inside a stream capture, only an "external" event record becomes a node that fires on replay
  const unsigned evflags = ev_external ? cudaEventRecordExternal : cudaEventRecordDefault;
  // tables: Kin / Kout for the register-load kernel, the full row table W for the TMA kernel
  char* tb = reinterpret_cast<char*>(w.tables);
  void* kin = nullptr;
  void* kout = nullptr;
  void* wfull = nullptr;
  size_t off = 0;
  if (p.use_tma) {
    wfull = tb;
  } else {
    if (p.has_in) { kin = tb + off; off += ((size_t)p.Lp * p.TS * p.table_bytes + 255) / 256 * 256; }
    if (p.has_out) { kout = tb + off; }
  }
  if (p.use_tma || p.has_in || p.has_out) {
    TabArgs ta;
    for (int m = 0; m < s.N; ++m) { ta.f.p[m] = A[m]; ta.f.I[m] = s.dims[m]; }
    ta.R = p.R;
    ta.TS = p.TS;
    ta.n_in = p.n_in;
    ta.n_out = p.n_out;
    ta.n_all = p.n_in + p.n_out;
    for (int k = 0; k < kMaxModes; ++k) {
      ta.in_modes[k] = k < p.n_in ? p.in_modes[k] : 0;
      ta.out_modes[k] = k < p.n_out ? p.out_modes[k] : 0;
      ta.all_modes[k] = k < p.n_in ? p.in_modes[k] : (k < ta.n_all ? p.out_modes[k - p.n_in] : 0);
    }
    ta.Lp = p.Lp;
    ta.G = p.G;
    ta.kin = kin;
    ta.kout = kout;
    ta.wfull = wfull;
    const int64_t rows = p.use_tma ? p.Lp * p.G : std::max(p.has_in ? p.Lp : 0, p.has_out ? p.G : 0);
    const int nb = (int)std::min<int64_t>((rows * p.TS + 255) / 256, 2048);
    dim3 grid(std::max(nb, 1), 3);
    if (p.prec == P_FP32) k_tables<P_FP32><<<grid, 256, 0, st>>>(ta);
    else if (p.prec == P_FP64) k_tables<P_FP64><<<grid, 256, 0, st>>>(ta);
    else k_tables<P_DF><<<grid, 256, 0, st>>>(ta);
    CPMG_CUDA_TRY(cudaGetLastError());
  }
  MainArgs ma;
  ma.Z = Z;
  ma.A1 = A[0];
  ma.I1 = p.I1;
  ma.SEG = p.SEG;
  ma.In = p.In;
  ma.Lp = p.Lp;
  ma.G = p.G;
  ma.F = p.Lp * p.G;
  ma.TX = p.TX;
  ma.TY = p.TY;
  ma.nseg = p.nseg;
  ma.C = p.C;
  ma.R = p.R;
  ma.has_in = p.has_in;
  ma.has_out = p.has_out;
  ma.first = p.mode == 0;
  ma.kin = kin;
  ma.kout = kout;
  ma.partial = w.partial;
  if (ev0) CPMG_CUDA_TRY(cudaEventRecordWithFlags(ev0, st, evflags));
  if (p.use_tma) {
    TmaArgs ta;
    ta.m = ma;
    ta.CPS = p.CPS;
    ta.S = p.S;
    ta.NC = p.TX * p.TY;
    ta.contiguous = p.contiguous;
    ta.ROWS = p.ROWS;
    ta.stage_stride = p.stage_stride;
    ta.stage_off = p.stage_off;
    ta.red_off = p.red_off;
    ta.w_off = p.w_off;
    ta.w_stride = 0;
    ta.bar_off = p.bar_off;
    ta.col_off = p.col_off;
    ta.err = err;
    ta.nunits = p.nunits;
    ta.wfull = w.tables;
    ta.tab_smem = 0;
    ta.tab_off = 0;
    const int block = ((ta.NC + 31) & ~31) + 32;
    TmaFn fn = pick_tma(p);
    fn<<<(unsigned)p.grid, block, p.smem_tma, st>>>(ta);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      char what[256];
      snprintf(what, sizeof(what), "k_mttkrp_tma launch (mode %d prec %d grid %lld block %d smem %zu)", p.mode,
               p.prec, (long long)p.nunits, block, p.smem_tma);
      set_last_error(e, what, __FILE__, __LINE__);
      return CPMG_CUDA_ERROR;
    }
  } else {
    const int block = p.TX * p.TY;
    MainFn fn = pick_kernel(p);
    const size_t smem = main_smem(p, block);
    fn<<<(unsigned)p.nunits, block, smem, st>>>(ma);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      char what[256];
      snprintf(what, sizeof(what), "k_mttkrp_main launch (mode %d prec %d grid %lld block %d smem %zu)", p.mode,
               p.prec, (long long)p.nunits, block, smem);
      set_last_error(e, what, __FILE__, __LINE__);
      return CPMG_CUDA_ERROR;
    }
  }
  if (ev1) CPMG_CUDA_TRY(cudaEventRecordWithFlags(ev1, st, evflags));
  if (!finish) return CPMG_OK;
  FinishArgs fa;
  fa.partial = w.partial;
  fa.rows = (p.mode == 0) ? p.I1 : p.In;
  fa.SEG = p.SEG;
  fa.nseg = p.nseg;
  fa.C = p.C;
  fa.R = p.R;
  fa.RP = p.RP;
  fa.first = p.mode == 0;
  fa.part8 = p.part_elem == 8;
  fa.nw = p.nw;
  fa.M = M;
  const int64_t tot = fa.rows * p.R;
  const int nb = (int)std::min<int64_t>((tot * 32 + 255) / 256, 8192);
  k_mttkrp_finish<<<std::max(nb, 1), 256, 0, st>>>(fa);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

}  // namespace cpmg
