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
  size_t per = (mode == 0) ? (size_t)SEG * RP : (size_t)RP;
  return (size_t)nunits * per * part_elem;
}
size_t MttkrpPlan::tables_bytes() const {
  size_t rows = (size_t)(has_in ? Lp : 0) + (size_t)(has_out ? G : 0);
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
  __device__ static double to_d(float a) { return (double)a; }
};
template <> struct Ops<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  __device__ static double mulz(double z, double a) { return z * a; }
  __device__ static double fmaz(double z, double a, double c) { return __fma_rn(z, a, c); }
  __device__ static double to_d(double a) { return a; }
};
template <> struct Ops<df> {
  __device__ static df zero() { return {0.f, 0.f}; }
  __device__ static df mul(df a, df b) { return df_mul(a, b); }
  __device__ static df fma(df a, df b, df c) { return df_add(c, df_mul(a, b)); }
  __device__ static df fmaz(float z, df a, df c) { return df_add(c, df_mul_f(z, a)); }
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
  int64_t Lp, G;
  void* kin;
  void* kout;
};

template <int PREC>
__global__ void k_tables(TabArgs a) {
  using Tab = typename Tr<PREC>::Tab;
  const int which = blockIdx.y;  // 0: Kin, 1: Kout
  const int nm = which == 0 ? a.n_in : a.n_out;
  const int* modes = which == 0 ? a.in_modes : a.out_modes;
  const int64_t rows = which == 0 ? a.Lp : a.G;
  Tab* out = reinterpret_cast<Tab*>(which == 0 ? a.kin : a.kout);
  if (nm == 0 || out == nullptr) return;
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

// FP32 kernels with up to 12 padded ranks fit 128 registers at 512 threads; everything
// else runs 256-thread CTAs.
constexpr int max_threads(int prec, int RP) { return (prec == P_FP32 && RP <= 12) ? 512 : 256; }

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
            for (int r = 0; r < RP; ++r) accm[q][r] = Ops<V>::fmaz(zb[k][q], w[r], accm[q][r]);
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
            for (int r = 0; r < RP; ++r) uu[r] = Ops<V>::fmaz(zb[k][q], a1[q][r], uu[r]);
#pragma unroll
          for (int r = 0; r < RP; ++r) accm[0][r] = Ops<V>::fma(uu[r], w[r], accm[0][r]);
        }
      }
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

// ------------------------------------------------------------------ finish kernel
struct FinishArgs {
  const void* partial;
  int64_t rows;  // I_1 (mode 1) or I_n
  int64_t SEG;
  int nseg, C, R, RP, first, part8;
  double* M;
};

__global__ void k_mttkrp_finish(FinishArgs a) {
  const int64_t total = a.rows * a.R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % a.rows;
    const int r = (int)(e / a.rows);
    double s = 0.0;
    if (a.first) {
      const int64_t seg = i / a.SEG, ii = i % a.SEG;
      for (int c = 0; c < a.C; ++c) {
        const int64_t u = seg * a.C + c;
        const int64_t idx = (u * a.SEG + ii) * a.RP + r;
        s += a.part8 ? reinterpret_cast<const double*>(a.partial)[idx]
                     : (double)reinterpret_cast<const float*>(a.partial)[idx];
      }
    } else {
      for (int sg = 0; sg < a.nseg; ++sg)
        for (int c = 0; c < a.C; ++c) {
          const int64_t u = (i * a.nseg + sg) * a.C + c;
          const int64_t idx = u * a.RP + r;
          s += a.part8 ? reinterpret_cast<const double*>(a.partial)[idx]
                       : (double)reinterpret_cast<const float*>(a.partial)[idx];
        }
    }
    a.M[i + a.rows * r] = s;
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

static size_t main_smem(const MttkrpPlan& p, int block) {
  if (p.mode != 0) return (size_t)((block + 31) / 32) * p.RP * p.part_elem;
  return (size_t)p.TY * p.SEG * p.RP * p.part_elem;
}

int mttkrp_plan(const Shape& s, int mode, int R, int prec, int zdtype, const void* Z, int num_sms,
                MttkrpPlan* out) {
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
  // chunking: enough CTAs to fill the GPU a few times over with little tail waste
  const int block = p.TX * p.TY;
  MainFn fn = pick_kernel(p);
  const size_t smem = main_smem(p, block);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  cudaGetLastError();
  const int64_t slots = (int64_t)num_sms * per_sm;
  const int64_t base = p.In * p.nseg;
  const int64_t cmax = std::max<int64_t>(1, F / ((int64_t)p.TY * 2));
  int bestC = 1;
  double best = -1.0;
  for (int64_t c = 1; c <= std::min<int64_t>(cmax, 256); ++c) {
    const int64_t units = base * c;
    const double waves = (double)units / (double)slots;
    const double eff = waves / std::ceil(waves);
    // prefer fuller last waves; once there is at least one full wave, favour fewer units
    const double score = (units < slots ? waves : eff) - 1e-4 * (double)c;
    if (score > best + 1e-9) { best = score; bestC = (int)c; }
    if (units >= 4 * slots) break;
  }
  p.C = bestC;
  p.nunits = base * p.C;
  *out = p;
  return CPMG_OK;
}

int mttkrp_run(const MttkrpPlan& p, const Shape& s, const void* Z, const double* const* A,
               const MttkrpScratch& w, double* M, cudaStream_t st, cudaEvent_t ev0,
               cudaEvent_t ev1) {
  // tables
  char* tb = reinterpret_cast<char*>(w.tables);
  void* kin = nullptr;
  void* kout = nullptr;
  size_t off = 0;
  if (p.has_in) { kin = tb + off; off += ((size_t)p.Lp * p.TS * p.table_bytes + 255) / 256 * 256; }
  if (p.has_out) { kout = tb + off; }
  if (p.has_in || p.has_out) {
    TabArgs ta;
    for (int m = 0; m < s.N; ++m) { ta.f.p[m] = A[m]; ta.f.I[m] = s.dims[m]; }
    ta.R = p.R;
    ta.TS = p.TS;
    ta.n_in = p.n_in;
    ta.n_out = p.n_out;
    for (int k = 0; k < kMaxModes; ++k) {
      ta.in_modes[k] = k < p.n_in ? p.in_modes[k] : 0;
      ta.out_modes[k] = k < p.n_out ? p.out_modes[k] : 0;
    }
    ta.Lp = p.Lp;
    ta.G = p.G;
    ta.kin = kin;
    ta.kout = kout;
    const int64_t rows = std::max(p.has_in ? p.Lp : 0, p.has_out ? p.G : 0);
    const int nb = (int)std::min<int64_t>((rows * p.TS + 255) / 256, 1024);
    dim3 grid(std::max(nb, 1), 2);
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
  const int block = p.TX * p.TY;
  MainFn fn = pick_kernel(p);
  const size_t smem = main_smem(p, block);
  if (ev0) CPMG_CUDA_TRY(cudaEventRecord(ev0, st));
  fn<<<(unsigned)p.nunits, block, smem, st>>>(ma);
  CPMG_CUDA_TRY(cudaGetLastError());
  if (ev1) CPMG_CUDA_TRY(cudaEventRecord(ev1, st));
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
  fa.M = M;
  const int64_t tot = fa.rows * p.R;
  const int nb = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  k_mttkrp_finish<<<std::max(nb, 1), 256, 0, st>>>(fa);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

}  // namespace cpmg
