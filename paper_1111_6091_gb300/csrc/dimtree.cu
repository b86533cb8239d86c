// Contractions of the partial MTTKRP W = Z x_3 A^(3)^T for the first two modes (see dimtree.cuh).
//
// W is small next to Z (R I_1 I_2 float64 against I_1 I_2 I_3 values), so these kernels only need
// to read it once with coalesced loads and enough loads in flight; the float64 arithmetic is one
// FMA per loaded value.
#include "dimtree.cuh"
#include "mttkrp.cuh"

namespace cpmg {

constexpr int kDtPhases = 16;  // warps of the mode-0 kernel, each summing every 16th j

// mode 0: block (32 lanes along i) x (16 warps along j), one r per blockIdx.y
template <typename TW>
__global__ void __launch_bounds__(32 * kDtPhases) k_dt_mode0(const TW* __restrict__ W, int64_t I1, int64_t I2,
                                                           const double* __restrict__ V, double* out,
                                                           int64_t ld_row, int64_t ld_col) {
  __shared__ double red[kDtPhases][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  const int r = blockIdx.y;
  const TW* Wr = W + (int64_t)r * I1 * I2;
  const double* Vr = V + (int64_t)r * I2;
  double acc = 0.0;
  if (i < I1) {
    int64_t j = w;
    // four independent loads in flight per step, summed in a fixed order
    for (; j + 3 * kDtPhases < I2; j += 4 * kDtPhases) {
      const double a0 = Wr[i + I1 * j], a1 = Wr[i + I1 * (j + kDtPhases)];
      const double a2 = Wr[i + I1 * (j + 2 * kDtPhases)], a3 = Wr[i + I1 * (j + 3 * kDtPhases)];
      acc = fma(a0, Vr[j], acc);
      acc = fma(a1, Vr[j + kDtPhases], acc);
      acc = fma(a2, Vr[j + 2 * kDtPhases], acc);
      acc = fma(a3, Vr[j + 3 * kDtPhases], acc);
    }
    for (; j < I2; j += kDtPhases) acc = fma(Wr[i + I1 * j], Vr[j], acc);
  }
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && i < I1) {
    double s = red[0][lane];
    for (int q = 1; q < kDtPhases; ++q) s += red[q][lane];
    out[i * ld_row + (int64_t)r * ld_col] = s;
  }
}

// mode 1: one warp per (j, r), lanes along i, a fixed shuffle tree
template <typename TW>
__global__ void __launch_bounds__(256) k_dt_mode1(const TW* __restrict__ W, int64_t I1, int64_t I2, int R,
                                                  const double* __restrict__ V, double* out, int64_t ld_row,
                                                  int64_t ld_col) {
  const int lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= I2 * R) return;
  const int64_t j = item % I2;
  const int r = (int)(item / I2);
  const TW* col = W + (int64_t)r * I1 * I2 + I1 * j;
  const double* Vr = V + (int64_t)r * I1;
  double acc = 0.0;
  int64_t i = lane;
  for (; i + 96 < I1; i += 128) {
    const double a0 = col[i], a1 = col[i + 32], a2 = col[i + 64], a3 = col[i + 96];
    acc = fma(a0, Vr[i], acc);
    acc = fma(a1, Vr[i + 32], acc);
    acc = fma(a2, Vr[i + 64], acc);
    acc = fma(a3, Vr[i + 96], acc);
  }
  for (; i < I1; i += 32) acc = fma(col[i], Vr[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[j * ld_row + (int64_t)r * ld_col] = acc;
}

// ------------------------------------------------------------------ W = X C (one pass over X)
constexpr int kWThreads = 128;
constexpr int kWTile = 256;    // columns of C staged in shared memory at a time
// columns of X whose loads are in flight together: FP32 keeps 32 (two rows per thread) or 16 (four
// rows): the bytes in flight per SM set the streaming rate; the float-pair and float64
// accumulators leave registers for 8
constexpr int w_unroll(int prec, int vw) { return prec == P_FP32 ? (vw <= 2 ? 32 : 16) : 8; }

// accumulation per precision: FP32 fma; float pairs (the product's error and the TwoSum error of
// the running sum go to the low word, folded back after every group of columns); float64 fma
template <int PREC> struct WAcc;
template <> struct WAcc<P_FP32> {
  using A = float;
  using S = float;
  __device__ static S stage(double c) { return (float)c; }
  __device__ static void add(A& a, float z, S c) { a = __fmaf_rn(z, c, a); }
  __device__ static void add(A& a, double z, S c) { a = __fmaf_rn((float)z, c, a); }
  __device__ static void norm(A&) {}
  __device__ static double out(A a) { return (double)a; }
};
template <> struct WAcc<P_DF> {
  using A = df;
  using S = float2;
  __device__ static S stage(double c) {
    const df d = df_from_double(c);
    return make_float2(d.hi, d.lo);
  }
  __device__ static void add(A& a, float z, S c) {
    const float p = __fmul_rn(z, c.x);
    float e = __fmaf_rn(z, c.x, -p);
    e = __fmaf_rn(z, c.y, e);
    const df s = df_two_sum(a.hi, p);
    a.hi = s.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, e));
  }
  __device__ static void norm(A& a) { a = df_two_sum(a.hi, a.lo); }
  __device__ static double out(A a) { return df_to_double(a); }
};
template <> struct WAcc<P_FP64> {
  using A = double;
  using S = double;
  __device__ static S stage(double c) { return c; }
  __device__ static void add(A& a, float z, S c) { a = __fma_rn((double)z, c, a); }
  __device__ static void add(A& a, double z, S c) { a = __fma_rn(z, c, a); }
  __device__ static void norm(A&) {}
  __device__ static double out(A a) { return a; }
};

template <typename TZ, int VW> struct WVec;
template <typename TZ> struct WVec<TZ, 1> {
  TZ v[1];
  __device__ void load(const TZ* p) { v[0] = __ldg(p); }
};
template <> struct WVec<float, 2> {
  float v[2];
  __device__ void load(const float* p) {
    const float2 x = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = x.x, v[1] = x.y;
  }
};
template <> struct WVec<float, 4> {
  float v[4];
  __device__ void load(const float* p) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
  }
};
template <> struct WVec<double, 2> {
  double v[2];
  __device__ void load(const double* p) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = x.x, v[1] = x.y;
  }
};

// Thread t of block b owns rows p0 .. p0 + VW - 1, p0 = (b * kWThreads + t) * VW (P % VW == 0 when
// VW > 1), and walks every column k in increasing order: the sum over k has a fixed order.
template <typename TZ, int PREC, int VW, int RP>
__global__ void __launch_bounds__(kWThreads) k_dt_w(const TZ* __restrict__ X, int64_t P, int64_t K, int R,
                                                    const double* __restrict__ C, double* __restrict__ W) {
  using Acc = WAcc<PREC>;
  using S = typename Acc::S;
  __shared__ S cs[kWTile * RP];
  const int64_t p0 = ((int64_t)blockIdx.x * kWThreads + threadIdx.x) * VW;
  const bool live = p0 < P;
  typename Acc::A acc[VW][RP];
#pragma unroll
  for (int v = 0; v < VW; ++v)
#pragma unroll
    for (int r = 0; r < RP; ++r) acc[v][r] = typename Acc::A{};
  for (int64_t k0 = 0; k0 < K; k0 += kWTile) {
    const int kt = (int)((K - k0) < kWTile ? (K - k0) : kWTile);
    __syncthreads();
    for (int e = threadIdx.x; e < kt * RP; e += kWThreads) {
      const int kk = e / RP, r = e % RP;
      cs[e] = Acc::stage(r < R ? C[(k0 + kk) + K * r] : 0.0);
    }
    __syncthreads();
    if (!live) continue;
    const TZ* xp = X + p0 + P * k0;
    int kk = 0;
    constexpr int U = w_unroll(PREC, VW);
    for (; kk + U <= kt; kk += U) {
      WVec<TZ, VW> x[U];
#pragma unroll
      for (int u = 0; u < U; ++u) x[u].load(xp + P * (kk + u));
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const S* c = cs + (kk + u) * RP;
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const S cr = c[r];
#pragma unroll
          for (int v = 0; v < VW; ++v) Acc::add(acc[v][r], x[u].v[v], cr);
        }
      }
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int r = 0; r < RP; ++r) Acc::norm(acc[v][r]);
    }
    for (; kk < kt; ++kk) {
      WVec<TZ, VW> x;
      x.load(xp + P * kk);
      const S* c = cs + kk * RP;
#pragma unroll
      for (int r = 0; r < RP; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) Acc::add(acc[v][r], x.v[v], c[r]);
    }
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int r = 0; r < RP; ++r) Acc::norm(acc[v][r]);
  }
  if (!live) return;
#pragma unroll
  for (int r = 0; r < RP; ++r)
    if (r < R)
#pragma unroll
      for (int v = 0; v < VW; ++v) W[p0 + v + P * r] = Acc::out(acc[v][r]);
}

// RPMAX: the largest padded rank instantiated (8 for the float-pair two-row kernel, which is
// only launched up to R = 8: its wider instantiations would spill)
template <typename TZ, int PREC, int VW, int RPMAX = 16>
static void launch_w_rp(const TZ* X, int64_t P, int64_t K, int R, const double* C, double* W, cudaStream_t st) {
  const unsigned grid = (unsigned)((P / VW + kWThreads - 1) / kWThreads);
  if (R <= 4) k_dt_w<TZ, PREC, VW, 4><<<grid, kWThreads, 0, st>>>(X, P, K, R, C, W);
  else if (R <= 8 || RPMAX <= 8) k_dt_w<TZ, PREC, VW, 8><<<grid, kWThreads, 0, st>>>(X, P, K, R, C, W);
  else if constexpr (RPMAX > 8) {
    if (R <= 12) k_dt_w<TZ, PREC, VW, 12><<<grid, kWThreads, 0, st>>>(X, P, K, R, C, W);
    else k_dt_w<TZ, PREC, VW, 16><<<grid, kWThreads, 0, st>>>(X, P, K, R, C, W);
  }
}

// ------------------------------------------------------------------ W = X C, FP32, streamed ring
// The FP32 W pass with its loads taken off the arithmetic warps. CTA b owns the PB consecutive rows
// p_b .. p_b + PB - 1 (PB about P / SMs, so one CTA per SM and no second wave). Column k of those
// rows is one contiguous run of 4 PB bytes, and a producer warp streams KS such runs per stage
// with cp.async.bulk into a ring of S stages. Consumer thread t owns rows 4t .. 4t + 3 of the block
// and accumulates, column after column, exactly the FMAs of k_dt_w's FP32 path in the same order,
// so both give the same bits. Every wait is bounded (about 2 s); on expiry *err is set and the
// CTA unwinds, after the copies it issued have landed.
constexpr int kRingStages = 4;
constexpr int kRingCols = 8;     // columns per stage
constexpr int kRingMaxPB = 4 * (1024 - 32);
constexpr size_t kRingCBytes = 64 * 1024;  // C as float, K x RP, must fit

__device__ __forceinline__ uint32_t ring_su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t ring_gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool ring_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(ring_su32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}
__device__ bool ring_wait(uint64_t* bar, uint32_t parity, const int* fail) {
  if (ring_try(bar, parity)) return true;
  const uint64_t t0 = ring_gtime();
  while (true) {
    if (ring_try(bar, parity)) return true;
    if ((fail && *reinterpret_cast<const volatile int*>(fail)) || ring_gtime() - t0 > 2000000000ull) return false;
  }
}

template <int RP>
__global__ void k_dt_w_ring(const float* __restrict__ X, int64_t P, int64_t K, int R, const double* __restrict__ C,
                            double* __restrict__ W, int PB, int nc, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kRingStages;
  int* fail = reinterpret_cast<int*>(smem + 128);
  float* cs = reinterpret_cast<float*>(smem + 256);
  const size_t cbytes = ((size_t)K * RP * 4 + 127) & ~(size_t)127;
  unsigned char* ring = smem + 256 + cbytes;
  const uint32_t stage_bytes = (uint32_t)kRingCols * (uint32_t)PB * 4u;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int ncw = nc >> 5;  // consumer warps
  const int64_t p0 = (int64_t)blockIdx.x * PB;
  const int plen = (int)((P - p0) < PB ? (P - p0) : PB);
  const int nst = (int)((K + kRingCols - 1) / kRingCols);
  if (t == 0) {
    for (int s2 = 0; s2 < kRingStages; ++s2) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ring_su32(&full[s2])), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ring_su32(&empty[s2])), "r"(ncw) : "memory");
    }
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int64_t e = t; e < K * RP; e += blockDim.x) {
    const int64_t k = e / RP;
    const int r = (int)(e % RP);
    cs[e] = r < R ? (float)C[k + K * r] : 0.f;
  }
  __syncthreads();
  if (warp == ncw) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int it = 0;
      for (; it < nst; ++it) {
        const int slot = it % kRingStages;
        if (it >= kRingStages &&
            !ring_wait(&empty[slot], (uint32_t)(((it / kRingStages) - 1) & 1), fail)) {
          atomicOr(fail, 1);
          break;
        }
        const int64_t k0 = (int64_t)it * kRingCols;
        const int cols = (int)((K - k0) < kRingCols ? (K - k0) : kRingCols);
        const uint32_t bytes = (uint32_t)plen * 4u;
        unsigned char* st = ring + (size_t)slot * stage_bytes;
        asm volatile("{\n\t.reg .b64 sx;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 sx, [%0], %1;\n\t}" ::"r"(
                         ring_su32(&full[slot])),
                     "r"(bytes * (uint32_t)cols)
                     : "memory");
        for (int j = 0; j < cols; ++j)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  ring_su32(st + (size_t)j * PB * 4)),
              "l"(X + p0 + P * (k0 + j)), "r"(bytes), "r"(ring_su32(&full[slot]))
              : "memory");
      }
      // copies still in flight must land before the CTA exits (only their own phase ends this)
      for (int j = (it > kRingStages ? it - kRingStages : 0); j < it; ++j)
        if (!ring_wait(&full[j % kRingStages], (uint32_t)((j / kRingStages) & 1), nullptr)) atomicOr(fail, 1);
    }
  } else {
    // ---------------------------------------------------------------- consumers
    const int q = 4 * t;  // first of this thread's four rows in the block
    const bool live = q < plen;
    float acc[4][RP];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int r = 0; r < RP; ++r) acc[v][r] = 0.f;
    for (int it = 0; it < nst; ++it) {
      const int slot = it % kRingStages;
      int ok = 1;
      if (lane == 0) ok = ring_wait(&full[slot], (uint32_t)((it / kRingStages) & 1), fail) ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        if (lane == 0) atomicOr(fail, 1);
        break;
      }
      __syncwarp();
      const int64_t k0 = (int64_t)it * kRingCols;
      const int cols = (int)((K - k0) < kRingCols ? (K - k0) : kRingCols);
      if (live) {
        const unsigned char* st = ring + (size_t)slot * stage_bytes + (size_t)q * 4;
        // one column: four rows times RP coefficients, the coefficients read four at a time
        auto column = [&](int j) {
          const float4 x = *reinterpret_cast<const float4*>(st + (size_t)j * PB * 4);
          const float4* c4 = reinterpret_cast<const float4*>(cs + (k0 + j) * RP);
#pragma unroll
          for (int r4 = 0; r4 < RP / 4; ++r4) {
            const float4 cq = c4[r4];
            const float cr[4] = {cq.x, cq.y, cq.z, cq.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int r = 4 * r4 + i;
              acc[0][r] = __fmaf_rn(x.x, cr[i], acc[0][r]);
              acc[1][r] = __fmaf_rn(x.y, cr[i], acc[1][r]);
              acc[2][r] = __fmaf_rn(x.z, cr[i], acc[2][r]);
              acc[3][r] = __fmaf_rn(x.w, cr[i], acc[3][r]);
            }
          }
        };
        if (cols == kRingCols) {
#pragma unroll
          for (int j = 0; j < kRingCols; ++j) column(j);
        } else {
          for (int j = 0; j < cols; ++j) column(j);
        }
      }
      __syncwarp();
      if (lane == 0)
        asm volatile("{\n\t.reg .b64 sx;\n\tmbarrier.arrive.shared::cta.b64 sx, [%0];\n\t}" ::"r"(
                         ring_su32(&empty[slot]))
                     : "memory");
    }
    if (live && !*reinterpret_cast<volatile int*>(fail)) {
#pragma unroll
      for (int r = 0; r < RP; ++r)
        if (r < R)
#pragma unroll
          for (int v = 0; v < 4; ++v) W[p0 + q + v + P * r] = (double)acc[v][r];
    }
  }
  __syncthreads();
  if (t == 0 && *fail && err) atomicOr(err, 1);
}

// launches the ring kernel when the shapes suit it; false: use k_dt_w
static bool launch_w_ring(const float* X, int64_t P, int64_t K, int R, const double* C, double* W, int num_sms,
                          int* err, cudaStream_t st) {
  const int RP = R <= 4 ? 4 : R <= 8 ? 8 : R <= 12 ? 12 : 16;
  if (P % 4 != 0 || reinterpret_cast<uintptr_t>(X) % 16 != 0 || (size_t)K * RP * 4 > kRingCBytes || num_sms < 1)
    return false;
  int64_t PB = ((P + num_sms - 1) / num_sms + 3) / 4 * 4;
  if (PB < 256) return false;  // too few rows per CTA for the copies to pay
  if (PB > kRingMaxPB) PB = kRingMaxPB;
  const int nc = (int)((PB / 4 + 31) / 32 * 32);
  const size_t cbytes = ((size_t)K * RP * 4 + 127) & ~(size_t)127;
  const size_t smem = 256 + cbytes + (size_t)kRingStages * kRingCols * PB * 4;
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) optin = 0;
  cudaGetLastError();
  if (smem > (size_t)optin) return false;
  const unsigned grid = (unsigned)((P + PB - 1) / PB);
  const unsigned block = (unsigned)(nc + 32);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, block, smem, st>>>(X, P, K, R, C, W, (int)PB, nc, err);
  };
  if (RP == 4) go(k_dt_w_ring<4>);
  else if (RP == 8) go(k_dt_w_ring<8>);
  else if (RP == 12) go(k_dt_w_ring<12>);
  else go(k_dt_w_ring<16>);
  return true;
}

int launch_dt_w(const void* X, int zdtype, int64_t P, int64_t K, int R, const double* C, int prec, double* W,
                int num_sms, cudaStream_t st, int* err) {
  if (R < 1 || R > 16 || P < 1 || K < 1) return CPMG_INVALID_ARG;
  if (zdtype == CPMG_F64 && prec == P_DF) prec = P_FP64;
  const uintptr_t xa = reinterpret_cast<uintptr_t>(X);
  // rows per thread: wider vector loads while the grid still covers every SM about twice
  auto fits = [&](int vw, int align) {
    return P % vw == 0 && xa % align == 0 && (P / vw + kWThreads - 1) / kWThreads >= 2 * (int64_t)num_sms;
  };
  if (zdtype == CPMG_F64) {
    const double* x = static_cast<const double*>(X);
    const bool v2 = fits(2, 16);
    if (prec == P_FP32) v2 ? launch_w_rp<double, P_FP32, 2>(x, P, K, R, C, W, st) : launch_w_rp<double, P_FP32, 1>(x, P, K, R, C, W, st);
    else v2 ? launch_w_rp<double, P_FP64, 2>(x, P, K, R, C, W, st) : launch_w_rp<double, P_FP64, 1>(x, P, K, R, C, W, st);
  } else {
    const float* x = static_cast<const float*>(X);
    // two rows per thread when that still gives about four CTAs per SM: twice the resident warps
    // of four rows per thread for the same bytes in flight
    const bool v2many = P % 2 == 0 && xa % 8 == 0 && (P / 2 + kWThreads - 1) / kWThreads >= 4 * (int64_t)num_sms;
    const int vw = v2many ? 2 : fits(4, 16) ? 4 : fits(2, 8) ? 2 : 1;
    switch (prec) {
      case P_FP32:
        if (launch_w_ring(x, P, K, R, C, W, num_sms, err, st)) break;
        vw == 4 ? launch_w_rp<float, P_FP32, 4>(x, P, K, R, C, W, st)
                : vw == 2 ? launch_w_rp<float, P_FP32, 2>(x, P, K, R, C, W, st)
                          : launch_w_rp<float, P_FP32, 1>(x, P, K, R, C, W, st);
        break;
      case P_DF:  // two rows of float-pair accumulators fit the registers up to R = 8
        (vw >= 2 && R <= 8) ? launch_w_rp<float, P_DF, 2, 8>(x, P, K, R, C, W, st)
                            : launch_w_rp<float, P_DF, 1>(x, P, K, R, C, W, st);
        break;
      default:
        vw >= 2 ? launch_w_rp<float, P_FP64, 2>(x, P, K, R, C, W, st) : launch_w_rp<float, P_FP64, 1>(x, P, K, R, C, W, st);
    }
  }
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

// mode 3 from V = Z x_1 A^(1)^T (R x I2 x I3, r fastest): out(k, r) = sum_j V(r, j, k) U(j, r).
// Thread (k, r), r fastest, so a warp reads whole r-runs of V; j in increasing order.
__global__ void __launch_bounds__(256) k_dt_vmode(const float* __restrict__ V, int64_t I2, int64_t I3, int R,
                                                  const double* __restrict__ U, double* out, int64_t ld_row,
                                                  int64_t ld_col) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= I3 * R) return;
  const int r = (int)(t % R);
  const int64_t k = t / R;
  const float* v = V + (int64_t)R * I2 * k + r;
  const double* u = U + (int64_t)r * I2;
  double acc = 0.0;
  int64_t j = 0;
  for (; j + 3 < I2; j += 4) {
    const double a0 = v[R * j], a1 = v[R * (j + 1)], a2 = v[R * (j + 2)], a3 = v[R * (j + 3)];
    acc = fma(a0, u[j], acc);
    acc = fma(a1, u[j + 1], acc);
    acc = fma(a2, u[j + 2], acc);
    acc = fma(a3, u[j + 3], acc);
  }
  for (; j < I2; ++j) acc = fma((double)v[R * j], u[j], acc);
  out[k * ld_row + (int64_t)r * ld_col] = acc;
}

template <typename TW>
static int dt_contract(const TW* W, int64_t I1, int64_t I2, int R, const double* V, int mode, double* out,
                       int64_t ld_row, int64_t ld_col, cudaStream_t st) {
  if (I1 < 1 || I2 < 1 || R < 1 || (mode != 0 && mode != 1)) return CPMG_INVALID_ARG;
  if (mode == 0) {
    const dim3 grid((unsigned)((I1 + 31) / 32), (unsigned)R);
    k_dt_mode0<TW><<<grid, 32 * kDtPhases, 0, st>>>(W, I1, I2, V, out, ld_row, ld_col);
  } else {
    const int64_t items = I2 * R;
    k_dt_mode1<TW><<<(unsigned)((items + 7) / 8), 256, 0, st>>>(W, I1, I2, R, V, out, ld_row, ld_col);
  }
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

int launch_dt_contract(const double* W, int64_t I1, int64_t I2, int R, const double* V, int mode, double* out,
                       int64_t ld_row, int64_t ld_col, cudaStream_t st) {
  return dt_contract(W, I1, I2, R, V, mode, out, ld_row, ld_col, st);
}

int launch_dt_contract_f(const float* W, int64_t I1, int64_t I2, int R, const double* V, int mode, double* out,
                         int64_t ld_row, int64_t ld_col, cudaStream_t st) {
  return dt_contract(W, I1, I2, R, V, mode, out, ld_row, ld_col, st);
}

int launch_dt_vmode(const float* V, int64_t I2, int64_t I3, int R, const double* U, double* out, int64_t ld_row,
                    int64_t ld_col, cudaStream_t st) {
  if (I2 < 1 || I3 < 1 || R < 1) return CPMG_INVALID_ARG;
  const int64_t n = I3 * R;
  k_dt_vmode<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(V, I2, I3, R, U, out, ld_row, ld_col);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

// transposed copy: dst (R x I, column-major) = src^T (src: I x R column-major)
__global__ void k_transpose_d(const double* __restrict__ src, int64_t I, int R, double* __restrict__ dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= I * R) return;
  const int r = (int)(t % R);
  const int64_t i = t / R;
  dst[r + (int64_t)R * i] = src[i + I * r];
}

int launch_transpose_d(const double* src, int64_t I, int R, double* dst, cudaStream_t st) {
  const int64_t n = I * R;
  k_transpose_d<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, I, R, dst);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

}  // namespace cpmg
