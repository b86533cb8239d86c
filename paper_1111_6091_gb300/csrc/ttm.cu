// n-mode products Y = Z x_n R-hat for the coarse tensors of Eq. ctensor_transformed.
//
// With L = prod_{m<n} I_m and G = prod_{m>n} I_m, Y(l, c, g) = sum_i R-hat(c, i) Z(l, i, g):
//   n = 1 : one GEMM   Y (Ic x G)  = R-hat (Ic x I_1) * Z (I_1 x G)
//   n > 1 : G GEMMs    Y_g (L x Ic) = Z_g (L x I_n) * R-hat^T (I_n x Ic)
// This file holds the CUDA-core version (float or double accumulation in the tensor's
// type); the tcgen05 tensor-core version lives in ttm_tc.cu.
#include "ttm.cuh"

#include <algorithm>

namespace cpmg {

struct GemmArgs {
  const void* A;
  const void* B;
  void* C;
  int64_t M, N, K, batch;
  int64_t sAm, sAk, sAb, sBk, sBn, sBb, sCm, sCn, sCb;
  int a_is_d, b_is_d;  // operand stored as float64 (R-hat) instead of the tensor type
};

constexpr int BM = 64, BN = 64, BK = 16;

template <typename T>
__device__ __forceinline__ T ld_op(const void* p, int64_t off, int is_d) {
  return is_d ? (T)reinterpret_cast<const double*>(p)[off] : (T)reinterpret_cast<const T*>(p)[off];
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_strided(GemmArgs g) {
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tm = tid % 16, tn = tid / 16;
  const int64_t b = blockIdx.z;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const char* Ab = nullptr;
  (void)Ab;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  const bool a_mfast = g.sAm == 1;
  const bool b_kfast = g.sBk == 1;
  for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      int mm, kk;
      if (a_mfast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int64_t m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < g.M && k < g.K) ? ld_op<T>(g.A, b * g.sAb + m * g.sAm + k * g.sAk, g.a_is_d) : (T)0;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int nn, kk;
      if (b_kfast) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      const int64_t n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < g.N && k < g.K) ? ld_op<T>(g.B, b * g.sBb + k * g.sBk + n * g.sBn, g.b_is_d) : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tm + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tn + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
    }
    __syncthreads();
  }
  T* C = reinterpret_cast<T*>(g.C);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t m = m0 + tm + 16 * i, n = n0 + tn + 16 * j;
      if (m < g.M && n < g.N) C[b * g.sCb + m * g.sCm + n * g.sCn] = acc[i][j];
    }
}

static void mode_geometry(const Shape& s, int mode, int64_t* L, int64_t* G) {
  *L = 1;
  *G = 1;
  for (int m = 0; m < mode; ++m) *L *= s.dims[m];
  for (int m = mode + 1; m < s.N; ++m) *G *= s.dims[m];
}

int ttm_mode(const Shape& s, const void* Z, int dtype, int mode, const double* Rh, int64_t Ic, void* Y,
             int tensor_cores, void* tc_scratch, int* err, cudaEvent_t ev0, cudaEvent_t ev1, bool ev_external,
             cudaStream_t st) {
  if (tensor_cores) {
    int r = CPMG_UNSUPPORTED;
    if (dtype == CPMG_F32 && tc_scratch && ttm_tc_supported(s, dtype, mode, Ic))
      r = ttm_mode_tc(s, reinterpret_cast<const float*>(Z), mode, Rh, Ic, reinterpret_cast<float*>(Y), tc_scratch,
                      err, ev0, ev1, ev_external, st);
    if (r != CPMG_UNSUPPORTED || tensor_cores == 2) return r;
  }
  int64_t L, G;
  mode_geometry(s, mode, &L, &G);
  const int64_t In = s.dims[mode];
  GemmArgs g{};
  if (mode == 0) {
    g.A = Rh; g.a_is_d = 1; g.sAm = 1; g.sAk = Ic; g.sAb = 0;
    g.B = Z; g.b_is_d = dtype == CPMG_F64; g.sBk = 1; g.sBn = In; g.sBb = 0;
    g.C = Y; g.sCm = 1; g.sCn = Ic; g.sCb = 0;
    g.M = Ic; g.N = G; g.K = In; g.batch = 1;
  } else {
    g.A = Z; g.a_is_d = dtype == CPMG_F64; g.sAm = 1; g.sAk = L; g.sAb = L * In;
    g.B = Rh; g.b_is_d = 1; g.sBk = Ic; g.sBn = 1; g.sBb = 0;
    g.C = Y; g.sCm = 1; g.sCn = L; g.sCb = L * Ic;
    g.M = L; g.N = Ic; g.K = In; g.batch = G;
  }
  if (g.batch > 65535) {
    // fold the batch into launches of at most 65535
    for (int64_t b0 = 0; b0 < g.batch; b0 += 65535) {
      GemmArgs h = g;
      const int64_t nb = std::min<int64_t>(65535, g.batch - b0);
      const size_t esz = dtype == CPMG_F64 ? 8 : 4;
      h.A = reinterpret_cast<const char*>(g.A) + b0 * g.sAb * esz;
      h.C = reinterpret_cast<char*>(g.C) + b0 * g.sCb * esz;
      h.batch = nb;
      dim3 grid((unsigned)((h.M + BM - 1) / BM), (unsigned)((h.N + BN - 1) / BN), (unsigned)nb);
      if (dtype == CPMG_F64) k_gemm_strided<double><<<grid, 256, 0, st>>>(h);
      else k_gemm_strided<float><<<grid, 256, 0, st>>>(h);
      CPMG_CUDA_TRY(cudaGetLastError());
    }
    return CPMG_OK;
  }
  dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + BN - 1) / BN), (unsigned)g.batch);
  if (dtype == CPMG_F64) k_gemm_strided<double><<<grid, 256, 0, st>>>(g);
  else k_gemm_strided<float><<<grid, 256, 0, st>>>(g);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

size_t ttm_max_intermediate(const Shape& s, int dtype, const double* const* Rhat, const int64_t* Ic) {
  Shape cur = s;
  size_t mx = 0;
  const size_t esz = dtype == CPMG_F64 ? 8 : 4;
  for (int n = 0; n < s.N; ++n) {
    if (!Rhat[n]) continue;
    cur.dims[n] = Ic[n];
    mx = std::max(mx, (size_t)cur.numel() * esz);
  }
  return mx;
}

int ttm_order(const Shape& s, int dtype, const double* const* Rhat, const int64_t* Ic, int tensor_cores, int* order) {
  int k = 0;
  bool shrink = true;
  for (int n = 0; n < s.N; ++n)
    if (Rhat[n] && Ic[n] > s.dims[n]) shrink = false;
  if (tensor_cores && dtype == CPMG_F32 && s.N > 2 && Rhat[0] && shrink) {
    order[k++] = 0;
    for (int n = s.N - 1; n >= 1; --n)
      if (Rhat[n]) order[k++] = n;
  } else {
    for (int n = 0; n < s.N; ++n)
      if (Rhat[n]) order[k++] = n;
  }
  return k;
}

int ttm_restrict(const Shape& s, const void* Z, int dtype, const double* const* Rhat, const int64_t* Ic,
                 void* Y, void* tmp0, void* tmp1, int tensor_cores, void* tc_scratch, int* err,
                 const cudaEvent_t* ev, bool ev_external, cudaStream_t st) {
  int order[kMaxModes];
  const int k = ttm_order(s, dtype, Rhat, Ic, tensor_cores, order);
  if (k == 0) {
    const size_t esz = dtype == CPMG_F64 ? 8 : 4;
    CPMG_CUDA_TRY(cudaMemcpyAsync(Y, Z, s.numel() * esz, cudaMemcpyDeviceToDevice, st));
    return CPMG_OK;
  }
  Shape cur = s;
  const void* src = Z;
  int flip = 0;
  for (int j = 0; j < k; ++j) {
    const int n = order[j];
    void* dst = (j == k - 1) ? Y : (flip ? tmp1 : tmp0);
    CPMG_TRY(ttm_mode(cur, src, dtype, n, Rhat[n], Ic[n], dst, tensor_cores, tc_scratch, err,
                      ev ? ev[2 * n] : nullptr, ev ? ev[2 * n + 1] : nullptr, ev_external, st));
    cur.dims[n] = Ic[n];
    src = dst;
    flip ^= 1;
  }
  return CPMG_OK;
}

}  // namespace cpmg
