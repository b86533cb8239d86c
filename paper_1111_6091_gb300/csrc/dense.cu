// Small float64 kernels: Grams and Hadamard products (Eq. Gamma), the R x R solves of ALS
// (Section 3) and BNGS (Section 5.2), normalization and sorting (Eq. ALSnorm), gradient
// norms (Eq. gradEqn, Eq. gradConv), the direct objective (Eq. CPfunctional), small GEMMs
// for the factor transfers (Eqs. coarseapprox_new, CGC_new, FASrhs, FASCGC), and the
// interpolation / Cholesky transform of the setup phase (Sections 4.1, 4.3, 4.4).
#include "dense.cuh"
#include "linalg.cuh"

#include <algorithm>
#include <cmath>

namespace cpmg {

constexpr int kR = kMaxRank;

// ------------------------------------------------------------------ Grams
__global__ void k_grams(FactorPtrArgs f, unsigned mask) {
  int m = -1, cnt = 0;
  for (int k = 0; k < f.N; ++k)
    if (mask & (1u << k)) {
      if (cnt == (int)blockIdx.x) { m = k; break; }
      ++cnt;
    }
  if (m < 0) return;
  __shared__ double part[256];
  const int R = f.R;
  const int64_t I = f.I[m];
  const double* A = f.A[m];
  double* G = f.gram + (size_t)m * R * R;
  // each pair's rows are split into stripes summed in parallel, then the stripes in order:
  // short dependent float64 chains (GB300's float64 FMA latency is long)
  const int npairs = R * (R + 1) / 2;
  const int stripes = (int)blockDim.x / npairs > 0 ? (int)blockDim.x / npairs : 1;
  const int t = threadIdx.x;
  if (t < stripes * npairs) {
    const int p = t % npairs, sidx = t / npairs;
    int r = 0, q = p;
    while (q >= R - r) { q -= R - r; ++r; }
    const int c = r + q;
    double acc = 0.0;
    for (int64_t i = sidx; i < I; i += stripes) acc = __fma_rn(A[i + I * r], A[i + I * c], acc);
    part[t] = acc;
  }
  __syncthreads();
  for (int p = t; p < npairs; p += blockDim.x) {
    int r = 0, q = p;
    while (q >= R - r) { q -= R - r; ++r; }
    const int c = r + q;
    double acc = 0.0;
    for (int k = 0; k < stripes; ++k) acc += part[k * npairs + p];
    G[r * R + c] = acc;
    G[c * R + r] = acc;
  }
}

int launch_grams(const FactorSet& f, unsigned mask, cudaStream_t st) {
  int cnt = 0;
  for (int k = 0; k < f.N; ++k) cnt += (mask >> k) & 1u;
  if (cnt == 0) return CPMG_OK;
  k_grams<<<cnt, 256, 0, st>>>(fargs(f), mask);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

// Gamma^(n) into shared memory (R x R, row-major), Hadamard product over m != n.
__device__ void load_gamma(const FactorPtrArgs& f, int n, double* G) {
  const int R = f.R;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < f.N; ++m)
      if (m != n) v *= f.gram[(size_t)m * R * R + e];
    G[e] = v;
  }
}

// A^(n) = M Gamma^+ ; thread 0 factorizes, all threads apply to rows.
__global__ void k_als_update(FactorPtrArgs f, int n, const double* __restrict__ M, int* status) {
  __shared__ double G[kR * kR], L[kR * kR], Pi[kR * kR], V[kR * kR], w[kR];
  __shared__ int chol_ok;
  const int R = f.R;
  load_gamma(f, n, G);
  __syncthreads();
  if (threadIdx.x == 0) {
    double dmax = 0.0;
    for (int i = 0; i < R; ++i) dmax = fmax(dmax, G[i * R + i]);
    const double eps = 2.220446049250313e-16;
    const double thresh = R * eps * (dmax > 0 ? dmax : 1.0);
    int ok = 1;
    for (int i = 0; i < R * R; ++i) L[i] = 0.0;
    for (int j = 0; j < R && ok; ++j) {
      double s = G[j * R + j];
      for (int k = 0; k < j; ++k) s -= L[j * R + k] * L[j * R + k];
      if (!(s > thresh)) { ok = 0; break; }
      L[j * R + j] = sqrt(s);
      for (int i = j + 1; i < R; ++i) {
        double t = G[i * R + j];
        for (int k = 0; k < j; ++k) t -= L[i * R + k] * L[j * R + k];
        L[i * R + j] = t / L[j * R + j];
      }
    }
    chol_ok = ok;
    if (!ok) {
      double Gc[kR * kR];
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
      if (status && blockIdx.x == 0) atomicOr(status, 2);
    }
  }
  __syncthreads();
  const int64_t I = f.I[n];
  double* A = f.A[n];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x[kR];
    for (int r = 0; r < R; ++r) x[r] = M[i + I * r];
    if (chol_ok) {
      for (int r = 0; r < R; ++r) {  // L y = m
        double s = x[r];
        for (int k = 0; k < r; ++k) s -= L[r * R + k] * x[k];
        x[r] = s / L[r * R + r];
      }
      for (int r = R - 1; r >= 0; --r) {  // L^T z = y
        double s = x[r];
        for (int k = r + 1; k < R; ++k) s -= L[k * R + r] * x[k];
        x[r] = s / L[r * R + r];
      }
      for (int r = 0; r < R; ++r) A[i + I * r] = x[r];
    } else {
      for (int r = 0; r < R; ++r) {
        double s = 0.0;
        for (int k = 0; k < R; ++k) s += x[k] * Pi[k * R + r];
        A[i + I * r] = s;
      }
    }
  }
}

static int rows_grid(int64_t I, int block) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((I + block - 1) / block, 1024));
}

int launch_als_update(const FactorSet& f, int mode, const double* M, int* status, cudaStream_t st) {
  k_als_update<<<rows_grid(f.dims[mode], 128), 128, 0, st>>>(fargs(f), mode, M, status);
  CPMG_CUDA_TRY(cudaGetLastError());
  return launch_grams(f, 1u << mode, st);
}

// ------------------------------------------------------------------ Gauss-Seidel
__global__ void k_gs_update(FactorPtrArgs f, int n, const double* __restrict__ M,
                            const double* __restrict__ F, int sweeps) {
  __shared__ double G[kR * kR];
  const int R = f.R;
  load_gamma(f, n, G);
  __syncthreads();
  const int64_t I = f.I[n];
  double* A = f.A[n];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x[kR], b[kR];
    for (int r = 0; r < R; ++r) {
      x[r] = A[i + I * r];
      b[r] = M[i + I * r] + (F ? F[i + I * r] : 0.0);
    }
    for (int it = 0; it < sweeps; ++it)
      for (int r = 0; r < R; ++r) {
        double s = b[r];
        for (int k = 0; k < R; ++k)
          if (k != r) s -= G[r * R + k] * x[k];
        x[r] = s / G[r * R + r];
      }
    for (int r = 0; r < R; ++r) A[i + I * r] = x[r];
  }
}

int launch_gs_update(const FactorSet& f, int mode, const double* M, const double* F, int sweeps,
                     cudaStream_t st) {
  k_gs_update<<<rows_grid(f.dims[mode], 128), 128, 0, st>>>(fargs(f), mode, M, F, sweeps);
  CPMG_CUDA_TRY(cudaGetLastError());
  return launch_grams(f, 1u << mode, st);
}

// ------------------------------------------------------------------ normalization
__global__ void k_norm_scales(FactorPtrArgs f, double* scale) {
  __shared__ double nrm[kMaxModes * kR];
  const int R = f.R;
  for (int e = threadIdx.x; e < f.N * R; e += blockDim.x) {
    const int m = e / R, r = e % R;
    nrm[e] = sqrt(f.gram[(size_t)m * R * R + r * R + r]);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double prod = 1.0;
    for (int m = 0; m < f.N; ++m) prod *= nrm[m * R + r];
    const double lam = nth_root(prod, f.N);
    for (int m = 0; m < f.N; ++m) {
      const double nr = nrm[m * R + r];
      scale[m * R + r] = nr > 0 ? lam / nr : 1.0;
    }
  }
}

__global__ void k_apply_scales(FactorPtrArgs f, const double* scale) {
  const int R = f.R;
  int64_t total = 0;
  for (int m = 0; m < f.N; ++m) total += f.I[m] * R;
  const int64_t ngram = (int64_t)f.N * R * R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total + ngram;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < total) {
      int64_t rem = e;
      int m = 0;
      while (rem >= f.I[m] * R) { rem -= f.I[m] * R; ++m; }
      const int r = (int)(rem / f.I[m]);
      f.A[m][rem] *= scale[m * R + r];
    } else {
      const int64_t g = e - total;
      const int m = (int)(g / (R * R));
      const int rs = (int)(g % (R * R));
      f.gram[g] *= scale[m * R + rs / R] * scale[m * R + rs % R];
    }
  }
}

// scale buffer: N*R doubles placed right after the Grams (the FactorSet allocator reserves it)
int launch_normalize(const FactorSet& f, cudaStream_t st) {
  double* scale = f.gram + (size_t)f.N * f.R * f.R;
  k_norm_scales<<<1, 128, 0, st>>>(fargs(f), scale);
  CPMG_CUDA_TRY(cudaGetLastError());
  int64_t total = (int64_t)f.N * f.R * f.R;
  for (int m = 0; m < f.N; ++m) total += f.dims[m] * f.R;
  k_apply_scales<<<rows_grid(total, 256), 256, 0, st>>>(fargs(f), scale);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

// ------------------------------------------------------------------ sort
__global__ void k_sort(FactorPtrArgs f, double* scratch) {
  __shared__ int perm[kR];
  __shared__ double lam[kR];
  const int R = f.R;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double prod = 1.0;
    for (int m = 0; m < f.N; ++m) prod *= sqrt(f.gram[(size_t)m * R * R + r * R + r]);
    lam[r] = nth_root(prod, f.N);
    perm[r] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < R; ++i) {  // stable insertion sort, decreasing lambda
      const int p = perm[i];
      int j = i - 1;
      while (j >= 0 && lam[perm[j]] < lam[p]) { perm[j + 1] = perm[j]; --j; }
      perm[j + 1] = p;
    }
  }
  __syncthreads();
  // copy out, then gather
  int64_t off = 0;
  for (int m = 0; m < f.N; ++m) {
    const int64_t n = f.I[m] * R;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) scratch[off + e] = f.A[m][e];
    off += n;
  }
  const int64_t ng = (int64_t)f.N * R * R;
  for (int64_t e = threadIdx.x; e < ng; e += blockDim.x) scratch[off + e] = f.gram[e];
  __syncthreads();
  off = 0;
  for (int m = 0; m < f.N; ++m) {
    const int64_t I = f.I[m];
    for (int64_t e = threadIdx.x; e < I * R; e += blockDim.x) {
      const int64_t i = e % I;
      const int r = (int)(e / I);
      f.A[m][e] = scratch[off + i + I * perm[r]];
    }
    off += I * R;
  }
  for (int64_t e = threadIdx.x; e < ng; e += blockDim.x) {
    const int m = (int)(e / (R * R));
    const int rs = (int)(e % (R * R));
    const int r = rs / R, s = rs % R;
    f.gram[e] = scratch[off + (int64_t)m * R * R + perm[r] * R + perm[s]];
  }
}

int launch_sort(const FactorSet& f, double* scratch, cudaStream_t st) {
  k_sort<<<1, 1024, 0, st>>>(fargs(f), scratch);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

// ------------------------------------------------------------------ H and gradient norms
__global__ void k_fas_op(FactorPtrArgs f, int n, const double* __restrict__ M, double* H) {
  __shared__ double G[kR * kR];
  const int R = f.R;
  load_gamma(f, n, G);
  __syncthreads();
  const int64_t I = f.I[n];
  const double* A = f.A[n];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < I * R;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % I;
    const int r = (int)(e / I);
    double s = 0.0;
    for (int k = 0; k < R; ++k) s += A[i + I * k] * G[k * R + r];
    H[e] = s - M[e];
  }
}

int launch_fas_op(const FactorSet& f, int mode, const double* M, double* H, cudaStream_t st) {
  k_fas_op<<<rows_grid(f.dims[mode] * f.R, 256), 256, 0, st>>>(fargs(f), mode, M, H);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += sh[w];
  }
  return s;
}

__global__ void k_grad_sq(FactorPtrArgs f, int n, const double* __restrict__ M, double* out, int slot,
                          int slot_ag) {
  __shared__ double G[kR * kR];
  __shared__ double sh[32];
  const int R = f.R;
  load_gamma(f, n, G);
  __syncthreads();
  const int64_t I = f.I[n];
  const double* A = f.A[n];
  double acc = 0.0, acc_ag = 0.0;
  for (int64_t e = threadIdx.x; e < I * R; e += blockDim.x) {
    const int64_t i = e % I;
    const int r = (int)(e / I);
    double s = 0.0;
    for (int k = 0; k < R; ++k) s += A[i + I * k] * G[k * R + r];
    const double g = s - M[e];
    acc += g * g;
    acc_ag += s * s;
  }
  const double tot = block_sum(acc, sh);
  __syncthreads();
  const double tot_ag = block_sum(acc_ag, sh);
  if (threadIdx.x == 0) {
    out[slot] = tot;
    if (slot_ag >= 0) out[slot_ag] = tot_ag;
  }
}

int launch_grad_sq(const FactorSet& f, int mode, const double* M, double* out, int slot, cudaStream_t st,
                   int slot_ag) {
  k_grad_sq<<<1, 512, 0, st>>>(fargs(f), mode, M, out, slot, slot_ag);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

__global__ void k_sq_norm(const double* X, int64_t n, double* out, int slot) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc += X[e] * X[e];
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) out[slot] = tot;
}

int launch_sq_norm(const double* X, int64_t n, double* out, int slot, cudaStream_t st) {
  k_sq_norm<<<1, 512, 0, st>>>(X, n, out, slot);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

// ------------------------------------------------------------------ direct f
struct FArgs {
  const void* Z;
  int dtype;
  int N, R;
  int64_t dims[kMaxModes];
  const double* A[kMaxModes];
  int64_t ncols;
  double* partial;
};

__global__ void k_f_direct(FArgs a) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const int64_t I1 = a.dims[0];
  double acc_d = 0.0, acc_z = 0.0;
  for (int64_t col = (int64_t)blockIdx.x * nwarp + warp; col < a.ncols; col += (int64_t)gridDim.x * nwarp) {
    double w[kR];
    for (int r = 0; r < a.R; ++r) w[r] = 1.0;
    int64_t rem = col;
    for (int m = 1; m < a.N; ++m) {
      const int64_t i = rem % a.dims[m];
      rem /= a.dims[m];
      for (int r = 0; r < a.R; ++r) w[r] *= a.A[m][i + a.dims[m] * r];
    }
    for (int64_t i = lane; i < I1; i += 32) {
      double x = 0.0;
      for (int r = 0; r < a.R; ++r) x = __fma_rn(a.A[0][i + I1 * r], w[r], x);
      const double z = a.dtype == CPMG_F32 ? (double)reinterpret_cast<const float*>(a.Z)[col * I1 + i]
                                           : reinterpret_cast<const double*>(a.Z)[col * I1 + i];
      const double d = z - x;
      acc_d = __fma_rn(d, d, acc_d);
      acc_z = __fma_rn(z, z, acc_z);
    }
  }
  const double sd = block_sum(acc_d, sh);
  __syncthreads();
  const double sz = block_sum(acc_z, sh);
  if (threadIdx.x == 0) {
    a.partial[2 * blockIdx.x] = sd;
    a.partial[2 * blockIdx.x + 1] = sz;
  }
}

__global__ void k_f_final(const double* partial, int nb, double* out) {
  // strided per-thread sums, then a fixed-order tree over threads
  __shared__ double sd[256], sz[256];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    a += partial[2 * k];
    b += partial[2 * k + 1];
  }
  sd[threadIdx.x] = a;
  sz[threadIdx.x] = b;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sd[threadIdx.x] += sd[threadIdx.x + h];
      sz[threadIdx.x] += sz[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sd[0];
    out[1] = sz[0];
  }
}

int launch_f_direct(const Shape& s, const void* Z, int dtype, const FactorSet& f, double* partial,
                    double* out, cudaStream_t st) {
  FArgs a;
  a.Z = Z;
  a.dtype = dtype;
  a.N = s.N;
  a.R = f.R;
  int64_t ncols = 1;
  for (int m = 0; m < kMaxModes; ++m) {
    a.dims[m] = m < s.N ? s.dims[m] : 1;
    a.A[m] = m < s.N ? f.A[m] : nullptr;
    if (m >= 1 && m < s.N) ncols *= s.dims[m];
  }
  a.ncols = ncols;
  a.partial = partial;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 7) / 8, 1024));
  k_f_direct<<<nb, 256, 0, st>>>(a);
  CPMG_CUDA_TRY(cudaGetLastError());
  k_f_final<<<1, 256, 0, st>>>(partial, nb, out);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

// ------------------------------------------------------------------ small GEMM
__global__ void k_dgemm_small(bool tA, int64_t m, int64_t k, int64_t l, double alpha,
                              const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
                              int64_t ldb, double beta, double* C, int64_t ldc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    double s = 0.0;
    if (!tA)
      for (int64_t q = 0; q < l; ++q) s = __fma_rn(A[i + lda * q], B[q + ldb * j], s);
    else
      for (int64_t q = 0; q < l; ++q) s = __fma_rn(A[q + lda * i], B[q + ldb * j], s);
    C[i + ldc * j] = (beta == 0.0) ? alpha * s : alpha * s + beta * C[i + ldc * j];
  }
}

int launch_dgemm_small(bool transA, int64_t m, int64_t k, int64_t l, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                       cudaStream_t st) {
  if (m * k == 0) return CPMG_OK;
  k_dgemm_small<<<rows_grid(m * k, 256), 256, 0, st>>>(transA, m, k, l, alpha, A, lda, B, ldb, beta, C, ldc);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (b == 0.0) ? a * x[e] : a * x[e] + b * y[e];
}

int launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  if (n == 0) return CPMG_OK;
  k_axpby<<<rows_grid(n, 256), 256, 0, st>>>(n, a, x, b, y);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

int launch_copy_d(double* dst, const double* src, int64_t n, cudaStream_t st) {
  CPMG_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return CPMG_OK;
}

// ------------------------------------------------------------------ interpolation
struct InterpArgs {
  int64_t I;
  int R, nblk;
  const double* U[CPMG_MAX_TEST_BLOCKS + 1];
  const double* wblk;
  double* Pw;
};

__global__ void k_interp(InterpArgs a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.I;
       i += (int64_t)gridDim.x * blockDim.x) {
    if ((i & 1) == 0) {  // coarse point: identity row
      a.Pw[2 * i] = 1.0;
      a.Pw[2 * i + 1] = 0.0;
      continue;
    }
    const int64_t f0 = i - 1, f1 = i + 1;  // fine indices of the coarse neighbours
    const bool two = f1 < a.I;
    double n00 = 0, n01 = 0, n11 = 0, b0 = 0, b1 = 0;
    for (int k = 0; k < a.nblk; ++k) {
      const double w = a.wblk[k];
      const double* U = a.U[k];
      for (int r = 0; r < a.R; ++r) {
        const double y = U[i + a.I * r];
        const double x0 = U[f0 + a.I * r];
        const double x1 = two ? U[f1 + a.I * r] : 0.0;
        n00 += w * x0 * x0;
        n01 += w * x0 * x1;
        n11 += w * x1 * x1;
        b0 += w * x0 * y;
        b1 += w * x1 * y;
      }
    }
    double w0, w1 = 0.0;
    if (!two) {
      w0 = n00 > 0 ? b0 / n00 : 1.0;
    } else {
      const double tr = n00 + n11;
      const double disc = sqrt((n00 - n11) * (n00 - n11) + 4.0 * n01 * n01);
      const double lmax = 0.5 * (tr + disc), lmin = 0.5 * (tr - disc);
      if (lmax <= 0.0 || lmin <= lmax / 1e12) {
        w0 = w1 = 0.5;
      } else {
        const double det = n00 * n11 - n01 * n01;
        w0 = (n11 * b0 - n01 * b1) / det;
        w1 = (n00 * b1 - n01 * b0) / det;
      }
    }
    a.Pw[2 * i] = w0;
    a.Pw[2 * i + 1] = w1;
  }
}

int launch_interp(int64_t I, int R, int nblk, const double* const* Uptr, const double* wblk,
                  double* Pw, cudaStream_t st) {
  InterpArgs a;
  a.I = I;
  a.R = R;
  a.nblk = nblk;
  for (int k = 0; k < CPMG_MAX_TEST_BLOCKS + 1; ++k) a.U[k] = k < nblk ? Uptr[k] : nullptr;
  a.wblk = wblk;
  a.Pw = Pw;
  k_interp<<<rows_grid(I, 128), 128, 0, st>>>(a);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

// B = P^T P (tridiagonal), B = L L^T with L lower bidiagonal, R-hat = L^{-1} P^T.
__global__ void k_transform(int64_t I, const double* __restrict__ Pw, double* Rhat, double* work) {
  const int64_t Ic = (I + 1) / 2;
  double* Ld = work;        // diagonal of L
  double* Ls = work + Ic;   // subdiagonal: L(j+1, j)
  if (threadIdx.x == 0) {
    double prev_sub = 0.0;
    for (int64_t j = 0; j < Ic; ++j) {
      double bjj = 1.0;                       // coarse point 2j
      if (2 * j + 1 < I) { const double v = Pw[2 * (2 * j + 1)]; bjj += v * v; }      // slot 0 of 2j+1
      if (j > 0) { const double v = Pw[2 * (2 * j - 1) + 1]; bjj += v * v; }          // slot 1 of 2j-1
      const double d = sqrt(bjj - prev_sub * prev_sub);
      Ld[j] = d;
      double bnext = 0.0;                      // B(j, j+1) from fine point 2j+1
      if (j + 1 < Ic && 2 * j + 1 < I) bnext = Pw[2 * (2 * j + 1)] * Pw[2 * (2 * j + 1) + 1];
      const double sub = (j + 1 < Ic) ? bnext / d : 0.0;
      Ls[j] = sub;
      prev_sub = sub;
    }
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) {
    // column i of P^T: P(i, c0) = Pw0, P(i, c0+1) = Pw1 (fine points only)
    const int64_t c0 = i / 2;
    const double p0 = Pw[2 * i];
    const double p1 = (i & 1) ? Pw[2 * i + 1] : 0.0;
    for (int64_t j = 0; j < c0; ++j) Rhat[j + Ic * i] = 0.0;
    double y = p0 / Ld[c0];
    Rhat[c0 + Ic * i] = y;
    for (int64_t j = c0 + 1; j < Ic; ++j) {
      const double b = (j == c0 + 1) ? p1 : 0.0;
      y = (b - Ls[j - 1] * y) / Ld[j];
      Rhat[j + Ic * i] = y;
    }
  }
}

int launch_transform(int64_t I, const double* Pw, double* Rhat, double* work, cudaStream_t st) {
  k_transform<<<1, 256, 0, st>>>(I, Pw, Rhat, work);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

__global__ void k_block_weights(int nblk, const double* a2, const double* g2, const double* ag2, double tau2,
                                double* w) {
  const int k = threadIdx.x;
  if (k < nblk) {
    const double g = g2[k];
    double v = (g <= tau2 * ag2[k]) ? 1e30 : a2[k] / g;
    if (!(v <= 1e30)) v = 1e30;
    w[k] = v;
  }
}

int launch_block_weights(int nblk, const double* a2, const double* g2, const double* ag2, double tau,
                         double* w, cudaStream_t st) {
  k_block_weights<<<1, 32, 0, st>>>(nblk, a2, g2, ag2, tau * tau, w);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

}  // namespace cpmg
