// One kernel for what follows an MTTKRP inside a relaxation sweep: the ordered reduction of
// the MTTKRP partial sums into M = Z_(n) Phi^(n), the R x R solve of the ALS update
// (A^(n) <- M Gamma^+, Section 3) or the Gauss-Seidel sweeps of BNGS (A^(n) Gamma = M + F,
// Section 5.2), the refresh of Upsilon^(n) = A^(n)^T A^(n) (Eq. Gamma), and optionally the
// normalization of Eq. ALSnorm that ends an ALS sweep.
//
// Every block inverts Gamma^(n) (the Hadamard product of the other Grams) in shared memory with
// R*R threads, then each warp handles rows of A^(n): lanes sum the partials of the row in a
// fixed order, a shuffle tree combines them, and lane r forms component r of M(i,:) Gamma^+.
// GB300's float64 units have long dependent latencies (tens of cycles per FMA, hundreds per
// division or square root), so the kernel keeps serial float64 chains short.  Each block then
// forms the Gram of its own rows; the last block to finish (atomic ticket) sums the block Grams
// in block order.  The summation orders depend only on the shapes, so results are bitwise
// reproducible.
#include "fused.cuh"
#include "linalg.cuh"

#include <algorithm>

namespace cpmg {

constexpr int kR = kMaxRank;
constexpr int kMaxThreads = 256;  // R*R threads invert Gamma, so R = 16 needs 256

struct FuseArgs {
  FactorPtrArgs f;
  int n;                  // mode
  int kind;               // 0: ALS (pseudoinverse), 1: Gauss-Seidel on A Gamma = M + F
  int gs_sweeps;
  const double* F;        // BNGS right-hand side (I_n x R) or null
  double* M;              // optional copy of M (I_n x R) or null
  const void* partial;
  int part8, first, nseg, C, nw, RP;
  int64_t SEG;
  double* gscratch;       // gridDim.x x R(R+1)/2
  int* ticket;
  int* status;
  int normalize;          // 1: apply Eq. ALSnorm to the whole factor set after the update
};

__device__ __forceinline__ double part_at(const FuseArgs& a, int64_t idx) {
  return a.part8 ? reinterpret_cast<const double*>(a.partial)[idx]
                 : (double)reinterpret_cast<const float*>(a.partial)[idx];
}

// Rarely taken or once-per-launch paths live in separate, non-inlined functions: the kernel
// runs once per mode update with a cold instruction cache, so the hot path is kept short.

// singular Gamma (thread 0): W = Gamma^+ from a symmetric eigendecomposition
__device__ __noinline__ void pinv_fallback(const double* G, double* W, double* V, double* w, int R) {
  const double eps = 2.220446049250313e-16;
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
      W[i * R + j] = s;
    }
}

// Gauss-Seidel sweeps of BNGS on one row: x Gamma = m + f, from the current row of A
__device__ __noinline__ void gs_row(const double* m, const FuseArgs& a, double* A, int64_t i, int64_t I,
                                    const double* G, const double* dinv) {
  const int R = a.f.R;
  double x[kR], b[kR];
  for (int r = 0; r < R; ++r) {
    x[r] = A[i + I * r];
    b[r] = m[r] + (a.F ? a.F[i + I * r] : 0.0);
  }
  for (int it = 0; it < a.gs_sweeps; ++it)
    for (int r = 0; r < R; ++r) {
      double t = b[r];
      for (int k = 0; k < R; ++k)
        if (k != r) t -= G[r * R + k] * x[k];
      x[r] = t * dinv[r];
    }
  for (int r = 0; r < R; ++r) A[i + I * r] = x[r];
}

// Eq. ALSnorm on the whole factor set (block-wide); scales also stored after the Grams
__device__ __noinline__ void normalize_all(const FuseArgs& a, double* nrm, double* sc) {
  const int N = a.f.N, R = a.f.R;
  for (int e = threadIdx.x; e < N * R; e += blockDim.x) {
    const int m = e / R, r = e % R;
    nrm[e] = sqrt(a.f.gram[(size_t)m * R * R + r * R + r]);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double prod = 1.0;
    for (int m = 0; m < N; ++m) prod *= nrm[m * R + r];
    const double lam = nth_root(prod, N);
    for (int m = 0; m < N; ++m) {
      const double nr = nrm[m * R + r];
      const double v = nr > 0 ? lam / nr : 1.0;
      sc[m * R + r] = v;
      a.f.gram[(size_t)N * R * R + m * R + r] = v;
    }
  }
  __syncthreads();
  for (int m = 0; m < N; ++m) {
    const int Im = (int)a.f.I[m];
    double* Am = a.f.A[m];
    for (int e = threadIdx.x; e < Im * R; e += blockDim.x) Am[e] *= sc[m * R + e / Im];
  }
  for (int e = threadIdx.x; e < N * R * R; e += blockDim.x) {
    const int m = e / (R * R), rs = e % (R * R);
    a.f.gram[e] *= sc[m * R + rs / R] * sc[m * R + rs % R];
  }
}

// RP: padded rank (4, 8, 12 or 16) sizing the per-row register arrays
template <int RP>
__global__ void __launch_bounds__(kMaxThreads) k_finish_update(FuseArgs a) {
  __shared__ double G[RP * RP], W[RP * RP], V[RP * RP], w[RP], dinv[RP];
  __shared__ double nrm[kMaxModes * RP], sc[kMaxModes * RP];
  __shared__ int inv_fail;
  __shared__ bool last;
  __shared__ double stripe[kMaxThreads];
  const int nwarps = blockDim.x >> 5;
  const int R = a.f.R;
  const int n = a.n;
  const int64_t I = a.f.I[n];
  double* A = a.f.A[n];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // Gamma^(n): the Hadamard product of the other Grams
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < a.f.N; ++m)
      if (m != n) v *= a.f.gram[(size_t)m * R * R + e];
    G[e] = v;
    W[e] = v;
  }
  __syncthreads();
  if (a.kind == 0) {
    double dmax = 0.0;
    for (int i = 0; i < R; ++i) dmax = fmax(dmax, G[i * R + i]);
    const double thresh = R * 2.220446049250313e-16 * (dmax > 0 ? dmax : 1.0);
    if (!gj_inverse(W, R, thresh, &inv_fail) && threadIdx.x == 0) {
      pinv_fallback(G, W, V, w, R);
      if (a.status && blockIdx.x == 0) atomicOr(a.status, 2);
    }
  } else {
    for (int r = threadIdx.x; r < R; r += blockDim.x) dinv[r] = 1.0 / G[r * R + r];
  }
  __syncthreads();

  // rows: one warp each
  const int64_t rows_per_block = (I + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * rows_per_block;
  const int64_t r1 = (r0 + rows_per_block < I) ? r0 + rows_per_block : I;
  for (int64_t i = r0 + warp; i < r1; i += nwarps) {
    double s[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) s[r] = 0.0;
    if (a.first) {
      const int64_t seg = i / a.SEG, ii = i % a.SEG;
      for (int c = lane; c < a.C; c += 32) {
        const int64_t base = ((seg * a.C + c) * a.SEG + ii) * a.RP;
#pragma unroll
        for (int r = 0; r < RP; ++r)
          if (r < R) s[r] += part_at(a, base + r);
      }
    } else {
      const int nt = a.nseg * a.C * a.nw;
      const int64_t u0 = i * a.nseg * a.C;
      for (int q = lane; q < nt; q += 32) {
        const int64_t base = ((u0 + q / a.nw) * a.nw + q % a.nw) * a.RP;
#pragma unroll
        for (int r = 0; r < RP; ++r)
          if (r < R) s[r] += part_at(a, base + r);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int r = 0; r < RP; ++r)
        if (r < R) s[r] += __shfl_xor_sync(0xffffffffu, s[r], o);
    }
    if (a.M && lane == 0)
      for (int r = 0; r < R; ++r) a.M[i + I * r] = s[r];
    if (a.kind == 0) {
      // A(i, :) = M(i, :) Gamma^+ : lane r forms component r
      if (lane < R) {
        double x = 0.0;
#pragma unroll
        for (int k = 0; k < RP; ++k)
          if (k < R) x = __fma_rn(s[k], W[k * R + lane], x);
        A[i + I * lane] = x;
      }
    } else if (lane == 0) {
      gs_row(s, a, A, i, I, G, dinv);
    }
  }
  __syncthreads();

  // Gram of this block's rows, then the ordered cross-block sum by the last block
  const int npairs = R * (R + 1) / 2;
  for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
    int r = 0, q = p;
    while (q >= R - r) { q -= R - r; ++r; }
    const int c = r + q;
    double acc = 0.0;
    for (int64_t i = r0; i < r1; ++i) acc = __fma_rn(A[i + I * r], A[i + I * c], acc);
    a.gscratch[(size_t)blockIdx.x * npairs + p] = acc;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(a.ticket, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  double* Gout = a.f.gram + (size_t)n * R * R;
  {
    // block partials summed in stripes, then the stripes in order (short float64 chains)
    const int stripes = (int)blockDim.x / npairs > 0 ? (int)blockDim.x / npairs : 1;
    const int t = threadIdx.x;
    if (t < stripes * npairs) {
      const int p = t % npairs, sidx = t / npairs;
      double acc = 0.0;
      for (int b = sidx; b < (int)gridDim.x; b += stripes) acc += a.gscratch[(size_t)b * npairs + p];
      stripe[t] = acc;
    }
    __syncthreads();
    for (int p = t; p < npairs; p += blockDim.x) {
      int r = 0, q = p;
      while (q >= R - r) { q -= R - r; ++r; }
      const int c = r + q;
      double acc = 0.0;
      for (int k = 0; k < stripes; ++k) acc += stripe[k * npairs + p];
      Gout[r * R + c] = acc;
      Gout[c * R + r] = acc;
    }
  }
  if (threadIdx.x == 0) *a.ticket = 0;
  if (!a.normalize) return;
  __syncthreads();
  normalize_all(a, nrm, sc);
}

int launch_finish_update(const MttkrpPlan& p, const MttkrpScratch& w, const FactorSet& f, int mode, int kind,
                         const double* F, int gs_sweeps, double* M, double* gscratch, int* ticket, int* status,
                         cudaStream_t st, bool normalize) {
  FuseArgs a;
  a.f = fargs(f);
  a.n = mode;
  a.kind = kind;
  a.gs_sweeps = gs_sweeps;
  a.F = F;
  a.M = M;
  a.partial = w.partial;
  a.part8 = p.part_elem == 8;
  a.first = p.mode == 0;
  a.nseg = p.nseg;
  a.C = p.C;
  a.nw = p.nw;
  a.RP = p.RP;
  a.SEG = p.SEG;
  a.gscratch = gscratch;
  a.ticket = ticket;
  a.status = status;
  a.normalize = normalize ? 1 : 0;
  const int64_t I = f.dims[mode];
  // few rows per block: GB300's float64 throughput per SM is low, so the per-row reductions and
  // solves are spread over many SMs (two warps per block when Gamma fits 64 threads)
  const int threads = f.R * f.R > 64 ? kMaxThreads : 64;
  const int warps = threads / 32;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((I + warps - 1) / warps, kFuseMaxBlocks));
  if (f.R <= 4) k_finish_update<4><<<nb, threads, 0, st>>>(a);
  else if (f.R <= 8) k_finish_update<8><<<nb, threads, 0, st>>>(a);
  else if (f.R <= 12) k_finish_update<12><<<nb, threads, 0, st>>>(a);
  else k_finish_update<16><<<nb, threads, 0, st>>>(a);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

}  // namespace cpmg
