// One kernel for what follows an MTTKRP inside a relaxation sweep: the ordered reduction of
// the MTTKRP partial sums into M = Z_(n) Phi^(n), the R x R solve of the ALS update
// (A^(n) <- M Gamma^+, Section 3) or the Gauss-Seidel sweeps of BNGS (A^(n) Gamma = M + F,
// Section 5.2), and the refresh of Upsilon^(n) = A^(n)^T A^(n) (Eq. Gamma).
//
// Every block factorizes Gamma^(n) (the Hadamard product of the other Grams) in shared memory,
// then each warp handles rows of A^(n): lanes sum the partials of the row in a fixed order, a
// shuffle tree combines them, lane 0 solves the row.  Each block then forms the Gram of its own
// rows; the last block to finish (atomic ticket) sums the block Grams in block order.  The
// summation orders depend only on the shapes, so results are bitwise reproducible.
#include "fused.cuh"
#include "linalg.cuh"

#include <algorithm>

namespace cpmg {

constexpr int kR = kMaxRank;
constexpr int kWarps = 8;

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
};

__device__ __forceinline__ double part_at(const FuseArgs& a, int64_t idx) {
  return a.part8 ? reinterpret_cast<const double*>(a.partial)[idx]
                 : (double)reinterpret_cast<const float*>(a.partial)[idx];
}

__global__ void __launch_bounds__(kWarps * 32) k_finish_update(FuseArgs a) {
  __shared__ double G[kR * kR], L[kR * kR], Pi[kR * kR], V[kR * kR], w[kR];
  __shared__ int chol_ok;
  __shared__ bool last;
  const int R = a.f.R;
  const int n = a.n;
  const int64_t I = a.f.I[n];
  double* A = a.f.A[n];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // Gamma^(n) and its factorization (same arithmetic as the separate ALS / GS kernels)
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < a.f.N; ++m)
      if (m != n) v *= a.f.gram[(size_t)m * R * R + e];
    G[e] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0 && a.kind == 0) {
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
      if (a.status && blockIdx.x == 0) atomicOr(a.status, 2);
    }
  }
  __syncthreads();

  // rows: one warp each
  const int64_t rows_per_block = (I + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * rows_per_block;
  const int64_t r1 = (r0 + rows_per_block < I) ? r0 + rows_per_block : I;
  for (int64_t i = r0 + warp; i < r1; i += kWarps) {
    double s[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) s[r] = 0.0;
    if (a.first) {
      const int64_t seg = i / a.SEG, ii = i % a.SEG;
      for (int c = lane; c < a.C; c += 32) {
        const int64_t base = ((seg * a.C + c) * a.SEG + ii) * a.RP;
#pragma unroll
        for (int r = 0; r < kR; ++r)
          if (r < R) s[r] += part_at(a, base + r);
      }
    } else {
      const int64_t nterm = (int64_t)a.nseg * a.C * a.nw;
      for (int64_t q = lane; q < nterm; q += 32) {
        const int64_t u = i * a.nseg * a.C + q / a.nw;
        const int64_t base = (u * a.nw + q % a.nw) * a.RP;
#pragma unroll
        for (int r = 0; r < kR; ++r)
          if (r < R) s[r] += part_at(a, base + r);
      }
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      if (r < R) {
        double v = s[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        s[r] = v;
      }
    }
    if (lane == 0) {
      if (a.M)
        for (int r = 0; r < R; ++r) a.M[i + I * r] = s[r];
      double x[kR];
      if (a.kind == 0) {
        if (chol_ok) {
          for (int r = 0; r < R; ++r) x[r] = s[r];
          for (int r = 0; r < R; ++r) {
            double t = x[r];
            for (int k = 0; k < r; ++k) t -= L[r * R + k] * x[k];
            x[r] = t / L[r * R + r];
          }
          for (int r = R - 1; r >= 0; --r) {
            double t = x[r];
            for (int k = r + 1; k < R; ++k) t -= L[k * R + r] * x[k];
            x[r] = t / L[r * R + r];
          }
        } else {
          for (int r = 0; r < R; ++r) {
            double t = 0.0;
            for (int k = 0; k < R; ++k) t += s[k] * Pi[k * R + r];
            x[r] = t;
          }
        }
      } else {
        double b[kR];
        for (int r = 0; r < R; ++r) {
          x[r] = A[i + I * r];
          b[r] = s[r] + (a.F ? a.F[i + I * r] : 0.0);
        }
        for (int it = 0; it < a.gs_sweeps; ++it)
          for (int r = 0; r < R; ++r) {
            double t = b[r];
            for (int k = 0; k < R; ++k)
              if (k != r) t -= G[r * R + k] * x[k];
            x[r] = t / G[r * R + r];
          }
      }
      for (int r = 0; r < R; ++r) A[i + I * r] = x[r];
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
  for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
    int r = 0, q = p;
    while (q >= R - r) { q -= R - r; ++r; }
    const int c = r + q;
    double acc = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) acc += a.gscratch[(size_t)b * npairs + p];
    Gout[r * R + c] = acc;
    Gout[c * R + r] = acc;
  }
  if (threadIdx.x == 0) *a.ticket = 0;
}

int launch_finish_update(const MttkrpPlan& p, const MttkrpScratch& w, const FactorSet& f, int mode, int kind,
                         const double* F, int gs_sweeps, double* M, double* gscratch, int* ticket, int* status,
                         cudaStream_t st) {
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
  const int64_t I = f.dims[mode];
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((I + kWarps - 1) / kWarps, kFuseMaxBlocks));
  k_finish_update<<<nb, kWarps * 32, 0, st>>>(a);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}

}  // namespace cpmg
