// Small dense linear algebra shared by several kernels (device code, one thread).
#pragma once
#include "common.cuh"

namespace cpmg {

// Symmetric Jacobi eigensolver (cyclic, one thread), for the pseudoinverse fallback.
// On exit G is overwritten, w holds eigenvalues, V (row-major, columns = vectors).
__device__ inline void jacobi_eig_dev(double* G, double* V, double* w, int R) {
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < R; ++j) V[i * R + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < R; ++i)
      for (int j = 0; j < R; ++j) {
        const double x = G[i * R + j] * G[i * R + j];
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < R - 1; ++p)
      for (int q = p + 1; q < R; ++q) {
        const double apq = G[p * R + q];
        if (apq == 0.0) continue;
        const double app = G[p * R + p], aqq = G[q * R + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < R; ++k) {  // columns p, q
          const double gkp = G[k * R + p], gkq = G[k * R + q];
          G[k * R + p] = c * gkp - s * gkq;
          G[k * R + q] = s * gkp + c * gkq;
        }
        for (int k = 0; k < R; ++k) {  // rows p, q
          const double gpk = G[p * R + k], gqk = G[q * R + k];
          G[p * R + k] = c * gpk - s * gqk;
          G[q * R + k] = s * gpk + c * gqk;
        }
        for (int k = 0; k < R; ++k) {
          const double vkp = V[k * R + p], vkq = V[k * R + q];
          V[k * R + p] = c * vkp - s * vkq;
          V[k * R + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < R; ++i) w[i] = G[i * R + i];
}

// In-place Gauss-Jordan inversion of the SPD matrix G (R x R, row-major) by R*R threads in
// parallel, without pivoting: step k divides by the k-th pivot, which is the Schur-complement
// diagonal that a Cholesky factorization tests (same threshold).  Returns false (in every
// thread) if a pivot is not above thresh.  On GB300 a dependent float64 division costs
// hundreds of cycles, so the R divisions sit on the critical path once, not once per row.
__device__ inline bool gj_inverse(double* G, int R, double thresh, int* fail) {
  const int t = threadIdx.x;
  const int i = t / R, j = t % R;
  const bool mine = t < R * R;
  if (t == 0) *fail = 0;
  __syncthreads();
  for (int k = 0; k < R; ++k) {
    const double p = G[k * R + k];
    double v = 0.0;
    if (mine) {
      const double aij = G[i * R + j], aik = G[i * R + k], akj = G[k * R + j];
      const double rp = 1.0 / p;
      if (i == k && j == k) v = rp;
      else if (i == k) v = akj * rp;
      else if (j == k) v = -aik * rp;
      else v = aij - aik * akj * rp;
    }
    if (t == 0 && !(p > thresh)) *fail = 1;
    __syncthreads();
    if (mine) G[i * R + j] = v;
    __syncthreads();
  }
  return *fail == 0;
}

// x^(1/N) for x >= 0 in float64 by Newton's method on y^N = x, started from the float
// estimate: each step roughly doubles the correct digits, so two steps reach float64 accuracy.
// (On GB300 this is far shorter than a float64 pow: the dependent float64 chain is ~10 ops.)
__device__ inline double nth_root(double x, int N) {
  if (!(x > 0.0)) return 0.0;
  if (N == 1) return x;
  if (x > 1e300 || x < 1e-300 || !isfinite(x)) return pow(x, 1.0 / N);
  const float xf = (float)x;
  double y = (xf > 0.f && isfinite(xf)) ? (double)powf(xf, 1.0f / (float)N) : pow(x, 1.0 / N);
  for (int it = 0; it < 2; ++it) {
    double yn1 = 1.0;  // y^(N-1)
    for (int k = 1; k < N; ++k) yn1 *= y;
    // y <- y - (y^N - x) / (N y^(N-1))
    y = y - (yn1 * y - x) / (N * yn1);
  }
  return y;
}

}  // namespace cpmg
