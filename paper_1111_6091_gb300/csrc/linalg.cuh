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

}  // namespace cpmg
