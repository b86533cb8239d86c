// Small float64 kernels of the relaxation sweeps and the multigrid operators.
#pragma once
#include "common.cuh"

namespace cpmg {

// Factor matrices A^(1..N) (float64, column-major I_n x R) plus their Grams
// Upsilon^(n) = A^(n)^T A^(n) (float64 R x R, stored N x R x R contiguously).
struct FactorSet {
  int N = 0, R = 0;
  int64_t dims[kMaxModes] = {0};
  double* A[kMaxModes] = {nullptr};
  double* gram = nullptr;
};

struct FactorPtrArgs {
  double* A[kMaxModes];
  int64_t I[kMaxModes];
  int N, R;
  double* gram;
};

inline FactorPtrArgs fargs(const FactorSet& f) {
  FactorPtrArgs a;
  for (int m = 0; m < kMaxModes; ++m) {
    a.A[m] = m < f.N ? f.A[m] : nullptr;
    a.I[m] = m < f.N ? f.dims[m] : 0;
  }
  a.N = f.N;
  a.R = f.R;
  a.gram = f.gram;
  return a;
}

// Upsilon^(m) for the listed modes (mode_mask bit m set), Eq. Gamma.
int launch_grams(const FactorSet& f, unsigned mode_mask, cudaStream_t st);

// ALS update of Section 3: A^(n) <- M (Gamma^(n))^+ with Gamma^(n) the Hadamard product of
// the other Grams; Cholesky with pivot test, pseudoinverse (Jacobi eigensolver) otherwise.
// Then refreshes Upsilon^(n).  status (device int) gets bit 1 when the pseudoinverse was used.
int launch_als_update(const FactorSet& f, int mode, const double* M, int* status, cudaStream_t st);

// BNGS update of Section 5.2: `sweeps` Gauss-Seidel sweeps on A^(n) Gamma^(n) = M + F
// (F may be null) from the current A^(n); then refreshes Upsilon^(n).
int launch_gs_update(const FactorSet& f, int mode, const double* M, const double* F, int sweeps,
                     cudaStream_t st);

// Eq. ALSnorm on all modes, using the Grams for the column norms; rescales the Grams too.
int launch_normalize(const FactorSet& f, cudaStream_t st);

// Reorder components by decreasing lambda (ties keep index order); permutes Grams too.
int launch_sort(const FactorSet& f, double* scratch_R2, cudaStream_t st);

// H = A^(n) Gamma^(n) - M  (Eq. FASop, = G^(n) of Eq. gradEqn); out may alias nothing.
int launch_fas_op(const FactorSet& f, int mode, const double* M, double* H, cudaStream_t st);

// sum_{i,r} (A^(n) Gamma^(n) - M)^2 into out[slot] (float64; deterministic) and, when
// slot_ag >= 0, sum (A^(n) Gamma^(n))^2 into out[slot_ag].
int launch_grad_sq(const FactorSet& f, int mode, const double* M, double* out, int slot,
                   cudaStream_t st, int slot_ag = -1);

// Squared Frobenius norm of a device matrix into out[slot].
int launch_sq_norm(const double* X, int64_t n, double* out, int slot, cudaStream_t st);

// f = 1/2 ||Z - [[A]]||^2 element by element in float64; also ||Z||^2.  partial: scratch of
// at least 2 * 1024 doubles.  out[0] = sum (z - x)^2, out[1] = sum z^2.
int launch_f_direct(const Shape& s, const void* Z, int dtype, const FactorSet& f, double* partial,
                    double* out, cudaStream_t st);

// C (m x k) = alpha * op(A) B + beta * C, all column-major float64; op(A) = A (m x l) or
// A^T (A is l x m).  Used for factor transfers R-hat A, P-hat A_c and FAS right-hand sides.
int launch_dgemm_small(bool transA, int64_t m, int64_t k, int64_t l, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                       cudaStream_t st);

// Elementwise y = a*x + b*y over n entries.
int launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);

// Least-squares interpolation weights for one mode (Section 4.4, Eqs. LSQinterp and
// interpweights).  U: nblk blocks of I x R column-major vectors (pointers in Uptr), each with
// weight wblk[k] (device).  Output Pw: I x 2 float64 (weights on the left / right coarse
// neighbour of each fine point; coarse rows carry 1 on the left slot).
int launch_interp(int64_t I, int R, int nblk, const double* const* Uptr, const double* wblk,
                  double* Pw, cudaStream_t st);

// R-hat = L^{-1} P^T (Ic x I, column-major, float64) from the interpolation weights, with
// B = P^T P = L L^T (tridiagonal, so L is bidiagonal).  Section 4.1.
int launch_transform(int64_t I, const double* Pw, double* Rhat, double* work, cudaStream_t st);

// LS block weights (Eq. interpweights): w[k] = a2[k] / g2[k], capped at 1e30; a gradient with
// g2 <= tau^2 ag2 (rounding level of the arithmetic that produced it) counts as zero (the cap).
int launch_block_weights(int nblk, const double* a2, const double* g2, const double* ag2, double tau,
                         double* w, cudaStream_t st);

// Copy / convert helpers.
int launch_copy_d(double* dst, const double* src, int64_t n, cudaStream_t st);

}  // namespace cpmg
