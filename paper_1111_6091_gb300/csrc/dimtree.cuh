// Dimension-tree reuse of a partial MTTKRP for third-order tensors.
//
// For N = 3 the products Z_(1) Phi^(1) and Z_(2) Phi^(2) (Eq. fineeq1, Eq. Phi) both contract
// mode 3 with A^(3).  W = Z x_3 A^(3)^T, an I_1 x I_2 x R array with
//   W(i, j, r) = sum_k z_{ijk} a^(3)_{kr},
// is formed once (one pass over Z: the mode-1 MTTKRP of the (I_1 I_2) x I_3 matricization), and
//   M^(1)(i, r) = sum_j W(i, j, r) a^(2)_{jr},    M^(2)(j, r) = sum_i W(i, j, r) a^(1)_{ir}
// follow from W alone.  An ALS or BNGS sweep updates A^(1) and A^(2) while A^(3) is unchanged, so
// both updates read the same W; only M^(3) needs a second pass over Z.  The same holds for all
// three products at one fixed point (the gradient of Eq. gradConv, the FAS right-hand sides of
// Eq. FASrhs, the LS weights of Eq. interpweights).
#pragma once
#include "common.cuh"

namespace cpmg {

// out(i, r) at out[i * ld_row + r * ld_col] = sum_j W(i, j, r) V(j, r)   (V: I2 x R col-major)
// when `mode` = 0; out(j, r) = sum_i W(i, j, r) V(i, r) (V: I1 x R) when `mode` = 1.
// W: I1 x I2 x R column-major float64.  Summation orders depend only on the sizes.
int launch_dt_contract(const double* W, int64_t I1, int64_t I2, int R, const double* V, int mode, double* out,
                       int64_t ld_row, int64_t ld_col, cudaStream_t st);
// The same with a float W (the tensor-core products of the split-BF16 path write float).
int launch_dt_contract_f(const float* W, int64_t I1, int64_t I2, int R, const double* V, int mode, double* out,
                         int64_t ld_row, int64_t ld_col, cudaStream_t st);

// Mode 3 from V = Z x_1 A^(1)^T, an R x I2 x I3 float array with r fastest (the tensor-core mode-1
// product's layout): out(k, r) at out[k * ld_row + r * ld_col] = sum_j V(r, j, k) U(j, r), U the
// I2 x R float64 factor A^(2).  Summation over j in increasing order.
int launch_dt_vmode(const float* V, int64_t I2, int64_t I3, int R, const double* U, double* out, int64_t ld_row,
                    int64_t ld_col, cudaStream_t st);

// dst (R x I column-major) = src^T for an I x R column-major float64 factor.
int launch_transpose_d(const double* src, int64_t I, int R, double* dst, cudaStream_t st);

// W(p, r) = sum_k X(p, k) C(k, r) for the P x K column-major matricization X of a tensor (float or
// float64 elements, `zdtype`) and a float64 K x R factor C, written as float64 P x R column-major.
// prec: P_FP32 (float products and sums), P_DF (float-pair sums, float64-accurate), P_FP64.  One
// pass over X with no partial sums: every thread owns whole rows and walks all K columns, with C
// staged in shared memory.  FP32 on float X, when the rows split into blocks of 256 or more per SM,
// streams each block's columns through a ring of bulk copies instead (same arithmetic, same bits);
// *err (may be null) receives 1 if one of its bounded waits expired.  Returns CPMG_INVALID_ARG for R
// outside 1..16.
int launch_dt_w(const void* X, int zdtype, int64_t P, int64_t K, int R, const double* C, int prec, double* W,
                int num_sms, cudaStream_t st, int* err = nullptr);

}  // namespace cpmg
