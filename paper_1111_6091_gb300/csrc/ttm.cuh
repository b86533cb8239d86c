// Restriction Z x_{n in I_c} R-hat^(n) (Eq. ctensor_transformed), one mode product at a time.
#pragma once
#include "common.cuh"

namespace cpmg {

// Y = Z x_n Rh (Rh: Ic x I_n column-major float64), Z, Y of type dtype, column-major.
int ttm_mode(const Shape& s, const void* Z, int dtype, int mode, const double* Rh, int64_t Ic, void* Y,
             int tensor_cores, cudaStream_t st);

// Full restriction over the modes with Rhat[n] != nullptr, in increasing n, using two
// ping-pong buffers of at least max intermediate size bytes each.  Y gets the result.
int ttm_restrict(const Shape& s, const void* Z, int dtype, const double* const* Rhat, const int64_t* Ic,
                 void* Y, void* tmp0, void* tmp1, int tensor_cores, cudaStream_t st);

// Bytes of the largest intermediate of ttm_restrict (for sizing tmp buffers).
size_t ttm_max_intermediate(const Shape& s, int dtype, const double* const* Rhat, const int64_t* Ic);

// tcgen05 path availability for this shape/mode (float tensors, aligned sizes).
bool ttm_tc_supported(const Shape& s, int dtype, int mode, int64_t Ic);
int ttm_mode_tc(const Shape& s, const float* Z, int mode, const double* Rh, int64_t Ic, float* Y,
                cudaStream_t st);

}  // namespace cpmg
