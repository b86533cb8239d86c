// Restriction Z x_{n in I_c} R-hat^(n) (Eq. ctensor_transformed), one mode product at a time.
#pragma once
#include "common.cuh"

namespace cpmg {

// Y = Z x_n Rh (Rh: Ic x I_n column-major float64), Z, Y of type dtype, column-major.
// tensor_cores: 0 = CUDA cores; 1 = tcgen05 split-BF16 where ttm_tc_supported, else CUDA cores;
// 2 = tcgen05 or CPMG_UNSUPPORTED.  tc_scratch holds ttm_tc_scratch_bytes(I_n) bytes; err
// receives 1 if a bounded device-side wait of the tensor-core kernel expired.
// ev0 / ev1 (may be null) bracket the tensor-core kernel; ev_external: recorded inside a graph
// capture.
int ttm_mode(const Shape& s, const void* Z, int dtype, int mode, const double* Rh, int64_t Ic, void* Y,
             int tensor_cores, void* tc_scratch, int* err, cudaEvent_t ev0, cudaEvent_t ev1, bool ev_external,
             cudaStream_t st);

// Full restriction over the modes with Rhat[n] != nullptr, in increasing n, using two
// ping-pong buffers of at least max intermediate size bytes each.  Y gets the result.
// ev: null or 2 events per mode (entries may be null) passed to ttm_mode.
int ttm_restrict(const Shape& s, const void* Z, int dtype, const double* const* Rhat, const int64_t* Ic,
                 void* Y, void* tmp0, void* tmp1, int tensor_cores, void* tc_scratch, int* err,
                 const cudaEvent_t* ev, bool ev_external, cudaStream_t st);

// The order in which ttm_restrict applies the mode products (writes the modes to order[], returns
// their count). Increasing n, except on the tensor-core float path when mode 1 is restricted and
// no mode grows. There it is mode 1, then the last mode down to mode 2: a middle mode with few
// rows in front of it pads its 128-row tensor-core tiles, and it then works on the smallest
// tensor. The first intermediate, which is the largest, is the same in both orders.
int ttm_order(const Shape& s, int dtype, const double* const* Rhat, const int64_t* Ic, int tensor_cores, int* order);

// Bytes of the largest intermediate of ttm_restrict (for sizing tmp buffers).
size_t ttm_max_intermediate(const Shape& s, int dtype, const double* const* Rhat, const int64_t* Ic);

// tcgen05 path availability for this shape and mode (float tensors, Ic <= 256).
bool ttm_tc_supported(const Shape& s, int dtype, int mode, int64_t Ic);
// Bytes of the split R-hat operand for a mode of size up to max_In (any Ic <= 256).
size_t ttm_tc_scratch_bytes(int64_t max_In);
int ttm_mode_tc(const Shape& s, const float* Z, int mode, const double* Rh, int64_t Ic, float* Y, void* scratch,
                int* err, cudaEvent_t ev0, cudaEvent_t ev1, bool ev_external, cudaStream_t st);

}  // namespace cpmg
