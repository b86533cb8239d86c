// tcgen05 tensor-core n-mode products (placeholder until the UMMA path is enabled).
#include "ttm.cuh"

namespace cpmg {

bool ttm_tc_supported(const Shape&, int, int, int64_t) { return false; }

int ttm_mode_tc(const Shape&, const float*, int, const double*, int64_t, float*, cudaStream_t) {
  return CPMG_UNSUPPORTED;
}

}  // namespace cpmg
