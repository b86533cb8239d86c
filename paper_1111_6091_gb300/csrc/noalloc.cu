// cpmg_mttkrp_noalloc: the MTTKRP for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all, or cannot afford it: an application whose
// memory pool (another framework's caching allocator, a preallocated arena) already owns
// the whole GPU, code that must not trigger the device-wide synchronization cudaFree and
// cudaMalloc can cause, or a host that hands this library only its inputs and outputs.
// This entry point serves them: it runs the same MTTKRP kernels as cpmg_mttkrp, but the
// kernels' scratch (the per-CTA partial sums and the Khatri-Rao tables) lives in one
// fixed array that is part of the library image, so the call allocates nothing.
//
// The array is CPMG_NOALLOC_SCRATCH_BYTES (8 MiB).  Every GPU on which this library is
// loaded reserves that much for the life of the process.  All calls share it: two calls
// whose work overlaps on the GPU (different streams, no ordering between them) race on
// it and corrupt each other's results.  Calls ordered on one stream are safe.  Nothing
// in the array needs to start at zero: each call writes every byte it later reads.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "mttkrp.cuh"

namespace {

constexpr size_t kScratchBytes = CPMG_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The shared scratch.  In host code `g_noalloc_scratch` names a host-side stand-in, not the
// device array: only the address returned by cudaGetSymbolAddress may reach a kernel.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per device.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return CPMG_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cpmg::set_last_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
      return CPMG_CUDA_ERROR;
    }
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return CPMG_OK;
}

}  // namespace

extern "C" int cpmg_mttkrp_noalloc(const cpmg_tensor* Z, int R, const double* const* A, int mode,
                                   int precision, double* M, void* cuda_stream) {
  using namespace cpmg;
  if (!Z || !Z->data || !A || !M) return CPMG_INVALID_ARG;
  if (Z->N < 2 || Z->N > CPMG_MAX_MODES || Z->mem != CPMG_MEM_DEVICE) return CPMG_INVALID_ARG;
  if (Z->dtype != CPMG_F32 && Z->dtype != CPMG_F64) return CPMG_INVALID_ARG;
  if (R < 1 || R > CPMG_MAX_RANK || mode < 0 || mode >= Z->N) return CPMG_INVALID_ARG;
  Shape s;
  s.N = Z->N;
  for (int n = 0; n < Z->N; ++n) {
    if (Z->dims[n] < 1 || !A[n]) return CPMG_INVALID_ARG;
    s.dims[n] = Z->dims[n];
  }
  int prec;
  switch (precision) {
    case CPMG_PREC_FP32: prec = P_FP32; break;
    case CPMG_PREC_FP64: prec = P_FP64; break;
    case CPMG_PREC_DF: prec = P_DF; break;
    default: return CPMG_INVALID_ARG;
  }
  int device = 0;
  CPMG_CUDA_TRY(cudaGetDevice(&device));
  int sms = 0;
  CPMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  void* base = nullptr;
  CPMG_TRY(scratch_address(device, &base));

  MttkrpPlan p;
  // The bulk-copy kernel needs a full Khatri-Rao row table; when that does not fit, the
  // register-load kernel (two small tables) serves instead.
  for (int attempt = 0; attempt < 2; ++attempt) {
    CPMG_TRY(mttkrp_plan(s, mode, R, prec, Z->dtype, Z->data, sms, &p, attempt == 0));
    // Fewer, larger work units until the partial sums and the tables fit the fixed scratch.
    while (p.partial_bytes() + p.tables_bytes() > kScratchBytes && p.C > 1) {
      p.C = (p.C + 1) / 2;
      p.nunits = p.In * p.nseg * p.C;
      // one unit per CTA, except the persistent kernel that spreads unit ranges over its CTAs
      p.grid = (p.use_tma && p.mode != 0) ? std::min<int64_t>(p.grid, p.nunits) : p.nunits;
    }
    if (p.partial_bytes() + p.tables_bytes() + 256 <= kScratchBytes) break;
  }
  const size_t tables = p.tables_bytes();
  if (p.partial_bytes() + tables > kScratchBytes) return CPMG_OUT_OF_BUDGET;
  MttkrpScratch w;
  w.tables = base;
  w.partial = static_cast<unsigned char*>(base) + (tables + 255) / 256 * 256;
  if ((tables + 255) / 256 * 256 + p.partial_bytes() > kScratchBytes) return CPMG_OUT_OF_BUDGET;
  return mttkrp_run(p, s, Z->data, A, w, M, reinterpret_cast<cudaStream_t>(cuda_stream));
}
