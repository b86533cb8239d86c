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
// it and corrupt each other's results.  Calls ordered on one stream are safe.
//
// Layout of the array: bytes [0, 256) hold the status word the bulk-copy kernel raises
// when one of its bounded waits expires (cleared at the start of every call); the
// Khatri-Rao tables follow, then the partial sums.  The tables and partial sums need no
// clearing: each call writes every byte of them it later reads.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "mttkrp.cuh"

namespace {

constexpr size_t kScratchBytes = CPMG_NOALLOC_SCRATCH_BYTES;
constexpr size_t kStatusBytes = 256;
constexpr int kMaxDevices = 64;

// The shared scratch.  In host code `g_noalloc_scratch` names a host-side stand-in, not the
// device array: only the address returned by cudaGetSymbolAddress may reach a kernel.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// When a bounded wait of the MTTKRP expired (status word non-zero), the partial sums are
// incomplete: overwrite M with NaN so that the caller cannot take it for a result.
__global__ void k_noalloc_poison(const int* status, double* M, int64_t n) {
  if (*reinterpret_cast<const volatile int*>(status) == 0) return;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    M[i] = nan;
}

std::mutex g_mu;
struct Slot {
  CUcontext ctx = nullptr;
  void* addr = nullptr;
};
Slot g_slot[kMaxDevices];

PFN_cuCtxGetCurrent_v4000 ctx_fn() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    cudaGetLastError();
  });
  return fn;
}

// Device address of the scratch in the current device's current context.  It is looked up
// once per (device, context): a new primary context (after cudaDeviceReset, say) holds a
// new copy of the array, and the lookup is repeated for it.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return CPMG_INVALID_ARG;
  // On a first call the context may not exist yet: cudaGetSymbolAddress creates it, and
  // the context is read again after it.
  CUcontext ctx = nullptr;
  PFN_cuCtxGetCurrent_v4000 get = ctx_fn();
  std::lock_guard<std::mutex> lock(g_mu);
  if (get && get(&ctx) == CUDA_SUCCESS && ctx && g_slot[device].addr && g_slot[device].ctx == ctx) {
    *out = g_slot[device].addr;
    return CPMG_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cpmg::set_last_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    return CPMG_CUDA_ERROR;
  }
  ctx = nullptr;
  if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  g_slot[device].ctx = ctx;   // a null context is never matched: the lookup then runs per call
  g_slot[device].addr = p;
  *out = p;
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
  const size_t avail = kScratchBytes - kStatusBytes;

  MttkrpPlan p;
  // The bulk-copy kernel needs a full Khatri-Rao row table; when that does not fit, the
  // register-load kernel (two small tables) serves instead.
  for (int attempt = 0; attempt < 2; ++attempt) {
    CPMG_TRY(mttkrp_plan(s, mode, R, prec, Z->dtype, Z->data, sms, &p, attempt == 0));
    // Fewer, larger work units until the partial sums and the tables fit the fixed scratch.
    while (p.partial_bytes() + p.tables_bytes() > avail && p.C > 1) {
      p.C = (p.C + 1) / 2;
      p.nunits = p.In * p.nseg * p.C;
      // one unit per CTA, except the persistent kernel that spreads unit ranges over its CTAs
      p.grid = (p.use_tma && p.mode != 0) ? std::min<int64_t>(p.grid, p.nunits) : p.nunits;
    }
    if (p.partial_bytes() + p.tables_bytes() + 256 <= avail) break;
  }
  const size_t tables = (p.tables_bytes() + 255) / 256 * 256;
  if (tables + p.partial_bytes() > avail) return CPMG_OUT_OF_BUDGET;
  unsigned char* b = static_cast<unsigned char*>(base);
  int* status = reinterpret_cast<int*>(b);
  MttkrpScratch w;
  w.tables = b + kStatusBytes;
  w.partial = b + kStatusBytes + tables;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  CPMG_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  CPMG_TRY(mttkrp_run(p, s, Z->data, A, w, M, st, nullptr, nullptr, status));
  const int64_t n = s.dims[mode] * (int64_t)R;
  k_noalloc_poison<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(status, M, n);
  CPMG_CUDA_TRY(cudaGetLastError());
  return CPMG_OK;
}
