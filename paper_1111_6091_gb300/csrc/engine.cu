// Host engine of libcpmg: context and device memory, MTTKRP plans, the relaxations
// (ALS of Section 3, BNGS of Section 5.2), the multigrid hierarchy, CP-AMG-mult
// (Algorithm 1), CP-FAS (Algorithm 2), FMG-CP-FAS (Algorithm 3), the setup/solve control of
// Section 6.1 and the C ABI declared in include/cpmg.h.  All arithmetic runs in the kernels;
// the host only orders launches and reads back scalars (g, f) for the control decisions.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.cuh"
#include "dense.cuh"
#include "dimtree.cuh"
#include "fused.cuh"
#include "mttkrp.cuh"
#include "ttm.cuh"

using namespace cpmg;

// ============================================================================ context
struct ProfEvents {
  cudaEvent_t a, b;
  double bytes;
  int kind;     // 0: FP32, 1: pairs of floats, 2: FP64 finest-level MTTKRP main kernel;
                // 3: tensor-core mode product of the restriction
  bool owned;   // recorded inside a CUDA graph: the graph keeps the events
};

struct cpmg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  size_t in_use = 0;
  int num_sms = 148;
  std::map<void*, size_t> sizes;
  // MTTKRP scratch
  void* mt_partial = nullptr;
  size_t mt_partial_cap = 0;
  void* mt_tables = nullptr;
  size_t mt_tables_cap = 0;
  std::map<std::string, MttkrpPlan> plans;
  // scalars
  double* dsc = nullptr;   // device scalars (4096)
  double* gscratch = nullptr;  // block Grams of the fused finish/update kernel
  double* hsc = nullptr;   // pinned host mirror
  int* dstatus = nullptr;
  // profiling of the finest-level MTTKRP main kernel
  bool profile = false;
  std::vector<ProfEvents> pending;
  std::vector<ProfEvents> pool;
  double prof_ms[6] = {0, 0, 0, 0, 0, 0};
  int64_t prof_launches[6] = {0, 0, 0, 0, 0, 0};
  double prof_bytes[6] = {0, 0, 0, 0, 0, 0};
  int64_t launches = 0;
  const void* prof_Z = nullptr;  // tensor whose MTTKRPs are profiled (the finest level)
  bool capturing = false;        // a CUDA graph capture is open on `stream`
  cpmg::BatchState* batch = nullptr;  // batched solver / request server (batch.cu)
};

namespace cpmg {
static thread_local char g_errbuf[512] = {0};
void set_last_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_errbuf, sizeof(g_errbuf), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}
}  // namespace cpmg

static int dalloc(cpmg_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return CPMG_OK;
  bytes = (bytes + 255) / 256 * 256;
  if (c->budget && c->in_use + bytes > c->budget) return CPMG_OUT_OF_BUDGET;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? CPMG_OUT_OF_BUDGET : CPMG_CUDA_ERROR;
  }
  c->sizes[*p] = bytes;
  c->in_use += bytes;
  return CPMG_OK;
}

static void dfree(cpmg_ctx* c, void* p) {
  if (!p) return;
  auto it = c->sizes.find(p);
  if (it != c->sizes.end()) {
    c->in_use -= it->second;
    c->sizes.erase(it);
  }
  cudaFree(p);
}

namespace cpmg {
int ctx_alloc(cpmg_ctx* c, void** p, size_t bytes) { return dalloc(c, p, bytes); }
void ctx_free(cpmg_ctx* c, void* p) { dfree(c, p); }
cudaStream_t ctx_stream(const cpmg_ctx* c) { return c->stream; }
int ctx_device(const cpmg_ctx* c) { return c->device; }
int ctx_sms(const cpmg_ctx* c) { return c->num_sms; }
size_t ctx_budget(const cpmg_ctx* c) { return c->budget; }
size_t ctx_in_use(const cpmg_ctx* c) { return c->in_use; }
void ctx_add_launches(cpmg_ctx* c, int64_t n) { c->launches += n; }
BatchState*& ctx_batch_state(cpmg_ctx* c) { return c->batch; }
}  // namespace cpmg

template <typename T>
static int dalloc_t(cpmg_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  int s = dalloc(c, &v, count * sizeof(T));
  *p = reinterpret_cast<T*>(v);
  return s;
}

// ============================================================================ factor sets
static size_t fs_doubles(int N, int R, const int64_t* dims) {
  size_t t = 0;
  for (int m = 0; m < N; ++m) t += (size_t)dims[m] * R;
  return t + (size_t)N * R * R + (size_t)N * R;
}

static int fs_alloc(cpmg_ctx* c, FactorSet* f, int N, int R, const int64_t* dims) {
  double* base = nullptr;
  CPMG_TRY(dalloc_t(c, &base, fs_doubles(N, R, dims)));
  f->N = N;
  f->R = R;
  size_t off = 0;
  for (int m = 0; m < kMaxModes; ++m) {
    f->dims[m] = m < N ? dims[m] : 0;
    f->A[m] = m < N ? base + off : nullptr;
    if (m < N) off += (size_t)dims[m] * R;
  }
  f->gram = base + off;
  return CPMG_OK;
}

static void fs_free(cpmg_ctx* c, FactorSet* f) {
  if (f->N > 0 && f->A[0]) dfree(c, f->A[0]);
  *f = FactorSet();
}

static int fs_copy(FactorSet& dst, const FactorSet& src, cudaStream_t st) {
  CPMG_CUDA_TRY(cudaMemcpyAsync(dst.A[0], src.A[0], fs_doubles(src.N, src.R, src.dims) * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
  return CPMG_OK;
}

static unsigned all_modes(int N) { return (1u << N) - 1u; }

// ============================================================================ MTTKRP
static std::string plan_key(const Shape& s, int mode, int R, int prec, int dtype, const void* Z) {
  char buf[256];
  int n = snprintf(buf, sizeof(buf), "%d|%d|%d|%d|%d|%d|", s.N, mode, R, prec, dtype,
                   (int)(reinterpret_cast<uintptr_t>(Z) % 16));
  std::string k(buf, n);
  for (int m = 0; m < s.N; ++m) k += std::to_string(s.dims[m]) + ",";
  return k;
}

static int get_plan(cpmg_ctx* c, const Shape& s, int mode, int R, int prec, int dtype, const void* Z,
                    const MttkrpPlan** out) {
  const std::string key = plan_key(s, mode, R, prec, dtype, Z);
  auto it = c->plans.find(key);
  if (it == c->plans.end()) {
    MttkrpPlan p;
    CPMG_TRY(mttkrp_plan(s, mode, R, prec, dtype, Z, c->num_sms, &p));
    it = c->plans.emplace(key, p).first;
  }
  *out = &it->second;
  return CPMG_OK;
}

static int ensure_scratch(cpmg_ctx* c, size_t partial, size_t tables) {
  if (partial > c->mt_partial_cap) {
    dfree(c, c->mt_partial);
    c->mt_partial = nullptr;
    c->mt_partial_cap = 0;
    const size_t want = std::max(partial, (size_t)1 << 20);
    CPMG_TRY(dalloc(c, &c->mt_partial, want));
    c->mt_partial_cap = want;
  }
  if (tables > c->mt_tables_cap) {
    dfree(c, c->mt_tables);
    c->mt_tables = nullptr;
    c->mt_tables_cap = 0;
    const size_t want = std::max(tables, (size_t)1 << 20);
    CPMG_TRY(dalloc(c, &c->mt_tables, want));
    c->mt_tables_cap = want;
  }
  return CPMG_OK;
}

static double algorithmic_bytes(const Shape& s, int mode, int R, int dtype) {
  const double esz = dtype == CPMG_F64 ? 8.0 : 4.0;
  double b = esz * (double)s.numel();
  for (int m = 0; m < s.N; ++m)
    if (m != mode) b += 4.0 * R * (double)s.dims[m];
  b += 4.0 * R * (double)s.dims[mode];
  return b;
}

static int profile_collect(cpmg_ctx* c) {
  if (c->pending.empty() || c->capturing) return CPMG_OK;
  CPMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof_ms[p.kind] += ms;
      c->prof_launches[p.kind] += 1;
      c->prof_bytes[p.kind] += p.bytes;
    }
    if (!p.owned) c->pool.push_back(p);
  }
  c->pending.clear();
  cudaGetLastError();
  return CPMG_OK;
}

// ============================================================================ CUDA graphs
// A relaxation sweep, a setup cycle or a CP-FAS V-cycle is a fixed sequence of launches (no
// host decisions inside), so it is captured once and replayed as one graph launch.  Graphs are
// owned by the object whose buffers they reference (a hierarchy, or one cp_als_sweep call) and
// are destroyed with it; a graph also records the finest-level tensor pointer it was captured
// with and is re-captured if that changes.
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  const void* z0 = nullptr;
  int64_t dlaunch = 0;
  int drefine = 0;
  std::vector<ProfEvents> events;
};

struct GraphCache {
  std::map<std::string, GraphEntry> m;
  void clear() {
    for (auto& kv : m) {
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      for (auto& e : kv.second.events) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
      }
    }
    m.clear();
  }
};

// A pair of timing events for one profiled launch (from the pool, or new and owned by the graph
// being captured), queued for profile_collect.
static int prof_events(cpmg_ctx* c, int kind, double bytes, cudaEvent_t* e0, cudaEvent_t* e1) {
  ProfEvents pe;
  if (!c->pool.empty() && !c->capturing) {
    pe = c->pool.back();
    c->pool.pop_back();
  } else {
    CPMG_CUDA_TRY(cudaEventCreate(&pe.a));
    CPMG_CUDA_TRY(cudaEventCreate(&pe.b));
  }
  pe.bytes = bytes;
  pe.owned = c->capturing;
  pe.kind = kind;
  c->pending.push_back(pe);
  *e0 = pe.a;
  *e1 = pe.b;
  return CPMG_OK;
}

namespace cpmg {
int ctx_profile_events(cpmg_ctx* c, int kind, double bytes, cudaEvent_t* e0, cudaEvent_t* e1) {
  *e0 = *e1 = nullptr;
  if (!c->profile) return CPMG_OK;
  if (c->pending.size() > 512) CPMG_TRY(profile_collect(c));  // recycle read-out event pairs
  return prof_events(c, kind, bytes, e0, e1);
}
}  // namespace cpmg

// Events for the tensor-core mode products of one restriction (2 per coarsened mode that runs
// on tcgen05), with the algorithmic bytes of each (float in + float out).
static int prof_ttm(cpmg_ctx* c, const Shape& s, int dtype, const double* const* Rh, const int64_t* Ic,
                    int tensor_cores, cudaEvent_t* ev) {
  for (int k = 0; k < 2 * kMaxModes; ++k) ev[k] = nullptr;
  if (!c->profile || !tensor_cores || dtype != CPMG_F32) return CPMG_OK;
  Shape cur = s;
  int order[kMaxModes];
  const int k = ttm_order(s, dtype, Rh, Ic, tensor_cores, order);
  for (int j = 0; j < k; ++j) {
    const int n = order[j];
    const double in = 4.0 * (double)cur.numel();
    const bool tc = ttm_tc_supported(cur, dtype, n, Ic[n]);
    cur.dims[n] = Ic[n];
    if (tc) CPMG_TRY(prof_events(c, 3, in + 4.0 * (double)cur.numel(), &ev[2 * n], &ev[2 * n + 1]));
  }
  return CPMG_OK;
}

// kind < 0: M = MTTKRP (reduced by the finish kernel).  kind 0 / 1: the MTTKRP followed by the
// fused reduction + ALS solve / Gauss-Seidel (with right-hand side F) + Gram refresh of mode n.
static int run_mttkrp_k(cpmg_ctx* c, const Shape& s, const void* Z, int dtype, const FactorSet& f, int mode,
                        int prec, double* M, int kind, const double* F, int gs_sweeps, bool normalize = false);

static int run_mttkrp(cpmg_ctx* c, const Shape& s, const void* Z, int dtype, const FactorSet& f, int mode,
                      int prec, double* M) {
  return run_mttkrp_k(c, s, Z, dtype, f, mode, prec, M, -1, nullptr, 0);
}

static int run_mttkrp_k(cpmg_ctx* c, const Shape& s, const void* Z, int dtype, const FactorSet& f, int mode,
                        int prec, double* M, int kind, const double* F, int gs_sweeps, bool normalize) {
  const MttkrpPlan* p = nullptr;
  CPMG_TRY(get_plan(c, s, mode, f.R, prec, dtype, Z, &p));
  CPMG_TRY(ensure_scratch(c, p->partial_bytes(), p->tables_bytes()));
  MttkrpScratch w;
  w.partial = c->mt_partial;
  w.tables = c->mt_tables;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile && Z == c->prof_Z)
    CPMG_TRY(prof_events(c, p->prec == P_FP32 ? 0 : (p->prec == P_DF ? 1 : 2), algorithmic_bytes(s, mode, f.R, dtype),
                         &e0, &e1));
  const double* Aptrs[kMaxModes];
  for (int m = 0; m < kMaxModes; ++m) Aptrs[m] = f.A[m];
  CPMG_TRY(mttkrp_run(*p, s, Z, Aptrs, w, M, c->stream, e0, e1, c->dstatus + 1, kind < 0, c->capturing));
  c->launches += (p->use_tma || p->has_in || p->has_out) ? 3 : 2;
  if (kind >= 0)
    CPMG_TRY(launch_finish_update(*p, w, f, mode, kind, F, gs_sweeps, nullptr, c->gscratch, c->dstatus + 2,
                                  c->dstatus, c->stream, normalize));
  if (c->pending.size() > 512) CPMG_TRY(profile_collect(c));
  return CPMG_OK;
}

// ============================================================================ levels
struct Level {
  Shape s;
  const void* Z = nullptr;
  int dtype = CPMG_F32;
  void* Zown = nullptr;
  bool co[kMaxModes] = {false};
  int64_t cd[kMaxModes] = {0};
  double* Rhat[kMaxModes] = {nullptr};
  double* Pw[kMaxModes] = {nullptr};
  FactorSet A, At, tf[CPMG_MAX_TEST_BLOCKS];
  double* F[kMaxModes] = {nullptr};
  double* H[kMaxModes] = {nullptr};
  double* buf = nullptr;   // backing store of F, H
  double* M = nullptr;     // I_max x R work
  double* W = nullptr;     // I_1 x I_2 x R partial MTTKRP of the dimension tree (third order)
  // split-BF16 tensor-core passes (float third-order levels of the dimension tree)
  float* Wf = nullptr;     // Z x_3 A^(3)^T, I_1 I_2 x R
  float* Vf = nullptr;     // Z x_1 A^(1)^T, R x I_2 x I_3
  double* AT = nullptr;    // a factor transposed (R x I_max), the tensor-core B operand
  void* tcs = nullptr;     // split-BF16 copy of AT
  double* twork = nullptr; // transform work (2 * Ic_max)
  double* blk = nullptr;   // block norms / weights (3 * (nt+1))
  bool coarsest() const {
    for (int n = 0; n < s.N; ++n)
      if (co[n]) return false;
    return true;
  }
};

// Third-order levels keep the dimension tree's W when it is small next to a pass over Z.
static bool dt_worth(const Shape& s, int R) { return s.N == 3 && s.dims[2] > 6 * (int64_t)R; }
static bool uses_bf16(const cpmg_opts* o) {
  return o->precision == CPMG_PREC_BF16X3 || o->precision == CPMG_PREC_MIXED_BF16;
}

constexpr int kBlkStride = 40;  // doubles of LS-weight bookkeeping per mode (Level::blk)

struct cpmg_hier {
  cpmg_ctx* c = nullptr;
  int N = 0, R = 0, nt = 0;
  std::vector<Level> L;
  void* tmp0 = nullptr;
  void* tmp1 = nullptr;
  double* sortbuf = nullptr;
  double* Aold = nullptr;  // backing of a FactorSet copy for the restart rule
  FactorSet Aprev;
  int ttm_tc = 0;
  void* tcs = nullptr;     // split R-hat operand of the tensor-core restriction
  GraphCache graphs;
};

// Buffers of the split-BF16 tensor-core passes: the two products W = Z x_3 A^(3)^T and
// V = Z x_1 A^(1)^T (float), the transposed factor they contract with, and its split copy.
static int tc_level_alloc(cpmg_ctx* c, Level& L, int R) {
  if (L.Wf || L.dtype != CPMG_F32 || !dt_worth(L.s, R) || !ttm_tc_supported(L.s, CPMG_F32, 0, R) ||
      !ttm_tc_supported(L.s, CPMG_F32, 2, R))
    return CPMG_OK;
  const int64_t P = L.s.dims[0] * L.s.dims[1], imax = std::max(L.s.dims[0], L.s.dims[2]);
  CPMG_TRY(dalloc(c, reinterpret_cast<void**>(&L.Wf), sizeof(float) * (size_t)P * R));
  CPMG_TRY(dalloc(c, reinterpret_cast<void**>(&L.Vf), sizeof(float) * (size_t)R * L.s.dims[1] * L.s.dims[2]));
  CPMG_TRY(dalloc_t(c, &L.AT, (size_t)R * imax));
  return dalloc(c, &L.tcs, ttm_tc_scratch_bytes(imax));
}

static int level_alloc(cpmg_ctx* c, Level& L, int R, int nt) {
  const int N = L.s.N;
  CPMG_TRY(fs_alloc(c, &L.A, N, R, L.s.dims));
  CPMG_TRY(fs_alloc(c, &L.At, N, R, L.s.dims));
  for (int t = 0; t < nt; ++t) CPMG_TRY(fs_alloc(c, &L.tf[t], N, R, L.s.dims));
  size_t tot = 0;
  int64_t imax = 1, icmax = 1;
  for (int n = 0; n < N; ++n) {
    tot += 2 * (size_t)L.s.dims[n] * R;
    imax = std::max(imax, L.s.dims[n]);
    icmax = std::max(icmax, (L.s.dims[n] + 1) / 2);
  }
  CPMG_TRY(dalloc_t(c, &L.buf, tot));
  size_t off = 0;
  for (int n = 0; n < N; ++n) {
    L.F[n] = L.buf + off;
    off += (size_t)L.s.dims[n] * R;
    L.H[n] = L.buf + off;
    off += (size_t)L.s.dims[n] * R;
  }
  CPMG_TRY(dalloc_t(c, &L.M, (size_t)imax * R));
  CPMG_TRY(dalloc_t(c, &L.twork, 2 * (size_t)icmax + 8));
  CPMG_TRY(dalloc_t(c, &L.blk, kBlkStride * kMaxModes));  // per mode: a2, g2, weights, |A Gamma|^2
  if (dt_worth(L.s, R)) CPMG_TRY(dalloc_t(c, &L.W, (size_t)L.s.dims[0] * L.s.dims[1] * R));
  for (int n = 0; n < N; ++n)
    if (L.co[n]) {
      CPMG_TRY(dalloc_t(c, &L.Rhat[n], (size_t)L.cd[n] * L.s.dims[n]));
      CPMG_TRY(dalloc_t(c, &L.Pw[n], 2 * (size_t)L.s.dims[n]));
    }
  return CPMG_OK;
}

static void level_free(cpmg_ctx* c, Level& L) {
  fs_free(c, &L.A);
  fs_free(c, &L.At);
  for (auto& t : L.tf) fs_free(c, &t);
  dfree(c, L.buf);
  dfree(c, L.M);
  dfree(c, L.W);
  dfree(c, L.Wf);
  dfree(c, L.Vf);
  dfree(c, L.AT);
  dfree(c, L.tcs);
  dfree(c, L.twork);
  dfree(c, L.blk);
  dfree(c, L.Zown);
  for (int n = 0; n < kMaxModes; ++n) {
    dfree(c, L.Rhat[n]);
    dfree(c, L.Pw[n]);
  }
  L = Level();
}

static void hier_destroy(cpmg_hier* h) {
  if (!h) return;
  cpmg_ctx* c = h->c;
  if (c->stream) cudaStreamSynchronize(c->stream);
  profile_collect(c);  // graph-owned profiling events leave the pending list before they die
  h->graphs.clear();
  for (auto& L : h->L) level_free(c, L);
  dfree(c, h->tmp0);
  dfree(c, h->tmp1);
  dfree(c, h->tcs);
  dfree(c, h->sortbuf);
  fs_free(c, &h->Aprev);
  delete h;
}

static int64_t coarsest_of(const cpmg_opts* o, int n, int R) {
  int64_t v = o->coarsest[n];
  if (v <= 0) v = R;
  return std::max<int64_t>(v, 1);
}

static int hier_build(cpmg_ctx* c, const Shape& s0, int dtype, int R, const cpmg_opts* o, cpmg_hier** out) {
  cpmg_hier* h = new cpmg_hier();
  h->c = c;
  h->N = s0.N;
  h->R = R;
  h->nt = o->n_t;
  Shape cur = s0;
  size_t tmpb = 0;
  size_t sortn = 0;
  for (int guard = 0; guard < 64; ++guard) {
    Level L;
    L.s = cur;
    L.dtype = dtype;
    bool any = false;
    for (int n = 0; n < cur.N; ++n) {
      L.co[n] = cur.dims[n] > coarsest_of(o, n, R);
      L.cd[n] = L.co[n] ? (cur.dims[n] + 1) / 2 : cur.dims[n];
      any = any || L.co[n];
    }
    h->L.push_back(L);
    if (!any) break;
    // intermediate sizes for this level's restriction
    Shape t = cur;
    const size_t esz = dtype == CPMG_F64 ? 8 : 4;
    for (int n = 0; n < cur.N; ++n)
      if (L.co[n]) {
        t.dims[n] = L.cd[n];
        tmpb = std::max(tmpb, (size_t)t.numel() * esz);
      }
    for (int n = 0; n < cur.N; ++n) cur.dims[n] = L.cd[n];
  }
  int st = CPMG_OK;
  for (size_t l = 0; l < h->L.size() && st == CPMG_OK; ++l) {
    st = level_alloc(c, h->L[l], R, h->nt);
    if (st == CPMG_OK && uses_bf16(o)) st = tc_level_alloc(c, h->L[l], R);
    if (st == CPMG_OK && l > 0) {
      const size_t esz = dtype == CPMG_F64 ? 8 : 4;
      st = dalloc(c, &h->L[l].Zown, (size_t)h->L[l].s.numel() * esz);
      h->L[l].Z = h->L[l].Zown;
    }
    sortn = std::max(sortn, fs_doubles(s0.N, R, h->L[l].s.dims));
  }
  if (st == CPMG_OK) st = dalloc(c, &h->tmp0, tmpb);
  if (st == CPMG_OK) st = dalloc(c, &h->tmp1, tmpb);
  if (st == CPMG_OK && dtype == CPMG_F32 && o->ttm_tensor_cores) {
    int64_t imax = 1;
    for (int n = 0; n < s0.N; ++n) imax = std::max(imax, s0.dims[n]);
    st = dalloc(c, &h->tcs, ttm_tc_scratch_bytes(imax));
  }
  if (st == CPMG_OK) st = dalloc_t(c, &h->sortbuf, sortn);
  if (st == CPMG_OK) st = fs_alloc(c, &h->Aprev, s0.N, R, s0.dims);
  if (st != CPMG_OK) {
    hier_destroy(h);
    return st;
  }
  *out = h;
  return CPMG_OK;
}

// ============================================================================ solver state
struct Solver {
  cpmg_ctx* c;
  cpmg_opts o;
  cudaStream_t st;
  int policy;
  bool refined = false;
  int refine_sweeps = 0;
  double g_best = -1.0;
  int stall = 0;
  double znorm = 0.0;
  double* sortbuf = nullptr;
  int ttm_tc = 0;
  GraphCache* gc = nullptr;     // graphs of the object being solved (null: no graphs)
  const void* z0 = nullptr;     // finest-level tensor the graphs reference
  bool use_graphs = true;

  int prec_for(int /*lvl*/, int dtype) const {
    const int hi = dtype == CPMG_F32 ? P_DF : P_FP64;
    switch (policy) {
      case CPMG_PREC_FP32: return P_FP32;
      case CPMG_PREC_FP64: return P_FP64;
      case CPMG_PREC_DF: return hi;
      case CPMG_PREC_BF16X3: return dtype == CPMG_F32 ? P_BF16 : P_FP64;
      case CPMG_PREC_MIXED_BF16: return refined ? hi : (dtype == CPMG_F32 ? P_BF16 : P_FP32);
      // Once refined, every level is: FP32 rounding on a coarse level would otherwise enter
      // each FAS correction at ~1e-7 relative, independent of the fine residual.
      default: return refined ? hi : P_FP32;
    }
  }
  int gprec(int dtype) const {
    if (policy == CPMG_PREC_FP64) return P_FP64;
    return dtype == CPMG_F32 ? P_DF : P_FP64;
  }
};

// ---------------------------------------------------------------- dimension tree (N = 3)
// W = Z x_3 A^(3)^T is the mode-1 MTTKRP of the (I_1 I_2) x I_3 matricization, so the MTTKRP
// kernels form it as they are; the mode-1 and mode-2 products then come from W (dimtree.cuh).
// Worth it when W (R I_1 I_2 float64, written once, read twice) is small next to a pass over Z.
static bool use_dt(const Solver& S, const Level& L, int R) {
  return S.o.dimension_tree && L.W && dt_worth(L.s, R);
}
static int dt_form_w(Solver& S, const Level& L, const FactorSet& f, int prec) {
  cpmg_ctx* c = S.c;
  const int64_t P = L.s.dims[0] * L.s.dims[1], K = L.s.dims[2];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile && L.Z == c->prof_Z) {
    // algorithmic traffic: Z once, A^(3) once, W written once
    const double bytes = (L.dtype == CPMG_F64 ? 8.0 : 4.0) * (double)(P * K) + 8.0 * f.R * (double)(K + P);
    const int eff = (L.dtype == CPMG_F64 && prec == P_DF) ? P_FP64 : prec;
    CPMG_TRY(prof_events(c, eff == P_FP32 ? 0 : (eff == P_DF ? 1 : 2), bytes, &e0, &e1));
  }
  if (e0) CPMG_CUDA_TRY(cudaEventRecordWithFlags(e0, S.st, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  CPMG_TRY(launch_dt_w(L.Z, L.dtype, P, K, f.R, f.A[2], prec, L.W, c->num_sms, S.st, c->dstatus + 1));
  if (e1) CPMG_CUDA_TRY(cudaEventRecordWithFlags(e1, S.st, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  c->launches += 1;
  return CPMG_OK;
}

// ---------------------------------------------------------------- split BF16 on tensor cores
// Both passes of the dimension tree as tcgen05 mode products (the restriction's kernel, Ic = R):
// W = Z x_3 A^(3)^T gives modes 1 and 2, V = Z x_1 A^(1)^T gives mode 3.  P_BF16 anywhere else
// (a level without the tree, a float64 tensor) runs the FP32 kernels.
static bool use_tc(const Solver& S, const Level& L, int R) { return L.Wf && use_dt(S, L, R); }
static int plain_prec(int prec) { return prec == P_BF16 ? P_FP32 : prec; }

static int tc_product(Solver& S, const Level& L, const FactorSet& f, int mode, float* Y) {
  cpmg_ctx* c = S.c;
  const int64_t In = L.s.dims[mode];
  CPMG_TRY(launch_transpose_d(f.A[mode], In, f.R, L.AT, S.st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile && L.Z == c->prof_Z) {
    // algorithmic traffic: Z once, the product written once
    const double out = mode == 0 ? (double)f.R * L.s.dims[1] * L.s.dims[2] : (double)f.R * L.s.dims[0] * L.s.dims[1];
    CPMG_TRY(prof_events(c, 5, 4.0 * (double)L.s.numel() + 4.0 * out, &e0, &e1));
  }
  CPMG_TRY(ttm_mode_tc(L.s, static_cast<const float*>(L.Z), mode, L.AT, f.R, Y, L.tcs, c->dstatus + 1, e0, e1,
                       c->capturing, S.st));
  c->launches += 3;
  return CPMG_OK;
}

// The N products M^(n) = Z_(n) Phi^(n) at one point f (all modes, no update between them),
// handed in mode order to use(n, M) with M = L.M (overwritten by the next mode).  With the
// dimension tree this streams Z twice instead of N times.
template <typename Fn>
static int mttkrp_all(Solver& S, const Level& L, const FactorSet& f, int prec, Fn&& use) {
  if (prec == P_BF16 && use_tc(S, L, f.R)) {
    CPMG_TRY(tc_product(S, L, f, 2, L.Wf));
    for (int n = 0; n < 2; ++n) {
      CPMG_TRY(launch_dt_contract_f(L.Wf, L.s.dims[0], L.s.dims[1], f.R, n == 0 ? f.A[1] : f.A[0], n, L.M, 1,
                                    L.s.dims[n], S.st));
      S.c->launches += 1;
      CPMG_TRY(use(n, L.M));
    }
    CPMG_TRY(tc_product(S, L, f, 0, L.Vf));
    CPMG_TRY(launch_dt_vmode(L.Vf, L.s.dims[1], L.s.dims[2], f.R, f.A[1], L.M, 1, L.s.dims[2], S.st));
    S.c->launches += 1;
    return use(2, L.M);
  }
  prec = plain_prec(prec);
  if (use_dt(S, L, f.R)) {
    CPMG_TRY(dt_form_w(S, L, f, prec));
    for (int n = 0; n < 2; ++n) {
      CPMG_TRY(launch_dt_contract(L.W, L.s.dims[0], L.s.dims[1], f.R, n == 0 ? f.A[1] : f.A[0], n, L.M, 1,
                                  L.s.dims[n], S.st));
      S.c->launches += 1;
      CPMG_TRY(use(n, L.M));
    }
    CPMG_TRY(run_mttkrp(S.c, L.s, L.Z, L.dtype, f, 2, prec, L.M));
    return use(2, L.M);
  }
  for (int n = 0; n < f.N; ++n) {
    CPMG_TRY(run_mttkrp(S.c, L.s, L.Z, L.dtype, f, n, prec, L.M));
    CPMG_TRY(use(n, L.M));
  }
  return CPMG_OK;
}

// One relaxation sweep, modes in increasing order: kind 0 = ALS update (Section 3), kind 1 =
// BNGS Gauss-Seidel update on A Gamma = M + F (Section 5.2).  `normalize_last`: Eq. ALSnorm in
// the last mode's update.  With the dimension tree, modes 1 and 2 read W (A^(3) is unchanged
// while they are updated) and only mode 3 streams Z again.
static int sweep_modes(Solver& S, const Level& L, FactorSet& f, int prec, int kind, bool hasF,
                       bool normalize_last) {
  const int gs = kind == 1 ? S.o.gs_sweeps : 0;
  // products taken outside the MTTKRP kernels go to the fused update kernel as one float64
  // partial row per output row
  MttkrpPlan q;
  q.mode = 1;
  q.nseg = 1;
  q.C = 1;
  q.nw = 1;
  q.RP = f.R;
  q.SEG = 1;
  q.part_elem = 8;
  MttkrpScratch w;
  w.partial = S.c->mt_partial;
  w.tables = S.c->mt_tables;
  double* rows = static_cast<double*>(S.c->mt_partial);
  auto update = [&](int n, bool norm) -> int {
    S.c->launches += 1;
    return launch_finish_update(q, w, f, n, kind, hasF ? L.F[n] : nullptr, gs, nullptr, S.c->gscratch,
                                S.c->dstatus + 2, S.c->dstatus, S.st, norm);
  };
  if (prec == P_BF16 && use_tc(S, L, f.R)) {
    CPMG_TRY(tc_product(S, L, f, 2, L.Wf));
    for (int n = 0; n < 2; ++n) {
      CPMG_TRY(launch_dt_contract_f(L.Wf, L.s.dims[0], L.s.dims[1], f.R, n == 0 ? f.A[1] : f.A[0], n, rows, f.R, 1,
                                    S.st));
      S.c->launches += 1;
      CPMG_TRY(update(n, false));
    }
    // mode 3 needs the updated A^(1) and A^(2): V = Z x_1 A^(1)^T, then the contraction with A^(2)
    CPMG_TRY(tc_product(S, L, f, 0, L.Vf));
    CPMG_TRY(launch_dt_vmode(L.Vf, L.s.dims[1], L.s.dims[2], f.R, f.A[1], rows, f.R, 1, S.st));
    S.c->launches += 1;
    return update(2, normalize_last);
  }
  prec = plain_prec(prec);
  if (use_dt(S, L, f.R)) {
    CPMG_TRY(dt_form_w(S, L, f, prec));
    for (int n = 0; n < 2; ++n) {
      CPMG_TRY(launch_dt_contract(L.W, L.s.dims[0], L.s.dims[1], f.R, n == 0 ? f.A[1] : f.A[0], n, rows, f.R, 1,
                                  S.st));
      S.c->launches += 1;
      CPMG_TRY(update(n, false));
    }
    return run_mttkrp_k(S.c, L.s, L.Z, L.dtype, f, 2, prec, nullptr, kind, hasF ? L.F[2] : nullptr, gs,
                        normalize_last);
  }
  for (int n = 0; n < f.N; ++n)
    CPMG_TRY(run_mttkrp_k(S.c, L.s, L.Z, L.dtype, f, n, prec, nullptr, kind, hasF ? L.F[n] : nullptr, gs,
                          normalize_last && n == f.N - 1));
  return CPMG_OK;
}

// One ALS iteration over all modes plus normalization (Section 3, Eq. ALSnorm).
static int als_sweep(Solver& S, const Level& L, int lvl, FactorSet& f) {
  const int prec = S.prec_for(lvl, L.dtype);
  // the last mode's update also normalizes (Eq. ALSnorm) in its final block
  CPMG_TRY(sweep_modes(S, L, f, prec, 0, false, true));
  if (lvl == 0 && prec != P_FP32 && prec != P_BF16) S.refine_sweeps++;
  return CPMG_OK;
}

static int relax_als(Solver& S, const Level& L, int lvl, FactorSet& f, int iters, bool sort) {
  for (int it = 0; it < iters; ++it) CPMG_TRY(als_sweep(S, L, lvl, f));
  if (sort) {
    CPMG_TRY(launch_sort(f, S.sortbuf, S.st));
    S.c->launches += 1;
  }
  return CPMG_OK;
}

// BNGS (Section 5.2): Gauss-Seidel on A Gamma = M + F per mode; top level normalizes + sorts.
static int relax_bngs(Solver& S, const Level& L, int lvl, FactorSet& f, bool hasF, int iters, bool top) {
  const int prec = S.prec_for(lvl, L.dtype);
  for (int it = 0; it < iters; ++it) {
    CPMG_TRY(sweep_modes(S, L, f, prec, 1, hasF, false));
    if (lvl == 0 && prec != P_FP32 && prec != P_BF16) S.refine_sweeps++;
    if (top) {
      CPMG_TRY(launch_normalize(f, S.st));
      CPMG_TRY(launch_sort(f, S.sortbuf, S.st));
      S.c->launches += 3;
    }
  }
  return CPMG_OK;
}

// g of Eq. gradConv on level L with float64-accurate MTTKRPs, in two parts: the launches
// (capturable: MTTKRPs, gradient norms, copies of the scalars to pinned host memory) and the
// host read after a synchronization.  Also yields ||M|| for the precision switch.
static int eval_g_launch(Solver& S, const Level& L, FactorSet& f) {
  const int prec = S.gprec(L.dtype);
  CPMG_TRY(mttkrp_all(S, L, f, prec, [&](int n, const double* M) -> int {
    CPMG_TRY(launch_grad_sq(f, n, M, S.c->dsc, n, S.st));
    CPMG_TRY(launch_sq_norm(M, L.s.dims[n] * f.R, S.c->dsc, 64 + n, S.st));
    S.c->launches += 2;
    return CPMG_OK;
  }));
  CPMG_CUDA_TRY(cudaMemcpyAsync(S.c->hsc, S.c->dsc, 128 * sizeof(double), cudaMemcpyDeviceToHost, S.st));
  CPMG_CUDA_TRY(cudaMemcpyAsync(S.c->hsc + 128, S.c->dstatus, 4 * sizeof(int), cudaMemcpyDeviceToHost, S.st));
  return CPMG_OK;
}

static int eval_g_read(Solver& S, int N, double* g, double* mnorm) {
  CPMG_CUDA_TRY(cudaStreamSynchronize(S.st));
  if (reinterpret_cast<const int*>(S.c->hsc + 128)[1] != 0) return CPMG_TIMEOUT;
  double sg = 0.0, sm = 0.0;
  for (int n = 0; n < N; ++n) {
    sg += S.c->hsc[n];
    sm += S.c->hsc[64 + n];
  }
  *g = std::sqrt(sg) / S.znorm;
  if (mnorm) *mnorm = std::sqrt(sm);
  if (!std::isfinite(*g)) return CPMG_NUMERIC;
  return CPMG_OK;
}

static int eval_g(Solver& S, const Level& L, FactorSet& f, double* g, double* mnorm) {
  CPMG_TRY(eval_g_launch(S, L, f));
  return eval_g_read(S, f.N, g, mnorm);
}

// MIXED policy: switch to float64-accurate sweeps once g is within a factor K of the
// FP32 floor, estimated as eps_32 ||M|| / ||Z|| (the size of one FP32 rounding of the
// MTTKRP seen through Eq. gradConv), or after 20 checks without a new smallest g.
static void maybe_switch(Solver& S, double g, double mnorm, double /*g_prev*/) {
  if ((S.policy != CPMG_PREC_MIXED && S.policy != CPMG_PREC_MIXED_BF16) || S.refined) return;
  const double K = S.o.mixed_switch > 0 ? S.o.mixed_switch : 4.0;
  // one rounding of the sweep's products: 2^-24 in FP32, about 2^-16 for split BF16
  const double u = S.policy == CPMG_PREC_MIXED_BF16 ? 1.52587890625e-05 : 5.960464477539063e-08;
  const double floor_est = K * u * mnorm / S.znorm;
  if (S.g_best < 0 || g < S.g_best) {
    S.g_best = g;
    S.stall = 0;
  } else {
    ++S.stall;
  }
  if (g < floor_est || S.stall >= 20) S.refined = true;
}

// Sweeps to run before the next exact g check: about half of the sweeps that the observed
// per-sweep contraction predicts are left, as a power of two in [1, 32].  The iterates do not
// depend on it; only the stopping point can move by at most that many sweeps.
static int next_check_interval(double g, double g_prev, int k_prev, double tol) {
  if (g_prev <= 0 || !(g > 0)) return 1;
  const double rho = std::pow(g / g_prev, 1.0 / std::max(k_prev, 1));
  int k;
  if (!(rho < 1.0)) {
    k = std::min(2 * k_prev, 32);
  } else {
    const double n_left = std::log(tol / g) / std::log(rho);
    const double half = 0.5 * n_left;
    k = 1;
    while (k * 2 <= half && k < 32) k *= 2;
  }
  return std::max(1, std::min(k, 32));
}

template <typename Fn>
static int graph_run(Solver& S, const std::string& key, Fn&& body) {
  if (!S.use_graphs || !S.gc) return body();
  cpmg_ctx* c = S.c;
  auto it = S.gc->m.find(key);
  if (it != S.gc->m.end() && it->second.z0 != S.z0) {
    CPMG_CUDA_TRY(cudaStreamSynchronize(S.st));
    CPMG_TRY(profile_collect(c));
    if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
    for (auto& e : it->second.events) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    S.gc->m.erase(it);
    it = S.gc->m.end();
  }
  if (it != S.gc->m.end()) {
    CPMG_CUDA_TRY(cudaGraphLaunch(it->second.exec, S.st));
    c->launches += it->second.dlaunch;
    S.refine_sweeps += it->second.drefine;
    for (auto& e : it->second.events) c->pending.push_back(e);
    if (c->pending.size() > 4096) CPMG_TRY(profile_collect(c));
    return CPMG_OK;
  }
  const int64_t l0 = c->launches;
  const int r0 = S.refine_sweeps;
  const size_t p0 = c->pending.size();
  CPMG_CUDA_TRY(cudaStreamBeginCapture(S.st, cudaStreamCaptureModeThreadLocal));
  c->capturing = true;
  int st = body();
  c->capturing = false;
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(S.st, &g);
  GraphEntry e;
  e.events.assign(c->pending.begin() + p0, c->pending.end());
  c->pending.resize(p0);
  cudaError_t ie = cudaSuccess;
  if (st == CPMG_OK && ce == cudaSuccess && g) ie = cudaGraphInstantiate(&e.exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (st != CPMG_OK || ce != cudaSuccess || !g || ie != cudaSuccess) {
    for (auto& ev : e.events) {
      cudaEventDestroy(ev.a);
      cudaEventDestroy(ev.b);
    }
    if (st != CPMG_OK) {
      cudaGetLastError();
      return st;
    }
    set_last_error(ce != cudaSuccess ? ce : ie, "graph capture", __FILE__, __LINE__);
    cudaGetLastError();
    return CPMG_CUDA_ERROR;
  }
  e.z0 = S.z0;
  e.dlaunch = c->launches - l0;
  e.drefine = S.refine_sweeps - r0;
  CPMG_CUDA_TRY(cudaGraphLaunch(e.exec, S.st));
  for (auto& ev : e.events) c->pending.push_back(ev);
  S.gc->m[key] = std::move(e);
  return CPMG_OK;
}

// Plans (and scratch sized for them) for every MTTKRP a solve can issue, so that nothing is
// planned or allocated while a graph is being captured.
static int preplan(cpmg_ctx* c, const std::vector<const Level*>& levels, int R) {
  size_t part = 0, tab = 0;
  for (const Level* L : levels) {
    for (int n = 0; n < L->s.N; ++n)
      for (int prec : {(int)P_FP32, (int)P_FP64, (int)P_DF}) {
        const MttkrpPlan* p = nullptr;
        CPMG_TRY(get_plan(c, L->s, n, R, prec, L->dtype, L->Z, &p));
        part = std::max(part, p->partial_bytes());
        tab = std::max(tab, p->tables_bytes());
      }
    if (L->W)  // the dimension tree: float64 rows of the W products for the fused update
      part = std::max(part, sizeof(double) * (size_t)std::max(L->s.dims[0], L->s.dims[1]) * R);
  }
  return ensure_scratch(c, part, tab);
}

static int tensor_norm(Solver& S, const Level& L, FactorSet& f, double* znorm) {
  double* partial = nullptr;
  CPMG_TRY(dalloc_t(S.c, &partial, 2 * 1024 + 8));
  int st = launch_f_direct(L.s, L.Z, L.dtype, f, partial, S.c->dsc + 200, S.st);
  if (st == CPMG_OK) {
    if (cudaMemcpyAsync(S.c->hsc + 200, S.c->dsc + 200, 2 * sizeof(double), cudaMemcpyDeviceToHost, S.st) !=
            cudaSuccess ||
        cudaStreamSynchronize(S.st) != cudaSuccess)
      st = CPMG_CUDA_ERROR;
  }
  dfree(S.c, partial);
  S.c->launches += 2;
  if (st == CPMG_OK) *znorm = std::sqrt(S.c->hsc[201]);
  return st;
}

static int eval_f(Solver& S, const Level& L, FactorSet& f, double* fval, double* znorm2) {
  double* partial = nullptr;
  CPMG_TRY(dalloc_t(S.c, &partial, 2 * 1024 + 8));
  int st = launch_f_direct(L.s, L.Z, L.dtype, f, partial, S.c->dsc + 200, S.st);
  if (st == CPMG_OK) {
    if (cudaMemcpyAsync(S.c->hsc + 200, S.c->dsc + 200, 2 * sizeof(double), cudaMemcpyDeviceToHost, S.st) !=
            cudaSuccess ||
        cudaStreamSynchronize(S.st) != cudaSuccess)
      st = CPMG_CUDA_ERROR;
  }
  dfree(S.c, partial);
  S.c->launches += 2;
  if (st == CPMG_OK) {
    *fval = 0.5 * S.c->hsc[200];
    if (znorm2) *znorm2 = S.c->hsc[201];
  }
  return st;
}

// ============================================================================ Algorithm 1
// Interpolation operators of one level (Sections 4.3, 4.4) and their transforms (Section 4.1).
static int build_operators(Solver& S, cpmg_hier* h, int lvl, bool first) {
  Level& L = h->L[lvl];
  const int R = h->R;
  const int prec = S.prec_for(lvl, L.dtype);
  int nb = 0;
  FactorSet* blocks[CPMG_MAX_TEST_BLOCKS + 1];
  for (int t = 0; t < h->nt; ++t) blocks[nb++] = &L.tf[t];
  if (!first) blocks[nb++] = &L.A;
  // per block, the gradients of every coarsened mode at the block's point (one all-modes MTTKRP);
  // mode n's norms sit at L.blk + kBlkStride n: a2 @0, g2 @8, weights @16, |A Gamma|^2 @24
  for (int k = 0; k < nb; ++k)
    CPMG_TRY(mttkrp_all(S, L, *blocks[k], prec, [&](int n, const double* M) -> int {
      if (!L.co[n]) return CPMG_OK;
      double* b = L.blk + kBlkStride * n;
      CPMG_TRY(launch_sq_norm(blocks[k]->A[n], L.s.dims[n] * R, b, k, S.st));
      CPMG_TRY(launch_grad_sq(*blocks[k], n, M, b, 8 + k, S.st, 24 + k));
      S.c->launches += 2;
      return CPMG_OK;
    }));
  for (int n = 0; n < L.s.N; ++n) {
    if (!L.co[n]) continue;
    const double* U[CPMG_MAX_TEST_BLOCKS + 1];
    for (int k = 0; k < nb; ++k) U[k] = blocks[k]->A[n];
    double* b = L.blk + kBlkStride * n;
    // a gradient at the rounding level of the MTTKRP that produced it counts as zero
    const double tau = prec == P_BF16 ? 1e-4 : prec == P_FP32 ? 1e-5 : 1e-12;
    CPMG_TRY(launch_block_weights(nb, b, b + 8, b + 24, tau, b + 16, S.st));
    CPMG_TRY(launch_interp(L.s.dims[n], R, nb, U, b + 16, L.Pw[n], S.st));
    CPMG_TRY(launch_transform(L.s.dims[n], L.Pw[n], L.Rhat[n], L.twork, S.st));
    S.c->launches += 3;
  }
  return CPMG_OK;
}

// Eq. coarseapprox_new: dst (coarse) = R-hat src (n in I_c) or src; Grams refreshed.
static int restrict_set(Solver& S, const Level& L, const FactorSet& src, FactorSet& dst) {
  const int R = src.R;
  for (int n = 0; n < src.N; ++n) {
    if (L.co[n])
      CPMG_TRY(launch_dgemm_small(false, L.cd[n], R, L.s.dims[n], 1.0, L.Rhat[n], L.cd[n], src.A[n],
                                  L.s.dims[n], 0.0, dst.A[n], L.cd[n], S.st));
    else
      CPMG_TRY(launch_copy_d(dst.A[n], src.A[n], L.s.dims[n] * R, S.st));
    S.c->launches += 1;
  }
  CPMG_TRY(launch_grams(dst, all_modes(dst.N), S.st));
  S.c->launches += 1;
  return CPMG_OK;
}

static int amg_mult(Solver& S, cpmg_hier* h, int lvl, bool first, bool relax_boot, bool upsweep) {
  Level& L = h->L[lvl];
  const cpmg_opts& o = S.o;
  if (!L.coarsest()) {
    Level& C = h->L[lvl + 1];
    for (int t = 0; t < h->nt; ++t) CPMG_TRY(relax_als(S, L, lvl, L.tf[t], o.nu1_setup, true));
    if (relax_boot) CPMG_TRY(relax_als(S, L, lvl, L.A, o.nu1_setup, true));
    CPMG_TRY(build_operators(S, h, lvl, first));
    CPMG_TRY(restrict_set(S, L, L.A, C.A));
    for (int t = 0; t < h->nt; ++t) CPMG_TRY(restrict_set(S, L, L.tf[t], C.tf[t]));
    const double* Rh[kMaxModes];
    for (int n = 0; n < kMaxModes; ++n) Rh[n] = (n < L.s.N && L.co[n]) ? L.Rhat[n] : nullptr;
    const int tc = h->tcs ? S.ttm_tc : 0;
    cudaEvent_t ev[2 * kMaxModes];
    CPMG_TRY(prof_ttm(S.c, L.s, L.dtype, Rh, L.cd, L.Z == S.c->prof_Z ? tc : 0, ev));
    CPMG_TRY(ttm_restrict(L.s, L.Z, L.dtype, Rh, L.cd, const_cast<void*>(C.Z), h->tmp0, h->tmp1, tc, h->tcs,
                          S.c->dstatus + 1, ev, S.c->capturing, S.st));
    S.c->launches += 3;
    CPMG_TRY(amg_mult(S, h, lvl + 1, first, relax_boot, upsweep));
    if (upsweep) {
      for (int n = 0; n < L.s.N; ++n) {  // Eq. CGC_new
        if (L.co[n])
          CPMG_TRY(launch_dgemm_small(true, L.s.dims[n], h->R, L.cd[n], 1.0, L.Rhat[n], L.cd[n], C.A.A[n],
                                      L.cd[n], 0.0, L.A.A[n], L.s.dims[n], S.st));
        else
          CPMG_TRY(launch_copy_d(L.A.A[n], C.A.A[n], L.s.dims[n] * h->R, S.st));
        S.c->launches += 1;
      }
      CPMG_TRY(launch_grams(L.A, all_modes(L.s.N), S.st));
      CPMG_TRY(relax_als(S, L, lvl, L.A, o.nu2_setup, true));
    }
  } else if (upsweep) {
    CPMG_TRY(relax_als(S, L, lvl, L.A, o.nuc_setup, true));
  }
  return CPMG_OK;
}

// ============================================================================ Algorithm 2
static int cp_fas(Solver& S, cpmg_hier* h, int lvl, bool hasF, int top) {
  Level& L = h->L[lvl];
  const cpmg_opts& o = S.o;
  const bool is_top = lvl == top;
  if (!L.coarsest()) {
    Level& C = h->L[lvl + 1];
    const int R = h->R;
    CPMG_TRY(relax_bngs(S, L, lvl, L.A, hasF, o.nu1, is_top));
    CPMG_TRY(restrict_set(S, L, L.A, C.At));  // coarse guess A~_c
    CPMG_TRY(fs_copy(C.A, C.At, S.st));
    const int prec_f = S.prec_for(lvl, L.dtype);
    const int prec_c = S.prec_for(lvl + 1, C.dtype);
    // r = F - H(A) on this level (Eq. FASrhs), kept in L.H[n]: all modes at the point A
    CPMG_TRY(mttkrp_all(S, L, L.A, prec_f, [&](int n, const double* M) -> int {
      CPMG_TRY(launch_fas_op(L.A, n, M, L.H[n], S.st));
      if (hasF) CPMG_TRY(launch_axpby(L.s.dims[n] * R, 1.0, L.F[n], -1.0, L.H[n], S.st));
      else CPMG_TRY(launch_axpby(L.s.dims[n] * R, 0.0, L.H[n], -1.0, L.H[n], S.st));
      return CPMG_OK;
    }));
    // H_c(A~_c) into C.F[n]: all modes at the point A~_c
    CPMG_TRY(mttkrp_all(S, C, C.At, prec_c, [&](int n, const double* M) -> int {
      return launch_fas_op(C.At, n, M, C.F[n], S.st);
    }));
    for (int n = 0; n < L.s.N; ++n) {
      // F_c = H_c(A~_c) + R-hat r   (identity for modes not coarsened)
      if (L.co[n])
        CPMG_TRY(launch_dgemm_small(false, L.cd[n], R, L.s.dims[n], 1.0, L.Rhat[n], L.cd[n], L.H[n],
                                    L.s.dims[n], 1.0, C.F[n], L.cd[n], S.st));
      else
        CPMG_TRY(launch_axpby(L.s.dims[n] * R, 1.0, L.H[n], 1.0, C.F[n], S.st));
      S.c->launches += 4;
    }
    CPMG_TRY(cp_fas(S, h, lvl + 1, true, top));
    for (int n = 0; n < L.s.N; ++n) {  // Eq. FASCGC: A += P-hat (A_c - A~_c)
      CPMG_TRY(launch_axpby(C.s.dims[n] * R, -1.0, C.At.A[n], 1.0, C.A.A[n], S.st));
      if (L.co[n])
        CPMG_TRY(launch_dgemm_small(true, L.s.dims[n], R, L.cd[n], 1.0, L.Rhat[n], L.cd[n], C.A.A[n],
                                    L.cd[n], 1.0, L.A.A[n], L.s.dims[n], S.st));
      else
        CPMG_TRY(launch_axpby(L.s.dims[n] * R, 1.0, C.A.A[n], 1.0, L.A.A[n], S.st));
      S.c->launches += 2;
    }
    CPMG_TRY(launch_grams(L.A, all_modes(L.s.N), S.st));
    CPMG_TRY(relax_bngs(S, L, lvl, L.A, hasF, o.nu2, is_top));
  } else {
    CPMG_TRY(relax_bngs(S, L, lvl, L.A, hasF, o.nuc, is_top));
  }
  return CPMG_OK;
}

// ============================================================================ ABI helpers
static int check_tensor(const cpmg_tensor* Z) {
  if (!Z || !Z->data) return CPMG_INVALID_ARG;
  if (Z->N < 2 || Z->N > CPMG_MAX_MODES) return CPMG_INVALID_ARG;
  if (Z->dtype != CPMG_F32 && Z->dtype != CPMG_F64) return CPMG_INVALID_ARG;
  if (Z->mem != CPMG_MEM_DEVICE && Z->mem != CPMG_MEM_HOST) return CPMG_INVALID_ARG;
  for (int n = 0; n < Z->N; ++n)
    if (Z->dims[n] < 1) return CPMG_INVALID_ARG;
  return CPMG_OK;
}

static Shape shape_of(const cpmg_tensor* Z) {
  Shape s;
  s.N = Z->N;
  for (int n = 0; n < Z->N; ++n) s.dims[n] = Z->dims[n];
  return s;
}

// Device view of the caller's tensor (copied in when it lives in host memory).
struct ZView {
  const void* dev = nullptr;
  void* own = nullptr;
};

static int resolve_tensor(cpmg_ctx* c, const cpmg_tensor* Z, ZView* v) {
  if (Z->mem == CPMG_MEM_DEVICE) {
    v->dev = Z->data;
    return CPMG_OK;
  }
  const size_t bytes = (size_t)shape_of(Z).numel() * (Z->dtype == CPMG_F64 ? 8 : 4);
  CPMG_TRY(dalloc(c, &v->own, bytes));
  CPMG_CUDA_TRY(cudaMemcpyAsync(v->own, Z->data, bytes, cudaMemcpyHostToDevice, c->stream));
  v->dev = v->own;
  return CPMG_OK;
}

static int factors_in(cpmg_ctx* c, int mem, double* const* A, FactorSet& f) {
  const cudaMemcpyKind k = mem == CPMG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (int n = 0; n < f.N; ++n) {
    if (!A[n]) return CPMG_INVALID_ARG;
    CPMG_CUDA_TRY(cudaMemcpyAsync(f.A[n], A[n], f.dims[n] * f.R * sizeof(double), k, c->stream));
  }
  return launch_grams(f, all_modes(f.N), c->stream);
}

static int factors_out(cpmg_ctx* c, int mem, const FactorSet& f, double* const* A) {
  const cudaMemcpyKind k = mem == CPMG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  for (int n = 0; n < f.N; ++n)
    CPMG_CUDA_TRY(cudaMemcpyAsync(A[n], f.A[n], f.dims[n] * f.R * sizeof(double), k, c->stream));
  return CPMG_OK;
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static Solver make_solver(cpmg_ctx* c, const cpmg_opts* o) {
  Solver S{c, *o, c->stream, o->precision};
  // stream capture is not available on the legacy default stream
  S.use_graphs = o->use_graphs != 0 && c->stream != nullptr;
  S.ttm_tc = o->ttm_tensor_cores ? 1 : 0;
  // the timeout flag of an earlier call that gave up is not this call's
  cudaMemsetAsync(c->dstatus + 1, 0, sizeof(int), c->stream);
  return S;
}

static int check_opts(const cpmg_opts* o) {
  if (!o) return CPMG_INVALID_ARG;
  if (o->precision < 0 || o->precision > 5) return CPMG_INVALID_ARG;
  if (o->n_t < 0 || o->n_t > CPMG_MAX_TEST_BLOCKS) return CPMG_INVALID_ARG;
  if (o->gs_sweeps < 0 || o->nu1 < 0 || o->nu2 < 0 || o->nuc < 0) return CPMG_INVALID_ARG;
  return CPMG_OK;
}

// ============================================================================ Algorithm 3
// FMG-CP-FAS: nu ALS iterations (normalized, sorted at the end) on the coarsest level from the
// level's current factors, then for each finer level: prolongate by P-hat (the transpose of
// R-hat; identity for modes not coarsened) and one CP-FAS cycle with F = 0 topped at that level.
// Leaves the finest-level result in h->L[0].A.
static int fmg_cycle(Solver& S, cpmg_hier* h, int nu) {
  const int Lc = (int)h->L.size() - 1;
  CPMG_TRY(relax_als(S, h->L[Lc], Lc, h->L[Lc].A, nu, true));
  for (int lvl = Lc - 1; lvl >= 0; --lvl) {
    Level& L = h->L[lvl];
    const Level& C = h->L[lvl + 1];
    for (int n = 0; n < L.s.N; ++n) {
      if (L.co[n])
        CPMG_TRY(launch_dgemm_small(true, L.s.dims[n], h->R, L.cd[n], 1.0, L.Rhat[n], L.cd[n], C.A.A[n],
                                    L.cd[n], 0.0, L.A.A[n], L.s.dims[n], S.st));
      else
        CPMG_TRY(launch_copy_d(L.A.A[n], C.A.A[n], L.s.dims[n] * h->R, S.st));
      S.c->launches += 1;
    }
    CPMG_TRY(launch_grams(L.A, all_modes(L.s.N), S.st));
    S.c->launches += 1;
    CPMG_TRY(cp_fas(S, h, lvl, false, lvl));
  }
  return CPMG_OK;
}

// ============================================================================ C ABI
extern "C" {

void cpmg_opts_default(cpmg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = CPMG_PREC_MIXED;
  o->tol = 1e-10;
  o->max_cycles = 500;
  o->max_als_iters = 10000;
  o->nu1_setup = 5;
  o->nu2_setup = 5;
  o->nuc_setup = 100;
  o->nu1 = 1;
  o->nu2 = 1;
  o->nuc = 50;
  o->n_t = 2;
  o->max_setup_cycles = 5;
  o->stag_eps = 0.1;
  o->gs_sweeps = 10;
  o->als_fallback = 0;
  o->mixed_switch = 4.0;
  o->check_every = 1;
  o->use_graphs = 1;
  o->ttm_tensor_cores = 1;
  o->dimension_tree = 1;
}

const char* cpmg_status_str(int s) {
  switch (s) {
    case CPMG_OK: return "ok";
    case CPMG_INVALID_ARG: return "invalid argument";
    case CPMG_OUT_OF_BUDGET: return "out of HBM budget";
    case CPMG_NOT_CONVERGED: return "not converged";
    case CPMG_NUMERIC: return "numeric failure (NaN/Inf)";
    case CPMG_TIMEOUT: return "timeout";
    case CPMG_CUDA_ERROR: return g_errbuf[0] ? g_errbuf : "CUDA error";
    case CPMG_PENDING: return "pending";
    case CPMG_CANCELLED: return "cancelled";
    case CPMG_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

int cpmg_create(cpmg_ctx** out, int device, size_t budget, void* stream) {
  if (!out) return CPMG_INVALID_ARG;
  *out = nullptr;
  CPMG_CUDA_TRY(cudaSetDevice(device));
  cpmg_ctx* c = new cpmg_ctx();
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->budget = budget;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
    c->num_sms = sms;
  int st = dalloc_t(c, &c->dsc, 4096);
  if (st == CPMG_OK) st = dalloc_t(c, &c->dstatus, 64);
  if (st == CPMG_OK) st = dalloc_t(c, &c->gscratch, (size_t)kFuseMaxBlocks * kMaxRank * (kMaxRank + 1) / 2);
  if (st == CPMG_OK && cudaMallocHost(&c->hsc, 4096 * sizeof(double)) != cudaSuccess) st = CPMG_CUDA_ERROR;
  if (st == CPMG_OK && cudaMemsetAsync(c->dsc, 0, 4096 * sizeof(double), c->stream) != cudaSuccess)
    st = CPMG_CUDA_ERROR;
  if (st == CPMG_OK && cudaMemsetAsync(c->dstatus, 0, 64 * sizeof(int), c->stream) != cudaSuccess)
    st = CPMG_CUDA_ERROR;
  if (st != CPMG_OK) {
    cpmg_destroy(c);
    return st;
  }
  *out = c;
  return CPMG_OK;
}

void cpmg_destroy(cpmg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  batch_state_destroy(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto& p : c->pool) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  std::vector<void*> ptrs;
  for (auto& kv : c->sizes) ptrs.push_back(kv.first);
  for (void* p : ptrs) dfree(c, p);
  if (c->hsc) cudaFreeHost(c->hsc);
  delete c;
}

int cpmg_set_stream(cpmg_ctx* c, void* stream) {
  if (!c) return CPMG_INVALID_ARG;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return CPMG_OK;
}

size_t cpmg_bytes_in_use(const cpmg_ctx* c) { return c ? c->in_use : 0; }

int64_t cpmg_launch_count(const cpmg_ctx* c) { return c ? c->launches : 0; }

int cpmg_profile_enable(cpmg_ctx* c, int enable) {
  if (!c) return CPMG_INVALID_ARG;
  c->profile = enable != 0;
  return CPMG_OK;
}

int cpmg_profile_read(cpmg_ctx* c, int kind, double* total_ms, int64_t* launches, double* bytes) {
  if (!c || kind < 0 || kind > 5) return CPMG_INVALID_ARG;
  CPMG_TRY(profile_collect(c));
  if (total_ms) *total_ms = c->prof_ms[kind];
  if (launches) *launches = c->prof_launches[kind];
  if (bytes) *bytes = c->prof_launches[kind] ? c->prof_bytes[kind] / c->prof_launches[kind] : 0.0;
  return CPMG_OK;
}

int cpmg_profile_reset(cpmg_ctx* c) {
  if (!c) return CPMG_INVALID_ARG;
  CPMG_TRY(profile_collect(c));
  for (int k = 0; k < 6; ++k) {
    c->prof_ms[k] = 0;
    c->prof_launches[k] = 0;
    c->prof_bytes[k] = 0;
  }
  return CPMG_OK;
}

int cpmg_mttkrp(cpmg_ctx* c, const cpmg_tensor* Z, int R, const double* const* A, int mode, int precision,
                double* M) {
  cudaGetLastError();  // an error left pending by the caller is not this call's
  if (!c || !A || !M) return CPMG_INVALID_ARG;
  CPMG_TRY(check_tensor(Z));
  if (Z->mem != CPMG_MEM_DEVICE) return CPMG_INVALID_ARG;
  if (R < 1 || R > CPMG_MAX_RANK || mode < 0 || mode >= Z->N) return CPMG_INVALID_ARG;
  int prec;
  switch (precision) {
    case CPMG_PREC_FP32: prec = P_FP32; break;
    case CPMG_PREC_FP64: prec = P_FP64; break;
    case CPMG_PREC_DF: prec = P_DF; break;
    default: return CPMG_INVALID_ARG;
  }
  const Shape s = shape_of(Z);
  FactorSet f;
  f.N = Z->N;
  f.R = R;
  for (int m = 0; m < Z->N; ++m) {
    if (!A[m]) return CPMG_INVALID_ARG;
    f.dims[m] = Z->dims[m];
    f.A[m] = const_cast<double*>(A[m]);
  }
  CPMG_TRY(run_mttkrp(c, s, Z->data, Z->dtype, f, mode, prec, M));
  CPMG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return CPMG_OK;
}

int cpmg_ttm(cpmg_ctx* c, const cpmg_tensor* Z, const double* const* Rhat, const int64_t* Ic, int tensor_cores,
             void* Y) {
  cudaGetLastError();  // an error left pending by the caller is not this call's
  if (!c || !Rhat || !Ic || !Y) return CPMG_INVALID_ARG;
  CPMG_TRY(check_tensor(Z));
  if (Z->mem != CPMG_MEM_DEVICE) return CPMG_INVALID_ARG;
  const Shape s = shape_of(Z);
  const double* Rh[kMaxModes];
  int64_t icv[kMaxModes];
  for (int n = 0; n < kMaxModes; ++n) {
    Rh[n] = n < s.N ? Rhat[n] : nullptr;
    icv[n] = n < s.N ? Ic[n] : 0;
    if (Rh[n] && icv[n] < 1) return CPMG_INVALID_ARG;
  }
  if (tensor_cores && Z->dtype != CPMG_F32) return CPMG_UNSUPPORTED;
  const size_t tb = ttm_max_intermediate(s, Z->dtype, Rh, icv);
  int64_t imax = 1;
  for (int n = 0; n < s.N; ++n) imax = std::max(imax, s.dims[n]);
  void *t0 = nullptr, *t1 = nullptr, *tcs = nullptr;
  int st = dalloc(c, &t0, tb);
  if (st == CPMG_OK) st = dalloc(c, &t1, tb);
  if (st == CPMG_OK && tensor_cores) st = dalloc(c, &tcs, ttm_tc_scratch_bytes(imax));
  cudaEvent_t ev[2 * kMaxModes];
  if (st == CPMG_OK) st = prof_ttm(c, s, Z->dtype, Rh, icv, tensor_cores, ev);
  if (st == CPMG_OK && cudaMemsetAsync(c->dstatus + 1, 0, sizeof(int), c->stream) != cudaSuccess)
    st = CPMG_CUDA_ERROR;
  if (st == CPMG_OK)
    st = ttm_restrict(s, Z->data, Z->dtype, Rh, icv, Y, t0, t1, tensor_cores ? 2 : 0, tcs, c->dstatus + 1, ev,
                      false, c->stream);
  if (st == CPMG_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = CPMG_CUDA_ERROR;
  if (st == CPMG_OK) {
    int dflag = 0;
    if (cudaMemcpy(&dflag, c->dstatus + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) st = CPMG_CUDA_ERROR;
    else if (dflag) st = CPMG_TIMEOUT;
  }
  dfree(c, t0);
  dfree(c, t1);
  dfree(c, tcs);
  return st;
}

int cpmg_eval_fg(cpmg_ctx* c, const cpmg_tensor* Z, int R, const double* const* A, double* f, double* g) {
  cudaGetLastError();  // an error left pending by the caller is not this call's
  if (!c || !A) return CPMG_INVALID_ARG;
  CPMG_TRY(check_tensor(Z));
  if (Z->mem != CPMG_MEM_DEVICE || R < 1 || R > CPMG_MAX_RANK) return CPMG_INVALID_ARG;
  cpmg_opts o;
  cpmg_opts_default(&o);
  Solver S = make_solver(c, &o);
  Level L;
  L.s = shape_of(Z);
  L.Z = Z->data;
  L.dtype = Z->dtype;
  FactorSet fs;
  CPMG_TRY(fs_alloc(c, &fs, Z->N, R, L.s.dims));
  int st = factors_in(c, CPMG_MEM_DEVICE, const_cast<double* const*>(A), fs);
  double* M = nullptr;
  int64_t imax = 1;
  for (int n = 0; n < Z->N; ++n) imax = std::max(imax, Z->dims[n]);
  if (st == CPMG_OK) st = dalloc_t(c, &M, (size_t)imax * R);
  L.M = M;
  double fv = 0, z2 = 0, gv = 0;
  if (st == CPMG_OK) st = eval_f(S, L, fs, &fv, &z2);
  S.znorm = std::sqrt(z2);
  if (st == CPMG_OK && g) st = eval_g(S, L, fs, &gv, nullptr);
  if (st == CPMG_OK) {
    if (f) *f = fv;
    if (g) *g = gv;
  }
  dfree(c, M);
  fs_free(c, &fs);
  return st;
}

int cp_als_sweep(cpmg_ctx* c, const cpmg_tensor* Z, int R, double* const* A, int nsweeps, const cpmg_opts* opts,
                 cpmg_result* res) {
  cudaGetLastError();  // an error left pending by the caller is not this call's
  const double t0 = now_s();
  if (!c || !A || nsweeps < 0) return CPMG_INVALID_ARG;
  CPMG_TRY(check_tensor(Z));
  CPMG_TRY(check_opts(opts));
  if (R < 1 || R > CPMG_MAX_RANK) return CPMG_INVALID_ARG;
  Solver S = make_solver(c, opts);
  ZView zv;
  Level L;
  L.s = shape_of(Z);
  L.dtype = Z->dtype;
  FactorSet fs;
  int64_t imax = 1;
  for (int n = 0; n < Z->N; ++n) imax = std::max(imax, Z->dims[n]);
  int st = resolve_tensor(c, Z, &zv);
  L.Z = zv.dev;
  c->prof_Z = L.Z;
  if (st == CPMG_OK) st = fs_alloc(c, &fs, Z->N, R, L.s.dims);
  if (st == CPMG_OK) st = dalloc_t(c, &L.M, (size_t)imax * R);
  if (st == CPMG_OK && opts->dimension_tree && dt_worth(L.s, R))
    st = dalloc_t(c, &L.W, (size_t)L.s.dims[0] * L.s.dims[1] * R);
  if (st == CPMG_OK && opts->dimension_tree && uses_bf16(opts)) st = tc_level_alloc(c, L, R);
  if (st == CPMG_OK) st = dalloc_t(c, &S.sortbuf, fs_doubles(Z->N, R, L.s.dims));
  if (st == CPMG_OK) st = factors_in(c, Z->mem, A, fs);
  double z2 = 0, fv = 0, g = -1, gprev = -1, mn = 0;
  int done = 0;
  bool conv = false;
  GraphCache gc;  // graphs of this call only
  S.gc = &gc;
  S.z0 = L.Z;
  if (st == CPMG_OK) st = tensor_norm(S, L, fs, &S.znorm);
  if (st == CPMG_OK) st = preplan(c, {&L}, R);
  // check_every > 0: exact g every check_every sweeps; check_every < 0: adaptive interval
  int k = opts->check_every > 0 ? opts->check_every : 1;
  while (st == CPMG_OK && done < nsweeps) {
    const bool check = opts->check_every != 0;
    const int kk = check ? std::min(k, nsweeps - done) : 1;
    const std::string key = "als" + std::to_string(kk) + (check ? "+g|" : "|") + (S.refined ? "r" : "f");
    st = graph_run(S, key, [&]() -> int {
      for (int j = 0; j < kk; ++j) CPMG_TRY(als_sweep(S, L, 0, fs));
      if (check) CPMG_TRY(eval_g_launch(S, L, fs));
      return CPMG_OK;
    });
    done += kk;
    if (st == CPMG_OK && check) {
      st = eval_g_read(S, fs.N, &g, &mn);
      if (st != CPMG_OK) break;
      if (g < opts->tol) { conv = true; break; }
      const bool was_refined = S.refined;
      maybe_switch(S, g, mn, gprev);
      if (opts->check_every < 0) k = (S.refined != was_refined) ? 1 : next_check_interval(g, gprev, kk, opts->tol);
      gprev = g;
    }
  }
  if (st == CPMG_OK) st = cudaStreamSynchronize(c->stream) == cudaSuccess ? CPMG_OK : CPMG_CUDA_ERROR;
  S.gc = nullptr;
  profile_collect(c);
  gc.clear();
  if (st == CPMG_OK) st = launch_sort(fs, S.sortbuf, c->stream);
  if (st == CPMG_OK) st = eval_f(S, L, fs, &fv, &z2);
  if (st == CPMG_OK) st = eval_g(S, L, fs, &g, nullptr);
  if (st == CPMG_OK) st = factors_out(c, Z->mem, fs, A);
  if (st == CPMG_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = CPMG_CUDA_ERROR;
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->f = fv;
    res->g = g;
    res->iters_als = done;
    res->levels = 1;
    res->refine_sweeps = S.refine_sweeps;
    res->seconds = now_s() - t0;
  }
  if (st == CPMG_OK && (!std::isfinite(fv) || !std::isfinite(g))) st = CPMG_NUMERIC;
  if (st == CPMG_OK && opts->check_every != 0 && !conv && !(g < opts->tol)) st = CPMG_NOT_CONVERGED;
  if (res) res->status = st;
  dfree(c, L.Wf);
  dfree(c, L.Vf);
  dfree(c, L.AT);
  dfree(c, L.tcs);
  dfree(c, L.W);
  dfree(c, L.M);
  dfree(c, S.sortbuf);
  fs_free(c, &fs);
  dfree(c, zv.own);
  c->prof_Z = nullptr;
  return st;
}

static int setup_cycles(Solver& S, cpmg_hier* h, int* cycles, std::vector<double>* hist) {
  double g_prev = -1.0;
  *cycles = 0;
  for (int cycle = 1; cycle <= S.o.max_setup_cycles; ++cycle) {
    const std::string key = std::string("setup|") + (cycle == 1 ? "1|" : "n|") + (S.refined ? "r" : "f");
    CPMG_TRY(graph_run(S, key, [&]() -> int {
      CPMG_TRY(amg_mult(S, h, 0, cycle == 1, true, true));
      return eval_g_launch(S, h->L[0], h->L[0].A);
    }));
    *cycles = cycle;
    double g = 0, mn = 0;
    CPMG_TRY(eval_g_read(S, h->N, &g, &mn));
    hist->push_back(g);
    if (g < S.o.tol) break;
    if (cycle >= 3 && g > (1.0 - S.o.stag_eps) * g_prev) break;
    maybe_switch(S, g, mn, -1.0);
    g_prev = g;
  }
  return CPMG_OK;
}

static int hier_preplan(cpmg_ctx* c, cpmg_hier* h) {
  std::vector<const Level*> lv;
  for (auto& L : h->L) lv.push_back(&L);
  return preplan(c, lv, h->R);
}

int mg_setup(cpmg_ctx* c, const cpmg_tensor* Z, int R, double* const* A_boot, double* const* A_test,
             const cpmg_opts* opts, cpmg_hier** out, cpmg_result* res) {
  cudaGetLastError();  // an error left pending by the caller is not this call's
  const double t0 = now_s();
  if (!c || !A_boot || !out) return CPMG_INVALID_ARG;
  *out = nullptr;
  CPMG_TRY(check_tensor(Z));
  CPMG_TRY(check_opts(opts));
  if (R < 1 || R > CPMG_MAX_RANK) return CPMG_INVALID_ARG;
  if (opts->n_t > 0 && !A_test) return CPMG_INVALID_ARG;
  Solver S = make_solver(c, opts);
  cpmg_hier* h = nullptr;
  CPMG_TRY(hier_build(c, shape_of(Z), Z->dtype, R, opts, &h));
  ZView zv;
  int st = resolve_tensor(c, Z, &zv);
  Level& L0 = h->L[0];
  L0.Z = zv.dev;
  c->prof_Z = L0.Z;
  S.sortbuf = h->sortbuf;
  if (st == CPMG_OK) st = factors_in(c, Z->mem, A_boot, L0.A);
  for (int t = 0; st == CPMG_OK && t < h->nt; ++t) st = factors_in(c, Z->mem, A_test + (size_t)t * Z->N, L0.tf[t]);
  if (st == CPMG_OK) st = tensor_norm(S, L0, L0.A, &S.znorm);
  S.gc = &h->graphs;
  S.z0 = L0.Z;
  if (st == CPMG_OK) st = hier_preplan(c, h);
  int cycles = 0;
  std::vector<double> hist;
  if (st == CPMG_OK) st = setup_cycles(S, h, &cycles, &hist);
  double fv = 0, g = hist.empty() ? -1 : hist.back();
  if (st == CPMG_OK) st = eval_f(S, L0, L0.A, &fv, nullptr);
  if (st == CPMG_OK) st = factors_out(c, Z->mem, L0.A, A_boot);
  for (int t = 0; st == CPMG_OK && t < h->nt; ++t) st = factors_out(c, Z->mem, L0.tf[t], A_test + (size_t)t * Z->N);
  if (st == CPMG_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = CPMG_CUDA_ERROR;
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->f = fv;
    res->g = g;
    res->iters_setup = cycles;
    res->levels = (int)h->L.size();
    res->refine_sweeps = S.refine_sweeps;
    res->status = st;
    res->seconds = now_s() - t0;
  }
  h->L[0].Z = nullptr;
  dfree(c, zv.own);
  c->prof_Z = nullptr;
  if (st != CPMG_OK) {
    hier_destroy(h);
    return st;
  }
  // remember the mixed-precision state for the solve phase
  h->ttm_tc = S.ttm_tc;
  *out = h;
  return CPMG_OK;
}

static int solve_cycles(Solver& S, cpmg_hier* h, int cycles_done, int* solve, int* restarted, int* als_iters,
                        double* g_out) {
  Level& L0 = h->L[0];
  double g_old = 0, mn = 0;
  CPMG_TRY(graph_run(S, std::string("g|") + (S.refined ? "r" : "f"),
                     [&]() -> int { return eval_g_launch(S, L0, L0.A); }));
  CPMG_TRY(eval_g_read(S, h->N, &g_old, &mn));
  maybe_switch(S, g_old, mn, -1.0);
  *solve = 0;
  *restarted = 0;
  *als_iters = 0;
  while (g_old >= S.o.tol && cycles_done + *solve < S.o.max_cycles) {
    CPMG_TRY(graph_run(S, std::string("fas|") + (S.refined ? "r" : "f"), [&]() -> int {
      CPMG_TRY(fs_copy(h->Aprev, L0.A, S.st));
      CPMG_TRY(cp_fas(S, h, 0, false, 0));
      return eval_g_launch(S, L0, L0.A);
    }));
    *solve += 1;
    double g_new = 0;
    CPMG_TRY(eval_g_read(S, h->N, &g_new, &mn));
    if (*solve > 5 && g_new >= g_old) {
      if (!*restarted) {
        *restarted = 1;
        // discard the new iterate; rebuild the operators by a down-sweep, boot factors frozen
        CPMG_TRY(graph_run(S, std::string("down|") + (S.refined ? "r" : "f"), [&]() -> int {
          CPMG_TRY(fs_copy(L0.A, h->Aprev, S.st));
          return amg_mult(S, h, 0, false, false, false);
        }));
        continue;
      }
      if (S.o.als_fallback) {
        CPMG_TRY(fs_copy(L0.A, h->Aprev, S.st));
        double g = g_old, gp = -1.0;
        int it = 0, k = 1;
        while (it < S.o.max_als_iters && g >= S.o.tol) {
          k = std::min(k, S.o.max_als_iters - it);
          const int kk = k;
          CPMG_TRY(graph_run(S, "als" + std::to_string(kk) + "+g|" + (S.refined ? "r" : "f"), [&]() -> int {
            for (int j = 0; j < kk; ++j) CPMG_TRY(als_sweep(S, L0, 0, L0.A));
            return eval_g_launch(S, L0, L0.A);
          }));
          it += kk;
          gp = g;
          CPMG_TRY(eval_g_read(S, h->N, &g, &mn));
          const bool was_refined = S.refined;
          maybe_switch(S, g, mn, -1.0);
          k = (S.refined != was_refined) ? 1 : next_check_interval(g, gp, kk, S.o.tol);
        }
        CPMG_TRY(launch_sort(L0.A, S.sortbuf, S.st));
        *als_iters = it;
        g_old = g;
        break;
      }
    }
    maybe_switch(S, g_new, mn, g_old);
    g_old = g_new;
  }
  *g_out = g_old;
  return CPMG_OK;
}

int mg_fas_solve(cpmg_ctx* c, cpmg_hier* h, const cpmg_tensor* Z, double* const* A, const cpmg_opts* opts,
                 cpmg_result* res) {
  cudaGetLastError();  // an error left pending by the caller is not this call's
  const double t0 = now_s();
  if (!c || !h || !A) return CPMG_INVALID_ARG;
  CPMG_TRY(check_tensor(Z));
  CPMG_TRY(check_opts(opts));
  if (Z->N != h->N) return CPMG_INVALID_ARG;
  for (int n = 0; n < Z->N; ++n)
    if (Z->dims[n] != h->L[0].s.dims[n] || Z->dtype != h->L[0].dtype) return CPMG_INVALID_ARG;
  Solver S = make_solver(c, opts);
  S.sortbuf = h->sortbuf;
  ZView zv;
  int st = resolve_tensor(c, Z, &zv);
  Level& L0 = h->L[0];
  L0.Z = zv.dev;
  c->prof_Z = L0.Z;
  if (st == CPMG_OK) st = factors_in(c, Z->mem, A, L0.A);
  if (st == CPMG_OK) st = tensor_norm(S, L0, L0.A, &S.znorm);
  S.gc = &h->graphs;
  S.z0 = L0.Z;
  if (st == CPMG_OK) st = hier_preplan(c, h);
  int solve = 0, restarted = 0, als_it = 0;
  double g = -1, fv = 0;
  if (st == CPMG_OK) st = solve_cycles(S, h, 0, &solve, &restarted, &als_it, &g);
  if (st == CPMG_OK) st = eval_f(S, L0, L0.A, &fv, nullptr);
  if (st == CPMG_OK) st = factors_out(c, Z->mem, L0.A, A);
  if (st == CPMG_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = CPMG_CUDA_ERROR;
  if (st == CPMG_OK && !(g < opts->tol)) st = CPMG_NOT_CONVERGED;
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->f = fv;
    res->g = g;
    res->iters_solve = solve;
    res->iters_als = als_it;
    res->restarted = restarted;
    res->levels = (int)h->L.size();
    res->refine_sweeps = S.refine_sweeps;
    res->status = st;
    res->seconds = now_s() - t0;
  }
  L0.Z = nullptr;
  dfree(c, zv.own);
  c->prof_Z = nullptr;
  return st;
}

int mg_fmg(cpmg_ctx* c, cpmg_hier* h, const cpmg_tensor* Z, double* const* A_coarsest, double* const* A, int nu,
           const cpmg_opts* opts, cpmg_result* res) {
  cudaGetLastError();  // an error left pending by the caller is not this call's
  const double t0 = now_s();
  if (!c || !h || !A || !A_coarsest || nu < 0) return CPMG_INVALID_ARG;
  CPMG_TRY(check_tensor(Z));
  CPMG_TRY(check_opts(opts));
  if (Z->N != h->N) return CPMG_INVALID_ARG;
  for (int n = 0; n < Z->N; ++n)
    if (Z->dims[n] != h->L[0].s.dims[n] || Z->dtype != h->L[0].dtype) return CPMG_INVALID_ARG;
  Solver S = make_solver(c, opts);
  S.sortbuf = h->sortbuf;
  ZView zv;
  int st = resolve_tensor(c, Z, &zv);
  Level& L0 = h->L[0];
  L0.Z = zv.dev;
  c->prof_Z = L0.Z;
  if (st == CPMG_OK) st = factors_in(c, Z->mem, A_coarsest, h->L.back().A);
  if (st == CPMG_OK) st = tensor_norm(S, L0, L0.A, &S.znorm);
  S.gc = &h->graphs;
  S.z0 = L0.Z;
  if (st == CPMG_OK) st = hier_preplan(c, h);
  if (st == CPMG_OK) st = fmg_cycle(S, h, nu);
  // the operators are rebuilt around the new factors by a down-sweep (boot factors frozen)
  if (st == CPMG_OK) st = amg_mult(S, h, 0, false, false, false);
  double g = -1, fv = 0;
  if (st == CPMG_OK) st = eval_g(S, L0, L0.A, &g, nullptr);
  if (st == CPMG_OK) st = eval_f(S, L0, L0.A, &fv, nullptr);
  if (st == CPMG_OK) st = factors_out(c, Z->mem, L0.A, A);
  if (st == CPMG_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = CPMG_CUDA_ERROR;
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->f = fv;
    res->g = g;
    res->iters_setup = 1;
    res->levels = (int)h->L.size();
    res->refine_sweeps = S.refine_sweeps;
    res->status = st;
    res->seconds = now_s() - t0;
  }
  L0.Z = nullptr;
  dfree(c, zv.own);
  c->prof_Z = nullptr;
  return st;
}

void cpmg_hier_free(cpmg_hier* h) { hier_destroy(h); }

int cpmg_hier_levels(const cpmg_hier* h) { return h ? (int)h->L.size() : 0; }

int cpmg_hier_level_info(const cpmg_hier* h, int level, int64_t* dims, int* coarsened, void* Y_device,
                         double* const* Rhat_host) {
  if (!h || level < 0 || level >= (int)h->L.size()) return CPMG_INVALID_ARG;
  const Level& L = h->L[level];
  for (int n = 0; n < L.s.N; ++n) {
    if (dims) dims[n] = L.s.dims[n];
    if (coarsened) coarsened[n] = L.co[n] ? 1 : 0;
  }
  cudaStream_t st = h->c->stream;
  if (Y_device) {
    if (!L.Z) return CPMG_INVALID_ARG;  // level 0 keeps no copy of the caller's tensor
    CPMG_CUDA_TRY(cudaMemcpyAsync(Y_device, L.Z, (size_t)L.s.numel() * (L.dtype == CPMG_F64 ? 8 : 4),
                                  cudaMemcpyDeviceToDevice, st));
  }
  if (Rhat_host)
    for (int n = 0; n < L.s.N; ++n)
      if (L.co[n] && Rhat_host[n])
        CPMG_CUDA_TRY(cudaMemcpyAsync(Rhat_host[n], L.Rhat[n], (size_t)L.cd[n] * L.s.dims[n] * sizeof(double),
                                      cudaMemcpyDeviceToHost, st));
  CPMG_CUDA_TRY(cudaStreamSynchronize(st));
  return CPMG_OK;
}

int cpmg_decompose(cpmg_ctx* c, const cpmg_tensor* Z, int R, double* const* A, double* const* A_test,
                   const cpmg_opts* opts, cpmg_result* res) {
  cudaGetLastError();  // an error left pending by the caller is not this call's
  const double t0 = now_s();
  if (!c || !A) return CPMG_INVALID_ARG;
  CPMG_TRY(check_tensor(Z));
  CPMG_TRY(check_opts(opts));
  if (R < 1 || R > CPMG_MAX_RANK) return CPMG_INVALID_ARG;
  if (opts->n_t > 0 && !A_test) return CPMG_INVALID_ARG;
  Solver S = make_solver(c, opts);
  cpmg_hier* h = nullptr;
  CPMG_TRY(hier_build(c, shape_of(Z), Z->dtype, R, opts, &h));
  S.sortbuf = h->sortbuf;
  ZView zv;
  int st = resolve_tensor(c, Z, &zv);
  Level& L0 = h->L[0];
  L0.Z = zv.dev;
  c->prof_Z = L0.Z;
  if (st == CPMG_OK) st = factors_in(c, Z->mem, A, L0.A);
  for (int t = 0; st == CPMG_OK && t < h->nt; ++t) st = factors_in(c, Z->mem, A_test + (size_t)t * Z->N, L0.tf[t]);
  if (st == CPMG_OK) st = tensor_norm(S, L0, L0.A, &S.znorm);
  S.gc = &h->graphs;
  S.z0 = L0.Z;
  if (st == CPMG_OK) st = hier_preplan(c, h);
  int cycles = 0, solve = 0, restarted = 0, als_it = 0;
  std::vector<double> hist;
  double g = -1, fv = 0;
  if (st == CPMG_OK) st = setup_cycles(S, h, &cycles, &hist);
  if (st == CPMG_OK) st = solve_cycles(S, h, cycles, &solve, &restarted, &als_it, &g);
  if (st == CPMG_OK) st = eval_f(S, L0, L0.A, &fv, nullptr);
  if (st == CPMG_OK) st = factors_out(c, Z->mem, L0.A, A);
  if (st == CPMG_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = CPMG_CUDA_ERROR;
  if (st == CPMG_OK && !(g < opts->tol)) st = CPMG_NOT_CONVERGED;
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->f = fv;
    res->g = g;
    res->iters_setup = cycles;
    res->iters_solve = solve;
    res->iters_als = als_it;
    res->restarted = restarted;
    res->levels = (int)h->L.size();
    res->refine_sweeps = S.refine_sweeps;
    res->status = st;
    res->seconds = now_s() - t0;
  }
  L0.Z = nullptr;
  dfree(c, zv.own);
  c->prof_Z = nullptr;
  hier_destroy(h);
  return st;
}

}  // extern "C"
