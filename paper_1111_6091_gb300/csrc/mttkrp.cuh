// MTTKRP: M = Z_(n) Phi^(n) (Eq. fineeq1, Eq. Phi) for a dense column-major tensor.
#pragma once
#include "common.cuh"

namespace cpmg {

// P_BF16 (split BF16 on tensor cores) is the engine's, never a plan's: the MTTKRP kernels here run
// P_FP32 in its place.
enum Prec { P_FP32 = 0, P_FP64 = 1, P_DF = 3, P_BF16 = 4 };

// Launch geometry and table layout for one (shape, mode, precision).
struct MttkrpPlan {
  int mode = 0;
  int prec = P_FP32;
  int zdtype = CPMG_F32;
  int R = 0, RP = 0, TS = 0;   // rank, padded rank, table row stride (elements)
  int VW = 1;                  // rows per thread per column
  int TX = 0, TY = 0;          // threads along rows, column groups per CTA
  int64_t I1 = 0;              // contiguous (first) mode size
  int64_t SEG = 0;             // rows covered by one CTA (TX*VW)
  int nseg = 1;
  int64_t In = 1;              // output rows for mode > 0 (1 for mode 0)
  int64_t Lp = 1, G = 1;       // inner / outer column counts (Kin rows, Kout rows)
  int C = 1;                   // chunks per (i_n, segment)
  int64_t nunits = 0;
  bool has_in = false, has_out = false;
  int in_modes[kMaxModes], n_in = 0;     // modes whose KR product forms Kin
  int out_modes[kMaxModes], n_out = 0;   // modes whose KR product forms Kout
  // shared-memory staging by bulk copies (TMA): eligibility and ring geometry
  bool use_tma = false;
  int CPS = 1, S = 2;          // columns per group per stage, stages
  int64_t ROWS = 0;            // rows per column held in a stage
  bool contiguous = false;     // a stage is one contiguous byte range
  uint32_t stage_stride = 0, w_off = 0, w_stride = 0, bar_off = 0, col_off = 0, stage_off = 0, red_off = 0;
  size_t smem_tma = 0;
  bool tab_smem = false;       // Khatri-Rao tables staged into shared memory
  uint32_t tab_off = 0;
  int nw = 1;                  // per-unit partials (consumer warps of the TMA kernel, mode > 0)
  int64_t grid = 0;            // CTAs launched (persistent over unit ranges for mode > 0)
  size_t table_bytes = 0;      // bytes of one table element (4, 8 or 8 for float2)
  size_t part_elem = 0;        // bytes of one partial entry
  size_t partial_bytes() const;
  size_t tables_bytes() const;  // A1 + Kin + Kout
};

// Launch-shape limits for mttkrp_plan (0 = the planner's own choice).
struct MttkrpLimits {
  int cps = 0;   // columns per column group per stage of the bulk-copy kernel
  int ty = 0;    // column groups per CTA
};

// allow_tma = false forces the register-load kernel (smaller scratch: no full row table).
int mttkrp_plan(const Shape& s, int mode, int R, int prec, int zdtype, const void* Z, int num_sms,
                MttkrpPlan* p, bool allow_tma = true, const MttkrpLimits* lim = nullptr);

// Device buffers the MTTKRP needs besides Z and the factors.
struct MttkrpScratch {
  void* tables = nullptr;      // A1 | Kin | Kout in the precision's table type
  void* partial = nullptr;
};

// Builds the tables from the float64 factors (device pointer array), runs the main
// kernel and the ordered reduction into M (float64, I_n x R column-major).
int mttkrp_run(const MttkrpPlan& p, const Shape& s, const void* Z, const double* const* A_dev_ptrs,
               const MttkrpScratch& w, double* M, cudaStream_t st, cudaEvent_t ev0 = nullptr,
               cudaEvent_t ev1 = nullptr, int* err = nullptr, bool finish = true, bool ev_external = false);

}  // namespace cpmg
