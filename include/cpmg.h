/*
 * cpmg.h — C ABI of libcpmg, a GB300 (sm_103a) implementation of the data-parallel
 * hot path of the adaptive algebraic multigrid method for low-rank canonical (CP)
 * tensor decomposition of De Sterck and Miller.
 *
 * The problem (Eq. CPfunctional): given a dense N-way tensor Z of size
 * I_1 x ... x I_N and a rank R, find factor matrices A^(1..N) (A^(n) is I_n x R)
 * minimizing f = 1/2 || Z - [[A^(1), ..., A^(N)]] ||^2.
 *
 * Conventions used by every call
 * ------------------------------
 *  - Tensors are dense and column-major: element (i_1, ..., i_N) (0-based) sits at
 *    offset i_1 + I_1 (i_2 + I_2 (i_3 + ...)).  This is the order under which the
 *    mode-n matricization of Section 2 (earlier modes fastest) is a plain reshape.
 *  - Factor matrices are float64, column-major I_n x R (element (i, r) at i + I_n r).
 *  - Memory space: `cpmg_tensor.mem` says whether Z, and every factor / TFM array
 *    passed with it in the same call, are device pointers (CPMG_MEM_DEVICE, on the
 *    context's device) or host pointers (CPMG_MEM_HOST; the library copies them to
 *    the device and the results back inside the call).
 *  - Ownership: the caller owns Z, the factor arrays and the TFM arrays.  Z is only
 *    read and must stay valid until the call returns.  The library owns contexts,
 *    hierarchies and all workspace memory (allocated with cudaMalloc on the
 *    context's device; released by cpmg_destroy / cpmg_hier_free).
 *  - Streams: work is issued on the stream given to cpmg_create (or
 *    cpmg_set_stream).  Every call below is synchronous with respect to the host:
 *    it returns after its results are in the caller's buffers.
 *  - Errors: every int-returning call returns a cpmg_status.  No call throws or
 *    aborts; a CUDA error is reported as CPMG_CUDA_ERROR and leaves the context
 *    usable only if the CUDA context itself is still usable.
 *  - Limits: 2 <= N <= CPMG_MAX_MODES, 1 <= R <= CPMG_MAX_RANK, every I_n >= 1.
 *
 * Precision: matricized-tensor-times-Khatri-Rao products (MTTKRP) and the
 * restriction (TTM) read Z in its own type.  Grams, Hadamard products, R x R
 * solves, f and g are always float64.  See cpmg_opts.precision.
 */
#ifndef CPMG_H
#define CPMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPMG_MAX_MODES 8
#define CPMG_MAX_RANK 16
#define CPMG_MAX_TEST_BLOCKS 4

typedef enum {
  CPMG_OK = 0,
  CPMG_INVALID_ARG = 1,    /* bad shape, rank, dtype, pointer or option              */
  CPMG_OUT_OF_BUDGET = 2,  /* the call would exceed the context's HBM budget         */
  CPMG_NOT_CONVERGED = 3,  /* iteration cap reached; outputs hold the last iterate   */
  CPMG_NUMERIC = 4,        /* NaN/Inf met in f, g or the factors                     */
  CPMG_TIMEOUT = 5,        /* a bounded device-side wait expired                     */
  CPMG_CUDA_ERROR = 6,     /* a CUDA runtime call failed                             */
  CPMG_PENDING = 7,        /* server: request not finished yet                       */
  CPMG_CANCELLED = 8,
  CPMG_UNSUPPORTED = 9     /* valid request this build does not handle              */
} cpmg_status;

typedef enum { CPMG_F32 = 0, CPMG_F64 = 1 } cpmg_dtype;
typedef enum { CPMG_MEM_DEVICE = 0, CPMG_MEM_HOST = 1 } cpmg_mem;

/* Arithmetic of the MTTKRP inside relaxation sweeps. */
typedef enum {
  CPMG_PREC_FP32 = 0,   /* float products, float accumulation (fastest; g floor ~1e-7 relative) */
  CPMG_PREC_FP64 = 1,   /* float64 products and accumulation: the plain FP64 path               */
  CPMG_PREC_MIXED = 2,  /* FP32 sweeps, then float64-accurate sweeps once g nears the FP32 floor */
  CPMG_PREC_DF = 3,     /* float64-accurate sweeps from the start (pairs of floats)              */
  CPMG_PREC_BF16X3 = 4, /* split-BF16 MTTKRPs on tcgen05 tensor cores: x = hi + lo in BF16, the
                           products hi*hi + hi*lo + lo*hi accumulated in FP32 (relative error near
                           2^-16 per product); third-order float tensors with I_3 > 6R (the
                           dimension tree's two passes), FP32 sweeps elsewhere                   */
  CPMG_PREC_MIXED_BF16 = 5 /* as MIXED, with split-BF16 sweeps before the switch                  */
} cpmg_precision;

typedef struct cpmg_ctx cpmg_ctx;    /* device, stream, workspaces, statistics            */
typedef struct cpmg_hier cpmg_hier;  /* a multigrid hierarchy: coarse tensors and operators */

typedef struct {
  int N;                             /* number of modes                                      */
  int64_t dims[CPMG_MAX_MODES];      /* I_1..I_N                                             */
  int dtype;                         /* cpmg_dtype                                           */
  int mem;                           /* cpmg_mem of data (and of the factor arrays)          */
  const void* data;                  /* column-major tensor                                  */
} cpmg_tensor;

/* Options.  cpmg_opts_default() fills the paper's parameters (Table tab:params and
 * Section 6.1): setup nu1 = nu2 = 5, nu_c = 100, n_t = 2; solve nu1 = nu2 = 1,
 * nu_c = 50; ten Gauss-Seidel sweeps; tol = 1e-10; at most 500 multilevel cycles,
 * 1e4 ALS iterations and 5 setup cycles; stagnation eps = 0.1. */
typedef struct {
  int precision;                     /* cpmg_precision                                       */
  double tol;                        /* stop when g < tol (Eq. gradConv, Eq. stopcrit)        */
  int max_cycles;                    /* multilevel cycles, setup + solve                      */
  int max_als_iters;
  int nu1_setup, nu2_setup, nuc_setup;
  int nu1, nu2, nuc;
  int n_t;                           /* test blocks (TFMs), <= CPMG_MAX_TEST_BLOCKS           */
  int max_setup_cycles;
  double stag_eps;
  int gs_sweeps;                     /* Gauss-Seidel sweeps in BNGS (Section 5.2)             */
  int64_t coarsest[CPMG_MAX_MODES];  /* I_{n,coarsest}: mode n is coarsened while I_n > this  */
  int als_fallback;                  /* 1: plain ALS after a second solve-phase stagnation    */
                                     /*    (an addition; the paper stops after one rebuild)   */
  double mixed_switch;               /* MIXED: switch to float64-accurate sweeps when
                                        g < mixed_switch * (FP32 floor estimate); <= 0: 4      */
  int check_every;                   /* cp_als_sweep: exact g every k sweeps (0 = never; < 0 =
                                        adaptive interval, at most 32, from the observed rate)  */
  int use_graphs;                    /* 1: capture sweeps / cycles as CUDA graphs and replay
                                        (needs a context stream other than the legacy default) */
  int ttm_tensor_cores;              /* 1: restriction of float tensors on tcgen05 tensor cores
                                        in split BF16 (3 products, FP32 accumulation); 0: FP32
                                        CUDA cores.  The coarse tensors only shape the FAS
                                        corrections, so either keeps the fine-level fixed point */
  int dimension_tree;                /* 1: on third-order levels with I_3 > 6 R, form
                                        W = Z x_3 A^(3)^T in one pass over Z and take the mode-1
                                        and mode-2 MTTKRPs from W (two passes per sweep, two for
                                        all three products at one point, instead of three); the
                                        products are the same sums in another order.  0: one pass
                                        per mode.  Not in the paper (a reuse of partial results). */
} cpmg_opts;

typedef struct {
  double f;                          /* 1/2 ||Z - [[A]]||^2, float64, at the returned factors */
  double g;                          /* Eq. gradConv at the returned factors                   */
  int iters_setup;                   /* setup (CP-AMG-mult) cycles                             */
  int iters_solve;                   /* solve (CP-FAS) cycles                                  */
  int iters_als;                     /* ALS iterations (cp_als_sweep, or the fallback)         */
  int levels;
  int restarted;                     /* solve-phase rebuild happened                           */
  int refine_sweeps;                 /* sweeps done with float64-accurate MTTKRP               */
  int status;
  double seconds;                    /* wall time of the call                                  */
} cpmg_result;

/* ---- context ---------------------------------------------------------------------- */
void cpmg_opts_default(cpmg_opts* opts);

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  hbm_budget_bytes caps the
 * workspace and hierarchy memory the context may allocate (0 = no cap).
 * Returns CPMG_INVALID_ARG for a null out-pointer, CPMG_CUDA_ERROR if the device
 * cannot be selected. */
int cpmg_create(cpmg_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);
void cpmg_destroy(cpmg_ctx* ctx);
int cpmg_set_stream(cpmg_ctx* ctx, void* cuda_stream);
const char* cpmg_status_str(int status);
/* Bytes of device memory the context currently holds. */
size_t cpmg_bytes_in_use(const cpmg_ctx* ctx);

/* ---- kernels exposed for verification (device pointers only) ------------------------ */

/* M = Z_(n) Phi^(n), the MTTKRP of Eq. fineeq1 / Eq. gradEqn with
 * Phi^(n) = A^(N) (.) ... (.) A^(n+1) (.) A^(n-1) (.) ... (.) A^(1) (Eq. Phi).
 * mode is 0-based.  A[m] are device float64 I_m x R; M is a device float64
 * I_n x R output.  precision: CPMG_PREC_FP32, CPMG_PREC_FP64 or CPMG_PREC_DF. */
int cpmg_mttkrp(cpmg_ctx* ctx, const cpmg_tensor* Z, int R, const double* const* A, int mode,
                int precision, double* M);

/* Y = Z x_{n : Rhat[n] != NULL} Rhat^(n), the restriction of Eq. ctensor_transformed applied
 * one mode at a time in increasing n.  Rhat[n] is a device float64 Ic_n x I_n column-major
 * matrix or NULL (mode not coarsened).  Y is a device tensor of Z's dtype with the coarse
 * sizes, column-major.  tensor_cores: 0 = CUDA-core GEMM in Z's type; 1 = tcgen05 tensor cores
 * in split BF16 (x = hi + lo, products hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor
 * memory; relative error near 2^-16 of sum |Rhat||Z|), float Z only, Ic_n <= 256, else
 * CPMG_UNSUPPORTED.  CPMG_TIMEOUT if a bounded device-side wait expired. */
int cpmg_ttm(cpmg_ctx* ctx, const cpmg_tensor* Z, const double* const* Rhat, const int64_t* Ic,
             int tensor_cores, void* Y);

/* Allocation-free MTTKRP (the paper has no counterpart: this exists for callers).
 * Same result and arguments as cpmg_mttkrp, without a context, for callers that cannot
 * allocate device memory (their own allocator already owns the GPU, or they cannot afford
 * the synchronization cudaMalloc/cudaFree may cause).  The kernels' scratch is a fixed
 * array of CPMG_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until the
 * process exits; the call itself allocates nothing.
 *  - Z, A, M: device pointers on the current device (Z->mem must be CPMG_MEM_DEVICE).
 *  - cuda_stream: the cudaStream_t to enqueue on (NULL = legacy default stream).  The call
 *    only enqueues work: M is ready when the stream reaches that point.
 *  - The first call on a device (and the first after the device's primary context was
 *    destroyed and recreated, e.g. by cudaDeviceReset) looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call before any
 *    stream capture.  Later calls in the same context reuse the address.
 *  - All calls share the array: calls whose work overlaps on the GPU (unordered streams)
 *    race and corrupt each other.  Calls ordered on one stream are safe.
 *  - A status word at the start of the array is cleared by each call.  If a bounded
 *    device-side wait of the MTTKRP kernel expires, the kernel raises that word and a last
 *    kernel of the same call overwrites every entry of M with NaN: the call cannot report
 *    the expiry in its return value (it only enqueues work), so a NaN in M is the signal.
 *  - Returns CPMG_OUT_OF_BUDGET when the problem's scratch (per-CTA partial sums and
 *    Khatri-Rao tables, even with the fewest work units) exceeds the array,
 *    CPMG_INVALID_ARG for bad shapes or pointers, CPMG_CUDA_ERROR on a failed CUDA call. */
#define CPMG_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
int cpmg_mttkrp_noalloc(const cpmg_tensor* Z, int R, const double* const* A, int mode, int precision,
                        double* M, void* cuda_stream);

/* f = 1/2 ||Z - [[A]]||^2 (Eq. CPfunctional, element by element in float64) and
 * g (Eq. gradConv, with float64-accurate MTTKRPs).  Either output may be NULL. */
int cpmg_eval_fg(cpmg_ctx* ctx, const cpmg_tensor* Z, int R, const double* const* A,
                 double* f, double* g);

/* ---- the solver calls --------------------------------------------------------------- */

/* ALS (Section 3): up to nsweeps iterations of block nonlinear Gauss-Seidel over modes
 * n = 1..N, each A^(n) <- Z_(n) Phi^(n) (Gamma^(n))^+ with Gamma^(n) the Hadamard product
 * of the other modes' Grams (Eq. Gamma), followed by the normalization of Eq. ALSnorm;
 * the components are sorted by decreasing lambda at the end (end of Section 3).
 * If opts->check_every != 0 the call stops at the first exact check with g < opts->tol.
 * A[0..N-1]: factor arrays, read as the start and overwritten with the result. */
int cp_als_sweep(cpmg_ctx* ctx, const cpmg_tensor* Z, int R, double* const* A, int nsweeps,
                 const cpmg_opts* opts, cpmg_result* result);

/* Setup phase (Section 4.5 Algorithm 1 CP-AMG-mult V-cycles, with the stagnation rule of
 * Eq. stagnation and the cycle cap of Section 6.1).  A_boot: the boot factor matrices
 * (BFMs), in/out.  A_test: n_t * N arrays, block t mode n at A_test[t*N + n], the test
 * factor matrices (TFMs), in/out (the updated fine-level TFMs are returned).  *out
 * receives a new hierarchy (free with cpmg_hier_free). */
int mg_setup(cpmg_ctx* ctx, const cpmg_tensor* Z, int R, double* const* A_boot,
             double* const* A_test, const cpmg_opts* opts, cpmg_hier** out, cpmg_result* result);

/* Solve phase (Section 5.3 Algorithm 2 CP-FAS V-cycles with F = 0 on the finest level)
 * until g < tol or the cycle cap, with the one-time rebuild of Section 6.1 (which uses
 * the hierarchy's stored TFMs) and, if opts->als_fallback, plain ALS after a second
 * stagnation.  A: in/out factors.  Z must be the tensor the hierarchy was built from. */
int mg_fas_solve(cpmg_ctx* ctx, cpmg_hier* hier, const cpmg_tensor* Z, double* const* A,
                 const cpmg_opts* opts, cpmg_result* result);
/* One FMG-CP-FAS cycle (Section 5.4 Algorithm 3) on a hierarchy from mg_setup, as the
 * "Multilevel + FMG" variant of Section 6.1 uses it between the setup and solve phases: nu ALS
 * iterations (normalized, components sorted at the end) on the coarsest level from A_coarsest,
 * then on each finer level the interpolated factors (P-hat times the coarser level's) and one
 * CP-FAS V-cycle with F = 0 topped at that level.  The hierarchy's operators are then rebuilt
 * around the new finest-level factors by one down-sweep of CP-AMG-mult (boot factors frozen, the
 * stored TFMs relaxed and updated), so mg_fas_solve can continue from A.
 * A_coarsest: N float64 column-major arrays of the coarsest level's sizes (cpmg_hier_level_info
 * of level cpmg_hier_levels - 1) x R, the coarsest-level start, read only.  A: N float64 I_n x R
 * column-major arrays, out: the finest-level factors.  Both in Z->mem memory, owned by the
 * caller.  nu >= 0 (the paper's experiments use 100).  result: f and g of A, levels.
 * Errors: INVALID_ARG (null pointers, nu < 0, Z not the hierarchy's tensor), CUDA_ERROR. */
int mg_fmg(cpmg_ctx* ctx, cpmg_hier* hier, const cpmg_tensor* Z, double* const* A_coarsest, double* const* A,
           int nu, const cpmg_opts* opts, cpmg_result* result);
void cpmg_hier_free(cpmg_hier* hier);
int cpmg_hier_levels(const cpmg_hier* hier);
/* Copy level `level`'s tensor dims (and, if Y != NULL, the device tensor itself, in the
 * level's dtype) and its R-hat operators (host float64 column-major arrays, NULL to skip). */
int cpmg_hier_level_info(const cpmg_hier* hier, int level, int64_t* dims, int* coarsened,
                         void* Y_device, double* const* Rhat_host);

/* The "Multilevel" solver of Section 6.1 in one call: mg_setup then mg_fas_solve.
 * Accepts host buffers (Z->mem == CPMG_MEM_HOST): the copies are part of the call. */
int cpmg_decompose(cpmg_ctx* ctx, const cpmg_tensor* Z, int R, double* const* A,
                   double* const* A_test, const cpmg_opts* opts, cpmg_result* result);

/* ---- batched form -------------------------------------------------------------------- */

/* CP-ALS (Section 3: for n = 1..N, A^(n) <- Z_(n) Phi^(n) (Gamma^(n))^+, then Eq. ALSnorm;
 * components sorted by decreasing lambda at the end) on `count` independent tensors at once,
 * each stopping when its g of Eq. gradConv drops below opts->tol or after opts->max_als_iters
 * sweeps.  Z[t]: tensor of order 2..4, float32 or float64, fewer than 2^32 elements;
 * R[t] in 1..8; A[t]: Z[t].N float64 I_n x R column-major factor arrays (initial
 * guess in, result out), owned by the caller and not aliased between tensors.  Memory: all
 * device pointers (Z[t].mem == CPMG_MEM_DEVICE), or, when Z[0].mem == CPMG_MEM_HOST, all host
 * pointers (every Z[t].mem must then be CPMG_MEM_HOST): the call copies every tensor and
 * factor array into one device block, solves there and copies the factors back (pinned host
 * buffers make the copies asynchronous DMA).  opts: precision (FP32 / DF / MIXED / FP64, as
 * for cp_als_sweep), tol, max_als_iters, mixed_switch; check_every > 0 = sweeps per launch and
 * between a tensor's first g evaluations (default 8 when <= 0).  Each tensor then sets its own
 * interval from its observed rate: about half the sweeps the rate predicts are left, a power-of-two
 * multiple of check_every up to 32, back to check_every while g does not fall; so its last
 * evaluation may come up to interval - 1 sweeps after g first fell below tol.  All sweeps of all tensors run in one cooperative persistent
 * kernel per check interval; each tensor's arithmetic does not depend on the rest of the batch,
 * so a tensor's factors are bitwise the same alone and in any batch.  The unit size is chosen by
 * timing candidates on the first call for a batch size class (cached in the context).
 * results[t] gets f (from the Gram identity 1/2(||Z||^2 - 2<M, A> + sum Hadamard of Grams),
 * float64), g, iters_als and status.  Returns CPMG_OK when every tensor converged, else the
 * first non-OK status among them (or the call's own error). */
int cpmg_batch_solve(cpmg_ctx* ctx, int count, const cpmg_tensor* Z, const int* R, double* const* const* A,
                     const cpmg_opts* opts, cpmg_result* results);

/* Host-only inspection of the batched form's work split (no GPU needed): the MTTKRP work units
 * of mode `mode` of one tensor (order N, sizes dims, rank R) at unit size unit_elements.  A unit
 * covers first-mode rows 64*rb .. 64*rb+63 (clipped) and columns c0..c1-1 of the mode's column
 * range: all columns of the mode-1 unfolding for mode 0; for mode n > 0 the columns that share
 * i_n = in_idx.  It writes its partial sums to slot k (per column chunk for mode 0; per i_n and
 * (chunk, row block) otherwise).  units: max_units x 5 int64 (rb, k, c0, c1, in_idx), may be
 * NULL when max_units = 0; *n_units receives the full count.  *nk: slots per output row (mode
 * > 0) or column chunks (mode 0); *partial_doubles: the partial-sum storage of all modes.
 * INVALID_ARG for N outside 2..4, R outside 1..8, a size < 1, 2^32 or more elements,
 * unit_elements < 1, or mode >= N. */
int cpmg_batch_plan(int N, const int64_t* dims, int R, int64_t unit_elements, int mode, int64_t* units,
                    int64_t max_units, int64_t* n_units, int* nk, int64_t* partial_doubles);

/* Failure-detection test hook of the batched form (the paper has no counterpart).  Every grid
 * barrier of the batched kernel is a bounded wait: after wait_limit_s seconds (default 2; here
 * 0 < wait_limit_s <= 60) the waiting CTAs give up, the kernel records the expiry and returns, and
 * cpmg_batch_solve returns CPMG_TIMEOUT with the context still usable.  unreachable_barrier != 0
 * makes the first barrier of every launch wait for one CTA more than the launch has, so that wait
 * always runs out: a test can see the timeout path without faulting or hanging the GPU.  Set it
 * back to 0 for normal work.  Applies to cpmg_batch_solve calls made after it. */
int cpmg_debug_config(cpmg_ctx* ctx, double wait_limit_s, int unreachable_barrier);

/* ---- served form ---------------------------------------------------------------------- */
/* A request server with continuous batching on the context.  Submitted CP-ALS problems (the
 * same problem statement as cpmg_batch_solve) queue in arrival order; a worker thread admits
 * them into the running batch while the HBM they hold (tensor, factors, MTTKRP partials and
 * Grams) fits the server's budget and fewer than max_active run; it runs sweeps_per_launch
 * sweeps of every running request per launch of the batched kernel, evaluates g, and retires
 * finished requests between launches, so requests join and leave while others are on the GPU.
 * A request's arithmetic does not depend on the other requests (same unit sizes, same sweep
 * counts between checks), so its result is bitwise the same alone and in the mix.
 * Once serving, the context accepts only server calls (other solver calls are not thread-safe
 * with the worker).  Z and A must stay valid until the request is polled as done. */

/* hbm_budget_bytes: admission cap (0 = none); max_active (<= 0: keep, default 1024);
 * sweeps_per_launch (<= 0: keep, default 8); unit_elements: fixed MTTKRP unit size for every
 * request (0: autotuned per shape class and cached in the context). */
int cpmg_server_config(cpmg_ctx* ctx, size_t hbm_budget_bytes, int max_active, int sweeps_per_launch,
                       int64_t unit_elements);
/* Queue a request; *ticket identifies it.  CPMG_OUT_OF_BUDGET if it alone exceeds the budget. */
int cpmg_server_submit(cpmg_ctx* ctx, const cpmg_tensor* Z, int R, double* const* A, const cpmg_opts* opts,
                       uint64_t* ticket);
/* Queue a request for the "Multilevel" driver of Section 6.1 (the same solve as cpmg_decompose:
 * setup cycles of Algorithm 1, then CP-FAS cycles of Algorithm 2) instead of batched ALS.  It runs
 * on one of the server's multilevel workers, each with a context and stream of its own, so its
 * launches overlap the batched requests'; its hierarchy (coarse tensors, operators, factor sets)
 * is held on the device from its start to its end and counted against the server's HBM budget.
 * Z: device tensor of order 2..CPMG_MAX_MODES; A: N device float64 I_n x R arrays (start in,
 * result out); A_test: opts->n_t x N device arrays (the test factor matrices, as for
 * cpmg_decompose), read only.  Z, A and A_test must stay valid until polled as done.  Its result
 * does not depend on the other requests.  A running multilevel request is not cancelled (it is
 * one solver call); a queued one is.  Same statuses as cpmg_server_submit. */
int cpmg_server_submit_multilevel(cpmg_ctx* ctx, const cpmg_tensor* Z, int R, double* const* A,
                                  double* const* A_test, const cpmg_opts* opts, uint64_t* ticket);
/* CPMG_PENDING while queued or running; CPMG_OK once done, with *result (seconds = latency
 * from submission); the ticket is then released.  CPMG_INVALID_ARG for an unknown ticket. */
int cpmg_server_poll(cpmg_ctx* ctx, uint64_t ticket, cpmg_result* result);
/* Cancel a request.  Queued: it leaves the queue at once and its factors are not touched.  Running:
 * the worker retires it after the launch in flight; its factors hold the last iterate (sorted) and
 * result f/g are those of that iterate.  Either way the next poll returns CPMG_OK with
 * result->status = CPMG_CANCELLED (or the request's own status if it finished first).  A finished
 * request is left as it is.  CPMG_INVALID_ARG for an unknown (or already polled) ticket. */
int cpmg_server_cancel(cpmg_ctx* ctx, uint64_t ticket);
/* Block until no request is queued or running (CPMG_PENDING after timeout_s seconds). */
int cpmg_server_wait(cpmg_ctx* ctx, double timeout_s);
/* Latency percentiles (submission to completion) and throughput (completions per second since
 * the first submission) over every completed request. */
int cpmg_server_stats(cpmg_ctx* ctx, double* p50_s, double* p99_s, double* req_per_s, int64_t* completed);

/* Per-kernel timing: when enabled, each launch of the finest-level MTTKRP main kernel is
 * bracketed by CUDA events on the context's stream; the statistics accumulate until reset.
 * kind: 0 = FP32 launches, 1 = float64-accurate (pairs of floats), 2 = FP64.  bytes_per_launch
 * is the algorithmic traffic: sizeof(z) * prod(I) + 4 R sum_n I_n.  kind 3 = the tensor-core
 * mode products of the restriction (finest level in the solvers, every one in cpmg_ttm), with
 * bytes_per_launch = 4 (numel in + numel out).  kind 4 = the launches of the batched kernel in
 * cpmg_batch_solve, with bytes_per_launch the mean over launches of: for every tensor active at
 * the launch, sizeof(z) * prod(I) per MTTKRP pass (N per sweep, N for the g evaluation) plus
 * 16 R sum_n I_n per sweep (float64 factors read and written).  kind 5 = the split-BF16
 * tensor-core passes over the finest-level tensor (CPMG_PREC_BF16X3 / MIXED_BF16), with
 * bytes_per_launch = 4 numel + 4 x the product's size. */
int cpmg_profile_enable(cpmg_ctx* ctx, int enable);
int cpmg_profile_read(cpmg_ctx* ctx, int kind, double* total_ms, int64_t* launches,
                      double* bytes_per_launch);
int cpmg_profile_reset(cpmg_ctx* ctx);
/* Number of kernel launches issued by this context since creation (all kinds). */
int64_t cpmg_launch_count(const cpmg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* CPMG_H */
