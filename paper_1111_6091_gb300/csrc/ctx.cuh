// Context services shared by the host sources of libcpmg (defined in engine.cu).
#pragma once
#include "common.cuh"

struct cpmg_ctx;

namespace cpmg {

// Device allocation through the context (counted against its HBM budget).
int ctx_alloc(cpmg_ctx* c, void** p, size_t bytes);
void ctx_free(cpmg_ctx* c, void* p);
cudaStream_t ctx_stream(const cpmg_ctx* c);
int ctx_device(const cpmg_ctx* c);
int ctx_sms(const cpmg_ctx* c);
size_t ctx_budget(const cpmg_ctx* c);
size_t ctx_in_use(const cpmg_ctx* c);
void ctx_add_launches(cpmg_ctx* c, int64_t n);
// Timing events for one launch of profiling kind `kind` (cpmg_profile_read) with `bytes` of
// algorithmic traffic; both null when profiling is off.  Record e0 before and e1 after the launch
// on the context's stream; the pair is read back by cpmg_profile_read.
int ctx_profile_events(cpmg_ctx* c, int kind, double bytes, cudaEvent_t* e0, cudaEvent_t* e1);

// Per-context state of the batched solver and the request server (batch.cu).
struct BatchState;
BatchState*& ctx_batch_state(cpmg_ctx* c);
void batch_state_destroy(cpmg_ctx* c);

}  // namespace cpmg
