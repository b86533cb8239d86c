// Fused MTTKRP finish + R x R solve + Gram refresh (see fused.cu).
#pragma once
#include "common.cuh"
#include "dense.cuh"
#include "mttkrp.cuh"

namespace cpmg {

constexpr int kFuseMaxBlocks = 256;

// kind 0: ALS update A^(n) <- M Gamma^+ ; kind 1: `gs_sweeps` Gauss-Seidel sweeps on
// A^(n) Gamma^(n) = M + F from the current A^(n).  M (optional) receives the reduced MTTKRP.
// gscratch: kFuseMaxBlocks * R (R + 1) / 2 doubles; ticket: a device int that starts at zero
// (the kernel returns it to zero).
// normalize: after the update, Eq. ALSnorm on the whole factor set (scales also written after
// the Grams, as launch_normalize does).
int launch_finish_update(const MttkrpPlan& p, const MttkrpScratch& w, const FactorSet& f, int mode, int kind,
                         const double* F, int gs_sweeps, double* M, double* gscratch, int* ticket, int* status,
                         cudaStream_t st, bool normalize = false);

}  // namespace cpmg
