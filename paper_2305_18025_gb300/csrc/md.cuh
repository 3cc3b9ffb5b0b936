// Molecular-dynamics state of a context (see md.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct bpimd_ctx;

namespace bpimd {
struct MDState {
  double *F;          // [N][P][3] total force
  double *F_ex;       // [N][P][3] exchange force
  double *acc;        // per-step energy accumulators
  double *VB;         // device scalar
  uint64_t counter;   // RNG counter (steps taken)
  bool ready;
};
void md_init(MDState *md);
void md_free(MDState *md);
int md_run(bpimd_ctx *ctx, double *pos, double *vel, int32_t nsteps, double *energies);
int evaluate(bpimd_ctx *ctx, const double *pos, double *V_B, double *F);
}  // namespace bpimd
