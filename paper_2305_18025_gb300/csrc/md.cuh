// Molecular-dynamics state of a context (see md.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pairs.cuh"

struct bpimd_ctx;

namespace bpimd {
struct MDState {
  double *F;                 // [N][P][3] total force of the current positions
  double *VB;                // device scalar: V^{[1,N]} of the last evaluation
  double *ubar_part;         // per-block U-bar partial sums of the last force pass
  double *ke_part;           // per-block kinetic-energy partial sums
  double *spring_part;       // per-block expected exterior-spring energies
  unsigned long long *step;  // device step counter (thermostat noise counter)
  int ext_blocks, ke_blocks, spring_blocks;
  cudaGraph_t graph;         // one captured step
  cudaGraphExec_t exec;
  double *g_pos, *g_vel;     // buffers the captured step is bound to
  uint64_t steps_taken;
  void *cell_block;          // cell-list buffers (Lennard-Jones in a box)
  CellList cells;
  bool ready;
};
void md_init(MDState *md);
void md_free(MDState *md);
int md_run(bpimd_ctx *ctx, double *pos, double *vel, int32_t nsteps, double *energies);
int evaluate(bpimd_ctx *ctx, const double *pos, double *V_B, double *F);
}  // namespace bpimd
