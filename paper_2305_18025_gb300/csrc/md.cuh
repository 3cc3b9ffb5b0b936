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
  // replica batches
  double *VBr;               // [R] V_B of every replica
  double *c2r;               // [R] thermostat amplitude sqrt((1 - c1^2) kT_r / m)
  int4 *ext_tab;             // (replica, particle block, bead index) of the pair-force pass
  int n_ext;
  int ext_cap;               // entries allocated for ext_tab and ubar_part (the 8-lane table)
  int *ext_first;            // [R+1] first ext_tab entry of each replica
  int *blk_first;            // [R+1] first block-table entry of each replica
};
void md_init(MDState *md);
void md_free(MDState *md);
int md_run(bpimd_ctx *ctx, double *pos, double *vel, int32_t nsteps, double *energies);
int evaluate(bpimd_ctx *ctx, const double *pos, double *V_B, double *F);
int evaluate_batched(bpimd_ctx *ctx, const double *pos, double *V_B, double *F);
int md_run_batched(bpimd_ctx *ctx, double *pos, double *vel, int32_t nsteps, double *energies);
int md_set_pair_tile(bpimd_ctx *ctx, int lanes);
}  // namespace bpimd
