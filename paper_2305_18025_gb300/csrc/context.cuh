// The context behind the opaque bpimd_ctx handle of the C ABI (internal).
#pragma once
#include <vector>

#include "bpimd_internal.cuh"
#include "md.cuh"

struct bpimd_ctx {
  bpimd_config cfg;
  cudaStream_t stream;
  bpimd::Workspace w;
  void *dev_block;     // single device allocation holding the workspace
  size_t dev_bytes;
  int *host_status;    // pinned
  double *d_pos, *d_F, *d_VB;  // staging for the _host entry point (lazy)
  // _host entry point with pinned buffers on a non-default stream: the whole
  // call (copies in, evaluation, copies out, status) as one CUDA graph,
  // captured for one (positions, forces) pair and replayed
  cudaGraph_t host_graph;
  cudaGraphExec_t host_exec;
  const void *hg_pos;
  void *hg_F;
  double *h_VB;      // pinned: V_B of the last replay
  int *h_status;     // pinned: status word of the last replay
  double *d_Vf, *d_Vb;         // diagnostic potentials (bpimd_get_potentials)
  bool evaluated;
  bpimd::MDState md;
  // stage profiling
  bool prof_on;
  int prof_max;
  std::vector<cudaEvent_t> prof_events;  // (BPIMD_NUM_STAGES + 1) per evaluation
  int prof_count;
  // replica batch (bpimd_create_batched); R == 0 for a single-system context
  int R;
  int maxN;
  long long total_elems;                  // 3 * sum_r N_r P_r
  std::vector<bpimd::Workspace> h_ws;     // per-replica workspaces (host copy)
  std::vector<long long> h_off;           // element offset of each replica
  bpimd::Workspace *d_ws;                 // device copies of h_ws
  int2 *d_bead_tab, *d_blk_tab;           // (replica, particle block), (replica, g block)
  int n_bead_tab, n_blk_tab;
  int *d_order;                           // replicas by decreasing N
  std::vector<int> h_order;               // the same order on the host
  int n_big;                              // replicas above BATCH_MAX_N (first in the order)
  long long *d_off;
  int tune_gmat_bpsm, tune_prob_bpsm;     // grid caps (blocks per SM) of the batched passes
  int pair_lanes;                         // lanes per particle of the batched pair forces (2, 4 or 8)
};
