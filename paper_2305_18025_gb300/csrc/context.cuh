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
  double *d_Vf, *d_Vb;         // diagnostic potentials (bpimd_get_potentials)
  bool evaluated;
  bpimd::MDState md;
  // stage profiling
  bool prof_on;
  int prof_max;
  std::vector<cudaEvent_t> prof_events;  // (BPIMD_NUM_STAGES + 1) per evaluation
  int prof_count;
};
