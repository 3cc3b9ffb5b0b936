// Molecular dynamics step (placeholder until the integrator lands).
#include "md.cuh"
#include "bpimd_internal.cuh"

namespace bpimd {
void md_init(MDState *md) { *md = MDState{}; }
void md_free(MDState *md) {
  cudaFree(md->F); cudaFree(md->F_ex); cudaFree(md->acc); cudaFree(md->VB);
  *md = MDState{};
}
int md_run(bpimd_ctx *, double *, double *, int32_t, double *) { return BPIMD_ERR_STATE; }
}  // namespace bpimd
