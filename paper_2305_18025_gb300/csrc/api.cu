// C ABI of the bpimd library: argument checks, workspace ownership, launch
// sequence of one evaluation of Algorithm 1 (appendix "Algorithm Pseudocode").
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "context.cuh"

using namespace bpimd;


namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int validate(const bpimd_config *c) {
  if (!c) return BPIMD_ERR_ARG;
  if (c->N < 1 || c->P < 2) return BPIMD_ERR_ARG;
  if (c->N > CHAIN_MAX_N) return BPIMD_ERR_ARG;
  if ((long long)c->N * c->P > (1LL << 31) / 3) return BPIMD_ERR_ARG;
  if (!finite_pos(c->m) || !finite_pos(c->omega_P) || !finite_pos(c->beta)) return BPIMD_ERR_ARG;
  if (!valid_precision(c->precision)) return BPIMD_ERR_ARG;
  if (c->flags & ~(BPIMD_FLAG_RECOMPUTE | BPIMD_FLAG_TEST_TIMEOUT)) return BPIMD_ERR_ARG;
  if (!(c->box_L >= 0.0) || !std::isfinite(c->box_L)) return BPIMD_ERR_ARG;
  return BPIMD_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int cuda_status(cudaError_t e) { return e == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA; }

int check_ptr(const void *p) {
  if (!p) return BPIMD_ERR_ARG;
  if (((uintptr_t)p) & 15) return BPIMD_ERR_ARG;
  return BPIMD_OK;
}

bool is_pinned(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

int read_status(bpimd_ctx *ctx) {
  cudaError_t e = cudaMemcpyAsync(ctx->host_status, ctx->w.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return BPIMD_ERR_CUDA;
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return BPIMD_ERR_CUDA;
  const int st = *ctx->host_status;
  if (st) {
    e = cudaMemsetAsync(ctx->w.status, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return BPIMD_ERR_CUDA;
    if (st & ST_TIMEOUT) return BPIMD_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return BPIMD_ERR_NONFINITE;
  }
  return BPIMD_OK;
}

}  // namespace

namespace bpimd {

size_t layout_workspace(Workspace &w, char *base) {
  const size_t N = w.N, NB = w.NB, NT = w.NT, gelems = NB * TILE2;
  const size_t gm_bytes = (w.mixed ? sizeof(float) : sizeof(double)) * gelems;
  const bool tables = !w.recomp;  // recompute mode: nothing O(N^2)
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    char *p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  w.R1 = (double *)take(sizeof(double) * 4 * N);
  w.RP = (double *)take(sizeof(double) * 4 * N);
  w.R1s = (float *)take(sizeof(float) * 8 * N);
  w.RPs = (float *)take(sizeof(float) * 8 * N);
  w.Eint = (double *)take(sizeof(double) * N);
  w.link = (double *)take(sizeof(double) * N);
  w.ccm = (double *)take(sizeof(double) * N);
  w.cce = (int *)take(sizeof(int) * N);
  w.nexp = (int *)take(sizeof(int) * N);
  w.Ap = (double *)take(sizeof(double) * N);
  w.C = (double *)take(sizeof(double) * (N + 1));
  w.gm = tables ? (void *)take(gm_bytes) : nullptr;
  w.ge = tables ? (int *)take(sizeof(int) * gelems) : nullptr;
  w.gbm = tables ? (void *)take(gm_bytes) : nullptr;
  w.gbe = tables ? (int *)take(sizeof(int) * gelems) : nullptr;
  w.yfm = (double *)take(sizeof(double) * (N + 1));
  w.yfe = (int *)take(sizeof(int) * (N + 1));
  w.ybm = (double *)take(sizeof(double) * (N + 1));
  w.ybe = (int *)take(sizeof(int) * (N + 1));
  w.alm = (void *)take(sizeof(double) * N);
  w.ale = (int *)take(sizeof(int) * N);
  w.scal = (double *)take(sizeof(double) * 4);
  w.scal_i = (int *)take(sizeof(int) * 4);
  w.rowpart = tables ? (double *)take(sizeof(double) * NB * TILE * 4) : nullptr;
  w.colpart = tables ? (double *)take(sizeof(double) * NB * TILE * 4) : nullptr;
  w.rowcnt = tables ? (int *)take(sizeof(int) * NT) : nullptr;
  w.colcnt = tables ? (int *)take(sizeof(int) * NT) : nullptr;
  w.status = (int *)take(sizeof(int) * 4);
  w.bk = w.blocks ? (unsigned long long *)take(sizeof(unsigned long long) * 4 * NT * TILE2) : nullptr;
  w.be = w.blocks ? (int *)take(sizeof(int) * 4 * NT * TILE2) : nullptr;
  return off;
}

// one evaluation of V_B and forces on ctx->stream
int evaluate(bpimd_ctx *ctx, const double *pos, double *V_B, double *F) {
  const Workspace &w = ctx->w;
  cudaStream_t s = ctx->stream;
  cudaEvent_t *ev = nullptr;
  if (ctx->prof_on && ctx->prof_count < ctx->prof_max)
    ev = &ctx->prof_events[(size_t)ctx->prof_count++ * (BPIMD_NUM_STAGES + 1)];
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  mark(0);
  if (launch_prep(w, pos, F, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  mark(1);
  if (launch_chains(w, V_B, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  mark(2);
  if (launch_prob_forces(w, pos, F, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  mark(3);
  ctx->evaluated = true;
  return BPIMD_OK;
}

// The host-buffer call as one replayed CUDA graph (pinned buffers, non-default
// stream): the copies in and out, the three evaluation kernels, and the copies
// of V_B and the status word into pinned context scalars.  Captured once per
// (positions, forces) pair; the staging buffers must exist.  Returns
// BPIMD_ERR_STATE when the graph cannot be built (the caller then takes the
// direct path), else the call's status.
int host_call_graph(bpimd_ctx *ctx, const double *positions, double *forces, size_t bytes) {
  cudaStream_t s = ctx->stream;
  if (!ctx->h_VB && (cudaMallocHost(&ctx->h_VB, sizeof(double)) != cudaSuccess ||
                     cudaMallocHost(&ctx->h_status, sizeof(int)) != cudaSuccess)) {
    cudaGetLastError();
    return BPIMD_ERR_STATE;
  }
  if (!ctx->host_exec || ctx->hg_pos != positions || ctx->hg_F != forces) {
    if (ctx->host_exec) { cudaGraphExecDestroy(ctx->host_exec); ctx->host_exec = nullptr; }
    if (ctx->host_graph) { cudaGraphDestroy(ctx->host_graph); ctx->host_graph = nullptr; }
    if (prepare_chains() != cudaSuccess) return BPIMD_ERR_STATE;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return BPIMD_ERR_STATE;
    }
    bool ok = cudaMemcpyAsync(ctx->d_pos, positions, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              evaluate(ctx, ctx->d_pos, ctx->d_VB, ctx->d_F) == BPIMD_OK &&
              cudaMemcpyAsync(forces, ctx->d_F, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
              cudaMemcpyAsync(ctx->h_VB, ctx->d_VB, sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
              cudaMemcpyAsync(ctx->h_status, ctx->w.status, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    cudaGraph_t g = nullptr;
    ok = (cudaStreamEndCapture(s, &g) == cudaSuccess) && ok && g;
    if (ok && cudaGraphInstantiate(&ctx->host_exec, g, 0) != cudaSuccess) {
      ctx->host_exec = nullptr;
      ok = false;
    }
    if (!ok) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return BPIMD_ERR_STATE;
    }
    ctx->host_graph = g;
    ctx->hg_pos = positions;
    ctx->hg_F = forces;
  }
  if (cudaGraphLaunch(ctx->host_exec, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return BPIMD_ERR_CUDA;
  ctx->evaluated = true;
  const int st = *ctx->h_status;
  if (st) {
    if (cudaMemsetAsync(ctx->w.status, 0, sizeof(int), s) != cudaSuccess) return BPIMD_ERR_CUDA;
    if (st & ST_TIMEOUT) return BPIMD_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return BPIMD_ERR_NONFINITE;
  }
  return BPIMD_OK;
}
}  // namespace bpimd

extern "C" {

int bpimd_create(bpimd_ctx **out, const bpimd_config *cfg, void *cuda_stream) {
  if (!out) return BPIMD_ERR_ARG;
  *out = nullptr;
  int rc = validate(cfg);
  if (rc != BPIMD_OK) return rc;
  bpimd_ctx *ctx = new (std::nothrow) bpimd_ctx();
  if (!ctx) return BPIMD_ERR_NOMEM;
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)cuda_stream;
  Workspace &w = ctx->w;
  w.N = cfg->N;
  w.P = cfg->P;
  w.inv_P = 1.0 / cfg->P;
  w.NT = (w.N + TILE - 1) / TILE;
  w.NB = w.NT * (w.NT + 1) / 2;
  set_precision(w, cfg->precision);
  w.m = cfg->m;
  w.omega_P = cfg->omega_P;
  w.beta = cfg->beta;
  w.k = cfg->m * cfg->omega_P * cfg->omega_P;
  w.half_k = 0.5 * w.k;
  w.cx = w.beta * w.half_k * LOG2E;
  w.recomp = (cfg->flags & BPIMD_FLAG_RECOMPUTE) || cfg->N > BPIMD_STORE_MAX_N;
  w.test_timeout = (cfg->flags & BPIMD_FLAG_TEST_TIMEOUT) != 0;
  w.blocks = 1;
  set_box(w, cfg->box_L);
  const size_t N = w.N;
  // one allocation: the workspace, then the diagnostic potentials
  const size_t wbytes = layout_workspace(w, nullptr);
  const size_t off = wbytes + 2 * align_up(sizeof(double) * (N + 1));
  ctx->dev_bytes = off;
  if (cudaMalloc(&ctx->dev_block, off) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return BPIMD_ERR_NOMEM;
  }
  char *b = (char *)ctx->dev_block;
  layout_workspace(w, b);
  ctx->d_Vf = (double *)(b + wbytes);
  ctx->d_Vb = (double *)(b + wbytes + align_up(sizeof(double) * (N + 1)));
  if (cudaMemsetAsync(ctx->dev_block, 0, off, ctx->stream) != cudaSuccess ||
      (!w.recomp && launch_gmat_padding(w, ctx->stream) != cudaSuccess) ||
      cudaMallocHost(&ctx->host_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->dev_block);
    delete ctx;
    return BPIMD_ERR_NOMEM;
  }
  *ctx->host_status = 0;
  md_init(&ctx->md);
  *out = ctx;
  return BPIMD_OK;
}

int bpimd_destroy(bpimd_ctx *ctx) {
  if (!ctx) return BPIMD_OK;
  cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->prof_events) cudaEventDestroy(e);
  md_free(&ctx->md);
  cudaFree(ctx->dev_block);
  cudaFree(ctx->d_pos);
  cudaFree(ctx->d_F);
  cudaFree(ctx->d_VB);
  if (ctx->host_exec) cudaGraphExecDestroy(ctx->host_exec);
  if (ctx->host_graph) cudaGraphDestroy(ctx->host_graph);
  if (ctx->h_VB) cudaFreeHost(ctx->h_VB);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  cudaFreeHost(ctx->host_status);
  delete ctx;
  return BPIMD_OK;
}

int bpimd_exchange_energy_forces(bpimd_ctx *ctx, const double *positions, double *V_B, double *forces) {
  if (!ctx) return BPIMD_ERR_ARG;
  if (ctx->R) return BPIMD_ERR_STATE;
  int rc;
  if ((rc = check_ptr(positions)) || (rc = check_ptr(forces))) return rc;
  if (V_B && (((uintptr_t)V_B) & 7)) return BPIMD_ERR_ARG;
  return evaluate(ctx, positions, V_B, forces);
}

int bpimd_exchange_energy_forces_host(bpimd_ctx *ctx, const double *positions, double *V_B, double *forces) {
  if (!ctx || !positions || !forces) return BPIMD_ERR_ARG;
  if (ctx->R) return BPIMD_ERR_STATE;
  const size_t bytes = sizeof(double) * 3 * (size_t)ctx->w.N * ctx->w.P;
  if (!ctx->d_pos) {
    if (cudaMalloc(&ctx->d_pos, bytes) != cudaSuccess || cudaMalloc(&ctx->d_F, bytes) != cudaSuccess ||
        cudaMalloc(&ctx->d_VB, sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return BPIMD_ERR_NOMEM;
    }
  }
  cudaStream_t s = ctx->stream;
  if (s != nullptr && !ctx->prof_on && is_pinned(positions) && is_pinned(forces)) {
    int rc = host_call_graph(ctx, positions, forces, bytes);
    if (rc != BPIMD_ERR_STATE) {  // BPIMD_ERR_STATE: the graph could not be built; take the direct path
      if (rc == BPIMD_OK && V_B) *V_B = *ctx->h_VB;
      return rc;
    }
  }
  if (cudaMemcpyAsync(ctx->d_pos, positions, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  int rc = evaluate(ctx, ctx->d_pos, ctx->d_VB, ctx->d_F);
  if (rc != BPIMD_OK) return rc;
  if (cudaMemcpyAsync(forces, ctx->d_F, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (V_B && cudaMemcpyAsync(V_B, ctx->d_VB, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return BPIMD_ERR_CUDA;
  return read_status(ctx);
}

int bpimd_sync(bpimd_ctx *ctx) {
  if (!ctx) return BPIMD_ERR_ARG;
  return read_status(ctx);
}

int bpimd_get_potentials(bpimd_ctx *ctx, double *V_fwd, double *V_bwd, double *Eint) {
  if (!ctx) return BPIMD_ERR_ARG;
  if (ctx->R) return BPIMD_ERR_STATE;
  if (!ctx->evaluated) return BPIMD_ERR_STATE;
  const size_t N = ctx->w.N;
  cudaStream_t s = ctx->stream;
  if (launch_diag_potentials(ctx->w, ctx->d_Vf, ctx->d_Vb, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (V_fwd && cudaMemcpyAsync(V_fwd, ctx->d_Vf, sizeof(double) * (N + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return BPIMD_ERR_CUDA;
  if (V_bwd && cudaMemcpyAsync(V_bwd, ctx->d_Vb, sizeof(double) * (N + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return BPIMD_ERR_CUDA;
  if (Eint && cudaMemcpyAsync(Eint, ctx->w.Eint, sizeof(double) * N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return BPIMD_ERR_CUDA;
  return read_status(ctx);
}

int bpimd_connection_probabilities(bpimd_ctx *ctx, double *M) {
  if (!ctx) return BPIMD_ERR_ARG;
  if (ctx->R) return BPIMD_ERR_STATE;
  int rc;
  if ((rc = check_ptr(M))) return rc;
  if (!ctx->evaluated) return BPIMD_ERR_STATE;
  return cuda_status(launch_dense_probabilities(ctx->w, M, ctx->stream));
}

int bpimd_step(bpimd_ctx *ctx, double *positions, double *velocities, int32_t nsteps, double *energies) {
  if (!ctx || nsteps < 0) return BPIMD_ERR_ARG;
  int rc;
  if ((rc = check_ptr(positions)) || (rc = check_ptr(velocities))) return rc;
  if (energies && (((uintptr_t)energies) & 7)) return BPIMD_ERR_ARG;
  rc = ctx->R ? md_run_batched(ctx, positions, velocities, nsteps, energies)
              : md_run(ctx, positions, velocities, nsteps, energies);
  if (rc != BPIMD_OK) return rc;
  return read_status(ctx);
}

int bpimd_profile_begin(bpimd_ctx *ctx, int max_evals) {
  if (!ctx || max_evals < 1 || max_evals > (1 << 20)) return BPIMD_ERR_ARG;
  const size_t need = (size_t)max_evals * (BPIMD_NUM_STAGES + 1);
  while (ctx->prof_events.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return BPIMD_ERR_CUDA;
    ctx->prof_events.push_back(e);
  }
  ctx->prof_max = max_evals;
  ctx->prof_count = 0;
  ctx->prof_on = true;
  return BPIMD_OK;
}

int bpimd_profile_end(bpimd_ctx *ctx, double *stage_ms, int *n_evals) {
  if (!ctx) return BPIMD_ERR_ARG;
  ctx->prof_on = false;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return BPIMD_ERR_CUDA;
  double acc[BPIMD_NUM_STAGES] = {0};
  for (int k = 0; k < ctx->prof_count; ++k) {
    cudaEvent_t *ev = &ctx->prof_events[(size_t)k * (BPIMD_NUM_STAGES + 1)];
    for (int i = 0; i < BPIMD_NUM_STAGES; ++i) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) != cudaSuccess) return BPIMD_ERR_CUDA;
      acc[i] += ms;
    }
  }
  if (stage_ms)
    for (int i = 0; i < BPIMD_NUM_STAGES; ++i) stage_ms[i] = acc[i];
  if (n_evals) *n_evals = ctx->prof_count;
  ctx->prof_count = 0;
  return BPIMD_OK;
}

const char *bpimd_status_string(int status) {
  switch (status) {
    case BPIMD_OK: return "ok";
    case BPIMD_ERR_ARG: return "invalid argument";
    case BPIMD_ERR_NONFINITE: return "non-finite value in positions or results";
    case BPIMD_ERR_CUDA: return "CUDA runtime error";
    case BPIMD_ERR_TIMEOUT: return "bounded device wait expired";
    case BPIMD_ERR_NOMEM: return "allocation failed";
    case BPIMD_ERR_STATE: return "call not valid in this state";
    case BPIMD_ERR_SIZE: return "problem larger than the fixed scratch of the allocation-free entry point";
    default: return "unknown status";
  }
}

const char *bpimd_version(void) { return "bpimd 0.2 (sm_103a)"; }

}  // extern "C"
