// C ABI of replica batches: many independent systems of uneven N, P, beta
// (same mass and precision) evaluated together, three launches per batch
// (bead pass with pair factors, both recursions of every replica,
// probabilities and forces), whatever the number of replicas -- plus one
// recursion launch per replica larger than BATCH_MAX_N, which takes the
// cluster kernel of single systems.
#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>

#include "context.cuh"

using namespace bpimd;

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool finite_positive(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

namespace bpimd {

int evaluate_batched(bpimd_ctx *ctx, const double *pos, double *V_B, double *F) {
  cudaStream_t s = ctx->stream;
  const int mode = ctx->cfg.precision;
  cudaEvent_t *ev = nullptr;
  if (ctx->prof_on && ctx->prof_count < ctx->prof_max)
    ev = &ctx->prof_events[(size_t)ctx->prof_count++ * (BPIMD_NUM_STAGES + 1)];
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  mark(0);
  if (launch_prep_batched(ctx->d_ws, ctx->d_bead_tab, ctx->n_bead_tab, ctx->d_blk_tab, ctx->n_blk_tab, ctx->d_off,
                          mode, pos, F, ctx->tune_gmat_bpsm, s) != cudaSuccess)
    return BPIMD_ERR_CUDA;
  mark(1);
  // replicas above BATCH_MAX_N (first in the order) take the cluster recursion
  // kernel of single systems, one launch each; the rest share one launch
  for (int k = 0; k < ctx->n_big; ++k) {
    const int r = ctx->h_order[k];
    if (launch_chains(ctx->h_ws[r], V_B ? V_B + r : nullptr, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  }
  if (launch_chains_batched(ctx->d_ws, ctx->d_order + ctx->n_big, ctx->R - ctx->n_big, ctx->maxN,
                            mode == BPIMD_MIXED32, V_B, s) != cudaSuccess)
    return BPIMD_ERR_CUDA;
  mark(2);
  if (launch_prob_forces_batched(ctx->d_ws, ctx->d_blk_tab, ctx->n_blk_tab, ctx->d_off, mode, pos, F,
                                 ctx->tune_prob_bpsm, s) != cudaSuccess)
    return BPIMD_ERR_CUDA;
  mark(3);
  ctx->evaluated = true;
  return BPIMD_OK;
}

}  // namespace bpimd

extern "C" {

int bpimd_create_batched(bpimd_ctx **out, const bpimd_config *cfg, int32_t R, const int32_t *N, const int32_t *P,
                         const double *omega_P, const double *beta, void *cuda_stream) {
  if (!out) return BPIMD_ERR_ARG;
  *out = nullptr;
  if (!cfg || !N || !P || !omega_P || !beta || R < 1 || R > (1 << 20)) return BPIMD_ERR_ARG;
  if (!finite_positive(cfg->m) || cfg->flags != 0 || cfg->box_L != 0.0) return BPIMD_ERR_ARG;
  if (!valid_precision(cfg->precision)) return BPIMD_ERR_ARG;
  long long total = 0;
  for (int r = 0; r < R; ++r) {
    if (N[r] < 1 || N[r] > BPIMD_STORE_MAX_N || P[r] < 2 || P[r] > (1 << 16)) return BPIMD_ERR_ARG;
    if (!finite_positive(omega_P[r]) || !finite_positive(beta[r])) return BPIMD_ERR_ARG;
    total += 3LL * N[r] * P[r];
  }
  if (total > (1LL << 40)) return BPIMD_ERR_ARG;
  bpimd_ctx *ctx = new (std::nothrow) bpimd_ctx();
  if (!ctx) return BPIMD_ERR_NOMEM;
  ctx->cfg = *cfg;
  ctx->cfg.N = 0;
  ctx->cfg.P = 0;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->R = R;
  ctx->total_elems = total;
  ctx->tune_gmat_bpsm = 8;
  ctx->pair_lanes = 4;
  ctx->tune_prob_bpsm = 8;
  ctx->h_ws.resize(R);
  ctx->h_off.resize(R);
  // host tables
  std::vector<int2> bead_tab, blk_tab;
  std::vector<int> order(R);
  long long off = 0;
  size_t wbytes = 0;
  for (int r = 0; r < R; ++r) {
    Workspace &w = ctx->h_ws[r];
    w.N = N[r];
    w.P = P[r];
    w.inv_P = 1.0 / P[r];
    w.NT = (w.N + TILE - 1) / TILE;
    w.NB = w.NT * (w.NT + 1) / 2;
    set_precision(w, cfg->precision);
    w.m = cfg->m;
    w.omega_P = omega_P[r];
    w.beta = beta[r];
    w.k = cfg->m * omega_P[r] * omega_P[r];
    w.half_k = 0.5 * w.k;
    w.cx = w.beta * w.half_k * LOG2E;
    w.blocks = N[r] > BATCH_MAX_N;  // those take the cluster recursion
    wbytes += align256(layout_workspace(w, nullptr));
    ctx->h_off[r] = off;
    off += 3LL * N[r] * P[r];
    for (int l0 = 0; l0 < N[r]; l0 += BEAD_BLOCK_PARTICLES) bead_tab.push_back(make_int2(r, l0));
    for (int b = 0; b < w.NB; ++b) blk_tab.push_back(make_int2(r, b));
    if (N[r] <= BATCH_MAX_N) ctx->maxN = std::max(ctx->maxN, N[r]);
    else ctx->n_big++;
  }
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return N[a] > N[b]; });
  ctx->h_order = order;
  ctx->n_bead_tab = (int)bead_tab.size();
  ctx->n_blk_tab = (int)blk_tab.size();
  // one allocation: workspaces, shared status word, tables
  const size_t o_ws = 0;
  const size_t o_status = o_ws + wbytes;
  const size_t o_dws = o_status + 256;
  const size_t o_bead = o_dws + align256(sizeof(Workspace) * R);
  const size_t o_blk = o_bead + align256(sizeof(int2) * bead_tab.size());
  const size_t o_order = o_blk + align256(sizeof(int2) * blk_tab.size());
  const size_t o_off = o_order + align256(sizeof(int) * R);
  const size_t bytes = o_off + align256(sizeof(long long) * R);
  if (cudaMalloc(&ctx->dev_block, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return BPIMD_ERR_NOMEM;
  }
  ctx->dev_bytes = bytes;
  char *base = (char *)ctx->dev_block;
  int *status = (int *)(base + o_status);
  size_t cur = o_ws;
  for (int r = 0; r < R; ++r) {
    Workspace &w = ctx->h_ws[r];
    const size_t b = layout_workspace(w, base + cur);
    cur += align256(b);
    w.status = status;  // one status word for the batch
  }
  ctx->w = ctx->h_ws[0];
  ctx->w.status = status;
  ctx->d_ws = (Workspace *)(base + o_dws);
  ctx->d_bead_tab = (int2 *)(base + o_bead);
  ctx->d_blk_tab = (int2 *)(base + o_blk);
  ctx->d_order = (int *)(base + o_order);
  ctx->d_off = (long long *)(base + o_off);
  cudaStream_t s = ctx->stream;
  bool ok = cudaMemsetAsync(base, 0, o_dws, s) == cudaSuccess &&
            cudaMemcpyAsync(ctx->d_ws, ctx->h_ws.data(), sizeof(Workspace) * R, cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync(ctx->d_bead_tab, bead_tab.data(), sizeof(int2) * bead_tab.size(),
                            cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(ctx->d_blk_tab, blk_tab.data(), sizeof(int2) * blk_tab.size(), cudaMemcpyHostToDevice,
                            s) == cudaSuccess &&
            cudaMemcpyAsync(ctx->d_order, order.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(ctx->d_off, ctx->h_off.data(), sizeof(long long) * R, cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            launch_gmat_padding_batched(ctx->d_ws, ctx->d_blk_tab, ctx->n_blk_tab, cfg->precision == BPIMD_MIXED32,
                                        s) == cudaSuccess &&
            cudaMallocHost(&ctx->host_status, sizeof(int)) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess;  // host tables go out of scope
  if (!ok) {
    cudaGetLastError();
    cudaFree(ctx->dev_block);
    if (ctx->host_status) cudaFreeHost(ctx->host_status);
    delete ctx;
    return BPIMD_ERR_NOMEM;
  }
  *ctx->host_status = 0;
  md_init(&ctx->md);
  *out = ctx;
  return BPIMD_OK;
}

int bpimd_exchange_energy_forces_batched(bpimd_ctx *ctx, const double *positions, double *V_B, double *forces) {
  if (!ctx || ctx->R == 0) return ctx ? BPIMD_ERR_STATE : BPIMD_ERR_ARG;
  if (!positions || !forces || (((uintptr_t)positions) & 15) || (((uintptr_t)forces) & 15)) return BPIMD_ERR_ARG;
  if (V_B && (((uintptr_t)V_B) & 7)) return BPIMD_ERR_ARG;
  return evaluate_batched(ctx, positions, V_B, forces);
}

int bpimd_batch_info(bpimd_ctx *ctx, int32_t *R, int64_t *elements, int64_t *offsets) {
  if (!ctx || ctx->R == 0) return ctx ? BPIMD_ERR_STATE : BPIMD_ERR_ARG;
  if (R) *R = ctx->R;
  if (elements) *elements = ctx->total_elems;
  if (offsets)
    for (int r = 0; r < ctx->R; ++r) offsets[r] = ctx->h_off[r];
  return BPIMD_OK;
}

int bpimd_batch_set_tuning(bpimd_ctx *ctx, int32_t pair_blocks_per_sm, int32_t prob_blocks_per_sm) {
  if (!ctx || ctx->R == 0) return ctx ? BPIMD_ERR_STATE : BPIMD_ERR_ARG;
  if (pair_blocks_per_sm < 1 || pair_blocks_per_sm > 64 || prob_blocks_per_sm < 1 || prob_blocks_per_sm > 64)
    return BPIMD_ERR_ARG;
  ctx->tune_gmat_bpsm = pair_blocks_per_sm;
  ctx->tune_prob_bpsm = prob_blocks_per_sm;
  return BPIMD_OK;
}

// Pair tile of the batched MD pair forces (lanes per particle).
int bpimd_batch_set_pair_tile(bpimd_ctx *ctx, int32_t lanes_per_particle) {
  if (!ctx) return BPIMD_ERR_ARG;
  if (ctx->R == 0) return BPIMD_ERR_STATE;
  if (lanes_per_particle != 2 && lanes_per_particle != 4 && lanes_per_particle != 8) return BPIMD_ERR_ARG;
  return md_set_pair_tile(ctx, lanes_per_particle);
}

}  // extern "C"
