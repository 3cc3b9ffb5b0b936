// Forward and backward potential recursions of a batch of independent
// replicas (uneven N, P, beta): one CTA per recursion per replica, all in one
// launch.
//
// Same mathematics and the same dependent-step code as chain.cu (Eq.
// our-forward-potential-recurrence, Eq. backward-potential-recursion in linear
// space, tiles of 32 rows; see chain_common.cuh).  A small replica has little
// O(N^2) bulk per tile, so instead of a cluster per recursion every role sits
// in one CTA of 16 warps and many recursions share the GPU at once:
//   * warp 0: the 32 dependent steps of row tile t (chain_tile);
//   * warps off warp 0's sub-partition, numbered q = 0..11: q < 4 stage the
//     next diagonal block (8 rows each), q = 4, 5 the next off-diagonal block
//     (16 rows each), q = 6 forms the prefix sums (forward), q >= 7 bulk;
//   * warps 4, 8, 12 and q >= 7 (8 warps): add source tile t-1 to the row
//     tiles >= t+1, one warp per row tile (16 loads in flight per lane).
// Y and the bulk row sums of the whole replica live in shared memory (24 bytes
// per particle), so N is bounded by BATCH_MAX_N.  Tiles meet at
// __syncthreads.  CTAs are ordered by decreasing N (longest chains first).
#include <type_traits>

#include "chain_common.cuh"

namespace bpimd {
namespace {

using namespace chain_detail;

constexpr int BATCH_THREADS = 512;
constexpr int BATCH_BULK_WARPS = 8;

struct SingleSmem {
  unsigned long long Kdm[2 * BLK];
  double Hom[2 * BLK];  // MIXED: floats
  double misc[2];
  long long nsum;  // sum of the exponent parts n carried by y_N
  int Kde[2 * BLK];
  int Hoe[2 * BLK];
  int misci[2];
};

__host__ __device__ constexpr size_t single_smem_bytes(int N) {
  return sizeof(SingleSmem) + (size_t)(N + 1) * (sizeof(double) + sizeof(int)) +
         (size_t)N * (sizeof(double) + sizeof(int));
}

// warp id -> role index q for warps off warp 0's sub-partition (-1 otherwise)
__device__ __forceinline__ int role_q(int wid) { return (wid & 3) ? wid - (wid >> 2) - 1 : -1; }

template <bool MIXED, bool BWD>
__device__ void run_single(const Workspace &w, unsigned char *smem_raw, double *V_B) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const int N = w.N, NT = w.NT;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  SingleSmem &sm = *(SingleSmem *)smem_raw;
  double *Ym = (double *)(smem_raw + sizeof(SingleSmem));
  double *Am = Ym + (N + 1);
  int *Ye = (int *)(Am + N);
  int *Ae = Ye + (N + 1);
  double *gYm = BWD ? w.ybm : w.yfm;
  int *gYe = BWD ? w.ybe : w.yfe;
  const M_t *gm = (const M_t *)chain_gm<BWD>(w);
  const int *ge = chain_ge<BWD>(w);
  const int q = role_q(wid);
  const int bulk = (q >= 7) ? 3 + (q - 7) : ((wid & 3) == 0 && wid > 0 ? (wid >> 2) - 1 : -1);

  for (int r = tid; r < N; r += blockDim.x) { Am[r] = 0.0; Ae[r] = XZERO_E; }
  if (tid == 0) { Ym[0] = 1.0; Ye[0] = 0; gYm[0] = 1.0; gYe[0] = 0; }
  if (!BWD && tid == 0) w.C[0] = 0.0;
  if (q >= 0 && q < 4) stage_diag<MIXED, BWD, 8>(w, 0, 8 * q, sm.Kdm, sm.Kde);
  if (q == 4 || q == 5) stage_offdiag<MIXED, BWD, 16>(w, 0, 16 * (q - 4), sm.Hom, sm.Hoe);
  __syncthreads();

  xd nxt{1.0, XZERO_E};
  xd cnext{1.0, 0};
  if (wid == 0 && lane < N) cnext = chain_coef<BWD>(w, lane);
  double carry = 0.0;
  long long ncarry = 0;
  for (int t = 0; t < NT; ++t) {
    const int buf = t & 1;
    if (wid == 0) {
      const int row = t * TILE + lane;
      const xd crow = cnext;
      if (row + TILE < N) cnext = chain_coef<BWD>(w, row + TILE);
      const xd A = (row < N) ? xd{Am[row], Ae[row]} : xd{0.0, XZERO_E};
      chain_tile<MIXED>(N, t, A, crow, nxt, sm.Kdm + buf * BLK, sm.Kde + buf * BLK, sm.Hom + buf * BLK,
                        sm.Hoe + buf * BLK, Ym, Ye, -1, gYm, gYe);
    } else if (q >= 0 && q < 4) {
      if (t + 1 < NT) stage_diag<MIXED, BWD, 8>(w, t + 1, 8 * q, sm.Kdm + (buf ^ 1) * BLK, sm.Kde + (buf ^ 1) * BLK);
    } else if (q == 4 || q == 5) {
      if (t + 1 < NT)
        stage_offdiag<MIXED, BWD, 16>(w, t + 1, 16 * (q - 4), sm.Hom + (buf ^ 1) * BLK, sm.Hoe + (buf ^ 1) * BLK);
    } else if (q == 6) {
      if (!BWD) prefix_tile(w, t, carry, ncarry);
    } else if (bulk >= 0 && t >= 1) {
      // source tile t-1 -> row tiles t+1.., one warp per row tile
      const int srcbase = (t - 1) * TILE;
      for (int T = t + 1 + bulk; T < NT; T += BATCH_BULK_WARPS) {
        const int r = T * TILE + lane;
        const size_t gbase = hidx(srcbase, r);
        xd acc{Am[r < N ? r : 0], Ae[r < N ? r : 0]};
        if (MIXED) {
          float sacc = 0.0f;
          int E = XZERO_E;
#pragma unroll
          for (int h = 0; h < TILE; h += 16) {
            float m[16];
            int e[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              m[i] = __ldg(gm + gbase + (h + i) * 32);
              e[i] = __ldg(ge + gbase + (h + i) * 32);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int v = srcbase + h + i;
              fmerge(sacc, E, mant_to_float(Ym[v]) * m[i], e[i] + Ye[v]);
            }
          }
          acc = xadd_int(acc, xd{f2d_int(sacc), E});
        } else {
          int E = XZERO_E;
          double m[16];
          int e[16];
          double sacc = 0.0;
#pragma unroll
          for (int h = 0; h < TILE; h += 16) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              m[i] = __ldg(gm + gbase + (h + i) * 32);
              e[i] = __ldg(ge + gbase + (h + i) * 32) + Ye[srcbase + h + i];
            }
            // one exponent per half tile: the second half rescales the first
            int Eh = XZERO_E;
#pragma unroll
            for (int i = 0; i < 16; ++i) Eh = max(Eh, e[i]);
            double hs = 0.0;
#pragma unroll
            for (int i = 0; i < 16; ++i) hs = fma(scale_nonpos(m[i], e[i] - Eh), Ym[srcbase + h + i], hs);
            const xd part = xadd_int(xd{sacc, E}, xnorm_int(xd{hs, Eh}));
            sacc = part.m;
            E = part.e;
          }
          acc = xadd_int(acc, xnorm_int(xd{sacc, E}));
        }
        acc = xnorm_int(acc);
        if (r < N) { Am[r] = acc.m; Ae[r] = acc.e; }
      }
    }
    __syncthreads();
  }
  pdl_trigger();  // the probability pass may launch during the epilogue
  if (!BWD) {
    // V^{[1,N]} = C'[N] - (ln(y_N) - n ln 2)/beta, normaliser 1/(N y_N), alpha_a = y_a/(N y_N)
    if (q == 6 && lane == 0) { sm.misc[0] = carry; sm.nsum = ncarry; }
    __syncthreads();
    const xd yN{Ym[N], Ye[N]};
    if (tid == 0) {  // the normaliser first: the alpha values wait for it
      const xd inv = xnorm(1.0 / (yN.m * (double)N), -yN.e);
      w.scal[1] = inv.m;
      w.scal_i[0] = inv.e;
      sm.misc[1] = inv.m;
      sm.misci[0] = inv.e;
    }
    __syncthreads();
    if (wid == 0) {  // V_B (a float64 log) on warp 0, alongside the alpha values
      if (lane == 0) {
        const double VB = reduced_potential(sm.misc[0], yN, sm.nsum, w.beta);
        w.scal[0] = VB;
        if (V_B) *V_B = VB;
        if (!isfinite(VB)) atomicOr(w.status, ST_NONFINITE);
      }
    } else {
      const xd inv{sm.misc[1], sm.misci[0]};
      for (int a = tid - 32; a < N; a += blockDim.x - 32) store_alpha<MIXED>(w, a, xd{Ym[a], Ye[a]}, inv);
    }
  }
}

// CTA 2k + d runs recursion d (0 forward, 1 backward) of replica order[k].
template <bool MIXED>
// Two CTAs per SM (64 registers a thread, no spills): each CTA's chain is
// latency-bound on one warp, so two replicas' recursions share an SM.
__global__ void __launch_bounds__(BATCH_THREADS, 2) chain_batched_kernel(const Workspace *__restrict__ ws,
                                                                         const int *__restrict__ order,
                                                                         double *V_B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  const int r = order[blockIdx.x >> 1];
  if (blockIdx.x & 1) run_single<MIXED, true>(ws[r], smem_raw, nullptr);
  else run_single<MIXED, false>(ws[r], smem_raw, V_B ? V_B + r : nullptr);
}

static_assert(single_smem_bytes(BATCH_MAX_N) <= 227 * 1024, "batched recursion state must fit in shared memory");
static_assert(BATCH_THREADS / 32 == 16, "role table assumes 16 warps");

}  // namespace

cudaError_t launch_chains_batched(const Workspace *ws, const int *order, int R, int maxN, bool mixed, double *V_B,
                                  cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && !done[dev]) {
    const int bytes = (int)single_smem_bytes(BATCH_MAX_N);
    e = cudaFuncSetAttribute(chain_batched_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(chain_batched_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  const size_t bytes = single_smem_bytes(maxN);
  e = mixed ? launch_pdl(chain_batched_kernel<true>, 2 * R, BATCH_THREADS, bytes, s, ws, order, V_B)
            : launch_pdl(chain_batched_kernel<false>, 2 * R, BATCH_THREADS, bytes, s, ws, order, V_B);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace bpimd
