// Forward and backward potential recursions, one thread-block cluster each
// (the two clusters run concurrently).
//
// Forward  (Eq. our-forward-potential-recurrence, linear-space form):
//   y_0 = 1,  y_{r+1} = c_{r+1} * S_r,  S_r = sum_{w<=r} y_w g(w+1, r+1)
// Backward (Eq. backward-potential-recursion, linear-space form), with rows
// r = N-1-a and sources w = N-1-b so that it has the same lower-triangular
// shape:  Y_0 = mu_N = 1, S_r = B_{a+1} = sum_{w<=r} Y_w g(a+1, b+1),
//   Y_{r+1} = mu_a = c_a * S_r   (c_0 := 1 for the last row, Y_N = B_1).
// Both are lower-triangular solves with the matrix H of pair factors g, and
// with K(w, r) = c_r H(w, r) each is  Y_{r+1} = sum_{w<=r} K(w, r) Y_w.
//
// GB300 facts behind the schedule (measured): a float64 FMA has a 64-cycle
// latency (plus ~40 before a shuffle can read it), while the integer form of
// the step below takes ~100 cycles including its shuffle with 64-bit
// mantissas and ~80 with the 32-bit words of MIXED; a release/acquire
// hand-off between warps inside a step costs far more than the step itself;
// a cluster barrier costs ~360 cycles and a distributed shared-memory access
// ~215.  So the rows are processed in tiles of 32 and
//   * all intra-tile work stays in one warp of the lead CTA (cluster rank 0):
//     warp 0 runs the 32 dependent steps of row tile t.  Lane j holds
//     c_r * (partial row sum) of row 32t+j and the partial sum of row
//     32(t+1)+j.  A step is one integer extended multiply-add on the current
//     row (the dependency chain: acc_j += K(i, j) y_i with integer
//     mantissas, 32-bit words in MIXED and 64-bit in FP64, chain_common.cuh),
//     one term of the next tile's row (off the chain), and a shuffle that
//     broadcasts the new Y;
//   * twelve other lead warps (none on warp 0's sub-partition) stage, for
//     tile t+1, the block of H from source tile t+1 to the rows of tile t+2
//     and the diagonal block pre-scaled by c; one more lead warp of the
//     forward cluster forms the prefix sums C, one tile of 32 per period;
//   * the O(N^2) bulk runs on the other CTAs of the cluster (seven, or
//     fifteen in the 16-CTA form used above N = 1280): row tile T belongs to
//     CTA 1 + T mod NH, which keeps its rows' partial sums in its own shared
//     memory.  In period t each of them adds source tile t-1 to
//     every row tile T >= t+1 it owns: one warp per (row tile, quarter of 8
//     sources), each reading its 8 values of Y from the lead's shared memory
//     and issuing its 16 loads at once; the quarters are then combined in a
//     fixed order, and the owner of tile t+1 writes that tile's finished
//     sums into the lead.
// The float64 pipe of an SM is shared by all its warps and is slow on GB300
// (a warp-wide float64 instruction occupies it for about 64 cycles), so
// outside the dependency chain the kernel uses integer and float32 work:
// staging converts and scales mantissas with integer arithmetic, and MIXED
// sums the next tile's rows in float32.
// Periods are separated by one cluster barrier (release/acquire), which also
// orders every distributed shared-memory access; nothing spins.
// Each recursion reads H from a copy of the pair factors laid out in its own
// (row, source) coordinates, so all block loads are coalesced.
// Every value is an extended number m * 2^e (int32 exponent), so no exp/log
// sits on the dependency chain.  MIXED: the bulk products are summed in
// float32 per 32-source tile and added to the float64 row accumulator; the
// tile hand-offs stay float64 and the dependent steps use the integer format.
#include <cooperative_groups.h>
#include <mutex>
#include <type_traits>

#include "chain_common.cuh"

namespace cg = cooperative_groups;

namespace bpimd {
namespace {

using namespace chain_detail;

// Bulk CTAs per recursion (NH): 7 in an 8-CTA cluster; 15 in a 16-CTA
// cluster (a non-portable size that GB300 grants on request) once N is large
// enough for the bulk work, rather than the chain, to set the pace.
constexpr int YRING = 128;                // Y values kept in the lead (4 tiles)

// Shared memory of the lead CTA.
struct LeadSmem {
  unsigned long long Kdm[2 * BLK];  // c-scaled diagonal blocks (double buffer)
  double Hom[2 * BLK];  // H(source of tile t, row of tile t+1) (double buffer; MIXED: floats)
  double Ym[YRING];     // Y_v at v mod YRING
  double Am[2 * TILE];  // bulk row sums of the next tile, written by its owner
  double misc[4];       // end of the forward recursion: C'[N], 1/(N y_N) mantissa
  long long nsum;       // sum of the exponent parts n carried by y_N
  int Kde[2 * BLK];
  int Hoe[2 * BLK];
  int Ye[YRING];
  int Ae[2 * TILE];
  int misci[4];         // 1/(N y_N) exponent
  unsigned long long T63[256];  // recompute mode: table of the integer-pipe power of two
};

// Shared memory of a bulk CTA: its rows' partial sums (local tile lt = T / 7),
// one slot of 8 Y values per warp, and the partial sums of the current period
// (4 quarter-tiles of 8 sources per owned row tile).
struct HelperSmem {
  double *Am;   // [ltiles][32]
  int *Ae;      // [ltiles][32]
  double *Pm;   // [4 * ltiles][32] partial sums of the period (MIXED: floats)
  int *Pe;      // [4 * ltiles][32]
  double *Yd;   // [32 warps][8] Y mantissas (MIXED: floats)
  int *Yx;      // [32 warps][8] exponents
};

__host__ __device__ constexpr int helper_tiles(int NT, int NH) { return (NT + NH - 1) / NH; }

__host__ __device__ constexpr size_t helper_smem_bytes(int NT, int NH) {
  return (size_t)helper_tiles(NT, NH) * TILE * (sizeof(double) + sizeof(int)) * 5 +
         (size_t)32 * 8 * (sizeof(double) + sizeof(int)) + 256 * sizeof(unsigned long long);
}

// Staging of the next tile's blocks from the stored factors or, in recompute
// mode, from the endpoint copies (the box flag is read at run time).
template <int MODE, bool BWD, bool RC, int NR>
__device__ __forceinline__ void stage_diag_any(const Workspace &w, int tt, int i0, unsigned long long *dm, int *de,
                                               const unsigned long long *T63) {
  if constexpr (!RC) stage_diag<MODE == BPIMD_MIXED32, BWD, NR>(w, tt, i0, dm, de);
  else if (w.pbc) stage_diag_rc<MODE, BWD, true, NR>(w, tt, i0, dm, de, T63);
  else stage_diag_rc<MODE, BWD, false, NR>(w, tt, i0, dm, de, T63);
}
template <int MODE, bool BWD, bool RC, int NR>
__device__ __forceinline__ void stage_offdiag_any(const Workspace &w, int tt, int i0, void *dm, int *de,
                                                  const unsigned long long *T63) {
  if constexpr (!RC) stage_offdiag<MODE == BPIMD_MIXED32, BWD, NR>(w, tt, i0, dm, de);
  else if (w.pbc) stage_offdiag_rc<MODE, BWD, true, NR>(w, tt, i0, dm, de, T63);
  else stage_offdiag_rc<MODE, BWD, false, NR>(w, tt, i0, dm, de, T63);
}

// Recompute mode: the 8 factors H(sb + i, r) of one bulk task (rows past N
// get extended zeros).
template <int MODE, bool BWD, typename M_t>
__device__ __forceinline__ void bulk_factors_rc(const Workspace &w, int r, int sb, const unsigned long long *T63,
                                                M_t (&m)[8], int (&e)[8]) {
  if (r >= w.N) {
#pragma unroll
    for (int i = 0; i < 8; ++i) { m[i] = (M_t)1.0; e[i] = XZERO_E; }
    return;
  }
  if (w.pbc) {
    RowEnds<MODE, BWD, true> re;
    re.load(w, r);
#pragma unroll
    for (int i = 0; i < 8; ++i) m[i] = re.h(w, sb + i, T63, e[i]);
  } else {
    RowEnds<MODE, BWD, false> re;
    re.load(w, r);
#pragma unroll
    for (int i = 0; i < 8; ++i) m[i] = re.h(w, sb + i, T63, e[i]);
  }
}

// MODE: precision form (the stored-factor kernels serve BPIMD_MIXED with the
// BPIMD_FP64 code: the same float64-mantissa layout); RC: recompute mode, H
// formed from the endpoint copies wherever it is used.
template <int MODE, bool BWD, int NHELP, bool RC>
__device__ void run_chain(const Workspace &w, unsigned char *smem_raw, double *V_B) {
  constexpr bool MIXED = MODE == BPIMD_MIXED32;
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const int N = w.N, NT = w.NT;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // H(src, row) in this recursion's own coordinates (both copies share the layout)
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const void *gm = BWD ? w.gbm : w.gm;
  const int *ge = BWD ? w.gbe : w.ge;
  double *gYm = BWD ? w.ybm : w.yfm;
  int *gYe = BWD ? w.ybe : w.yfe;
  LeadSmem *lead_local = (LeadSmem *)smem_raw;
  // the lead's shared memory as seen from this CTA (distributed shared memory)
  LeadSmem *lead = cluster.map_shared_rank(lead_local, 0);

  if (rank == 0) {
    LeadSmem &sm = *lead_local;
    // Staging warps are the lead's warps off warp 0's sub-partition (warp id
    // not a multiple of 4), numbered q = 0, 1, ...: q < 8 stage four rows each
    // of the diagonal block, 8 <= q < 12 eight rows each of the off-diagonal
    // block, q == 12 forms the prefix sums (forward recursion), q == 13
    // copies each finished tile of Y to global memory one period later.
    if (tid < 2 * TILE) { sm.Am[tid] = 0.0; sm.Ae[tid] = XZERO_E; }
    if (tid == 0) { sm.Ym[0] = 1.0; sm.Ye[0] = 0; gYm[0] = 1.0; gYe[0] = 0; }
    if (!BWD && tid == 0) w.C[0] = 0.0;
    const int q = (wid & 3) ? wid - (wid >> 2) - 1 : -1;  // staging index (-1: SMSP of warp 0)
    if (RC) {
      pairg::table_init(sm.T63);
      __syncthreads();
    }
    if (q >= 0 && q < 8) stage_diag_any<MODE, BWD, RC, 4>(w, 0, 4 * q, sm.Kdm, sm.Kde, sm.T63);
    if (q >= 8 && q < 12) stage_offdiag_any<MODE, BWD, RC, 8>(w, 0, 8 * (q - 8), sm.Hom, sm.Hoe, sm.T63);
    cluster.sync();

    xd nxt{1.0, XZERO_E};  // warp 0: partial sum of row 32(t+1)+lane over source tile t
    xd cnext{1.0, 0};      // warp 0: coefficient of its row in the coming tile
    if (wid == 0 && lane < N) cnext = chain_coef<BWD>(w, lane);
    double carry = 0.0;    // prefix-sum warp (forward): running reduced prefix sum C'
    long long ncarry = 0;  // and the running sum of the exponent parts n
    for (int t = 0; t < NT; ++t) {
      const int buf = t & 1;
      if (wid == 0) {
        // ---------------------------------------------- dependent steps of tile t
        const int row = t * TILE + lane;
        const xd crow = cnext;
        if (row + TILE < N) cnext = chain_coef<BWD>(w, row + TILE);  // prefetch for tile t+1
        chain_tile<MIXED>(N, t, xd{sm.Am[buf * TILE + lane], sm.Ae[buf * TILE + lane]}, crow, nxt,
                          sm.Kdm + buf * BLK, sm.Kde + buf * BLK, sm.Hom + buf * BLK, sm.Hoe + buf * BLK,
                          sm.Ym, sm.Ye, YRING - 1, nullptr, nullptr);
      } else if (q >= 0 && q < 8) {
        if (t + 1 < NT)
          stage_diag_any<MODE, BWD, RC, 4>(w, t + 1, 4 * q, sm.Kdm + (buf ^ 1) * BLK, sm.Kde + (buf ^ 1) * BLK,
                                          sm.T63);
      } else if (q >= 8 && q < 12) {
        if (t + 1 < NT)
          stage_offdiag_any<MODE, BWD, RC, 8>(w, t + 1, 8 * (q - 8), sm.Hom + (buf ^ 1) * BLK,
                                             sm.Hoe + (buf ^ 1) * BLK, sm.T63);
      } else if (q == 13) {
        // export Y of tile t-1 from the ring to global memory, off the chain
        // warp (a release barrier after global stores would wait for them)
        if (t >= 1) {
          const int v = (t - 1) * TILE + lane + 1;
          if (v <= N) { gYm[v] = sm.Ym[v & (YRING - 1)]; gYe[v] = sm.Ye[v & (YRING - 1)]; }
        }
      } else if (!BWD && q == 12) {
        prefix_tile(w, t, carry, ncarry);
      }
      cluster.sync();
    }
    pdl_trigger();  // the probability pass may launch during the epilogue
    if (q == 13) {  // the last tile's Y
      const int v = (NT - 1) * TILE + lane + 1;
      if (v <= N) { gYm[v] = sm.Ym[v & (YRING - 1)]; gYe[v] = sm.Ye[v & (YRING - 1)]; }
    }
    if (!BWD) {
      // V^{[1,N]} = C'[N] - (ln(y_N) - n ln 2)/beta, normaliser 1/(N y_N), alpha_a = y_a/(N y_N)
      if (q == 12 && lane == 0) { sm.misc[0] = carry; sm.nsum = ncarry; }
      __syncthreads();
      const xd yN{sm.Ym[N & (YRING - 1)], sm.Ye[N & (YRING - 1)]};
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
        for (int a = tid - 32; a < N; a += blockDim.x - 32) store_alpha<MIXED>(w, a, xd{gYm[a], gYe[a]}, inv);
      }
    }
  } else {
    // ------------------------------------------------------------ bulk CTA
    HelperSmem hs;
    unsigned char *p = smem_raw;
    const int lt_max = helper_tiles(NT, NHELP);
    hs.Am = (double *)p; p += sizeof(double) * lt_max * TILE;
    hs.Pm = (double *)p; p += sizeof(double) * 4 * lt_max * TILE;
    hs.Yd = (double *)p; p += sizeof(double) * 32 * 8;
    hs.Ae = (int *)p; p += sizeof(int) * lt_max * TILE;
    hs.Pe = (int *)p; p += sizeof(int) * 4 * lt_max * TILE;
    hs.Yx = (int *)p; p += sizeof(int) * 32 * 8;
    unsigned long long *T63 = (unsigned long long *)p;  // recompute mode
    const int h = (int)rank - 1;  // owns row tiles T with T mod NHELP == h
    const int nwarps = (int)(blockDim.x >> 5);
    for (int q = tid; q < lt_max * TILE; q += blockDim.x) { hs.Am[q] = 0.0; hs.Ae[q] = XZERO_E; }
    if (RC) pairg::table_init(T63);
    cluster.sync();
    for (int t = 0; t < NT; ++t) {
      const int T0 = (t + 1) + ((h - (t + 1) % NHELP) + NHELP) % NHELP;  // first owned row tile >= t+1
      const int nunits = (t >= 1 && T0 < NT) ? (NT - 1 - T0) / NHELP + 1 : 0;
      if (nunits > 0) {
        const int srcbase = (t - 1) * TILE;
        // task k: row tile T0 + (k/4)*7, sources srcbase + 8(k%4) .. +7 (source tile t-1)
        for (int k = wid; k < 4 * nunits; k += nwarps) {
          const int u = k >> 2, q = k & 3;
          const int r = (T0 + u * NHELP) * TILE + lane;
          const int sb = srcbase + 8 * q;
          M_t *Ym = (M_t *)hs.Yd + wid * 8;
          int *Yx = hs.Yx + wid * 8;
          if (lane < 8) {  // this warp's 8 values of Y, from the lead
            const int v = sb + lane;
            const double ym = lead->Ym[v & (YRING - 1)];
            Ym[lane] = MIXED ? (M_t)mant_to_float(ym) : (M_t)ym;
            Yx[lane] = lead->Ye[v & (YRING - 1)];
          }
          __syncwarp();
          const size_t gbase = hidx(sb, r);  // + i * 32 for source sb + i
          if (MIXED) {
            float m[8];
            int e[8];
            if (RC) {
              bulk_factors_rc<MODE, BWD>(w, r, sb, T63, m, e);
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                m[i] = __ldg((const float *)gm + gbase + i * 32);
                e[i] = __ldg(ge + gbase + i * 32);
              }
            }
            float sacc = 0.0f;
            int E = XZERO_E;
#pragma unroll
            for (int i = 0; i < 8; ++i) fmerge(sacc, E, (float)Ym[i] * m[i], e[i] + Yx[i]);
            ((float *)hs.Pm)[k * TILE + lane] = sacc;
            hs.Pe[k * TILE + lane] = E;
          } else {
            double m[8];
            int e[8];
            int E = XZERO_E;
            if (RC) {
              bulk_factors_rc<MODE, BWD>(w, r, sb, T63, m, e);
#pragma unroll
              for (int i = 0; i < 8; ++i) e[i] += Yx[i];
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                m[i] = __ldg((const double *)gm + gbase + i * 32);
                e[i] = __ldg(ge + gbase + i * 32) + Yx[i];
              }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) E = max(E, e[i]);
            double sacc = 0.0;
#pragma unroll
            for (int i = 0; i < 8; ++i) sacc = fma(scale_nonpos(m[i], e[i] - E), (double)Ym[i], sacc);
            hs.Pm[k * TILE + lane] = sacc;
            hs.Pe[k * TILE + lane] = E;
          }
          __syncwarp();
        }
        __syncthreads();
        // combine the four quarters of each owned row tile in a fixed order
        for (int u = wid; u < nunits; u += nwarps) {
          const int T = T0 + u * NHELP, lt = T / NHELP;
          xd acc{hs.Am[lt * TILE + lane], hs.Ae[lt * TILE + lane]};
          if (MIXED) {
            float sacc = 0.0f;
            int E = XZERO_E;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              fmerge(sacc, E, ((const float *)hs.Pm)[(4 * u + q) * TILE + lane], hs.Pe[(4 * u + q) * TILE + lane]);
            acc = xadd_int(acc, xd{f2d_int(sacc), E});
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              acc = xadd_int(acc, xnorm_int(xd{hs.Pm[(4 * u + q) * TILE + lane], hs.Pe[(4 * u + q) * TILE + lane]}));
          }
          acc = xnorm_int(acc);
          hs.Am[lt * TILE + lane] = acc.m;
          hs.Ae[lt * TILE + lane] = acc.e;
          if (T == t + 1) {  // finished: hand the tile's sums to the lead
            const int slot = ((t + 1) & 1) * TILE + lane;
            lead->Am[slot] = acc.m;
            lead->Ae[slot] = acc.e;
          }
        }
      }
      cluster.sync();
    }
  }
}

// Cluster size CL (CTAs per recursion) is given at launch; blocks [0, CL) run
// the forward recursion, [CL, 2 CL) the backward one.
template <int MODE, int CL, bool RC>
__global__ void __launch_bounds__(CHAIN_THREADS, 1) chain_kernel(Workspace w, double *V_B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  if (blockIdx.x < CL) run_chain<MODE, false, CL - 1, RC>(w, smem_raw, V_B);
  else run_chain<MODE, true, CL - 1, RC>(w, smem_raw, V_B);
}

constexpr size_t chain_smem_bytes(int N, int CL) {
  const size_t lead = sizeof(LeadSmem);
  const size_t help = helper_smem_bytes((N + TILE - 1) / TILE, CL - 1);
  return lead > help ? lead : help;
}
static_assert(chain_smem_bytes(CHAIN_MAX_N, CHAIN_CLUSTER) <= 227 * 1024,
              "recursion state for the largest N must fit in shared memory");
constexpr int CHAIN_CLUSTER_LARGE = 16;
constexpr int LARGE_CLUSTER_MIN_NT = 41;  // N > 1280: the bulk work would set the pace with 7 bulk CTAs

template <int MODE, int CL, bool RC>
cudaError_t launch_chain_cluster(const Workspace &w, double *V_B, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * CL);
  cfg.blockDim = dim3(CHAIN_THREADS);
  cfg.dynamicSmemBytes = chain_smem_bytes(w.N, CL);
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, chain_kernel<MODE, CL, RC>, w, V_B);
}

// The kernel variant of a workspace: stored factors serve BPIMD_MIXED with the
// float64-layout code; the recompute mode has one variant per precision form.
template <int CL>
cudaError_t launch_chain_variant(const Workspace &w, double *V_B, cudaStream_t s) {
  if (!w.recomp)
    return w.mixed ? launch_chain_cluster<BPIMD_MIXED32, CL, false>(w, V_B, s)
                   : launch_chain_cluster<BPIMD_FP64, CL, false>(w, V_B, s);
  switch (w.mode) {
    case BPIMD_FP64: return launch_chain_cluster<BPIMD_FP64, CL, true>(w, V_B, s);
    case BPIMD_MIXED: return launch_chain_cluster<BPIMD_MIXED, CL, true>(w, V_B, s);
    default: return launch_chain_cluster<BPIMD_MIXED32, CL, true>(w, V_B, s);
  }
}
static_assert(CHAIN_THREADS % 32 == 0 && CHAIN_THREADS / 32 >= 19 && CHAIN_THREADS / 32 <= 32,
              "the lead needs 14 warps off warp 0's sub-partition (staging, prefix sums, Y export); a bulk CTA has at most 32 Y slots");

}  // namespace

// Once per process and device (host calls that must not sit between the
// launches of an evaluation): raise the dynamic shared-memory limit of the
// recursion kernels to the maximum, allow the 16-CTA clusters, and check that
// two of them can be resident (else the 8-CTA form is used for every N).
namespace {
// per device: set up once under g_chain_mutex (two host threads making their
// first calls on one device must not both write these)
std::mutex g_chain_mutex;
bool g_chain_ready[64] = {false};
bool g_large_cluster[64] = {false};

template <int MODE, int CL, bool RC>
cudaError_t prepare_chain_kernel() {
  const int bytes = (int)chain_smem_bytes(CHAIN_MAX_N, CL);
  cudaError_t e =
      cudaFuncSetAttribute(chain_kernel<MODE, CL, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && CL > 8)
    e = cudaFuncSetAttribute(chain_kernel<MODE, CL, RC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}
template <int CL>
cudaError_t prepare_chain_variants() {
  cudaError_t e = prepare_chain_kernel<BPIMD_MIXED32, CL, false>();
  if (e == cudaSuccess) e = prepare_chain_kernel<BPIMD_FP64, CL, false>();
  if (e == cudaSuccess) e = prepare_chain_kernel<BPIMD_FP64, CL, true>();
  if (e == cudaSuccess) e = prepare_chain_kernel<BPIMD_MIXED, CL, true>();
  if (e == cudaSuccess) e = prepare_chain_kernel<BPIMD_MIXED32, CL, true>();
  return e;
}

template <int CL>
bool clusters_fit() {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * CL);
  cfg.blockDim = dim3(CHAIN_THREADS);
  cfg.dynamicSmemBytes = chain_smem_bytes(CHAIN_MAX_N, CL);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  const bool ok =
      cudaOccupancyMaxActiveClusters(&n, chain_kernel<BPIMD_MIXED32, CL, false>, &cfg) == cudaSuccess && n >= 2;
  cudaGetLastError();
  return ok;
}
}  // namespace

cudaError_t prepare_chains() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_chain_mutex);
  if (g_chain_ready[dev]) return cudaSuccess;
  e = prepare_chain_variants<CHAIN_CLUSTER>();
  if (e != cudaSuccess) return e;
  bool large = prepare_chain_variants<CHAIN_CLUSTER_LARGE>() == cudaSuccess;
  cudaGetLastError();
  large = large && clusters_fit<CHAIN_CLUSTER_LARGE>();
  g_large_cluster[dev] = large;
  g_chain_ready[dev] = true;
  return cudaSuccess;
}

cudaError_t launch_chains(const Workspace &w, double *V_B, cudaStream_t s) {
  cudaError_t e = prepare_chains();
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);
  bool large_ok;
  {
    std::lock_guard<std::mutex> lock(g_chain_mutex);
    large_ok = g_large_cluster[dev];
  }
  const bool large = large_ok && w.NT >= LARGE_CLUSTER_MIN_NT;
  return large ? launch_chain_variant<CHAIN_CLUSTER_LARGE>(w, V_B, s) : launch_chain_variant<CHAIN_CLUSTER>(w, V_B, s);
}

}  // namespace bpimd
