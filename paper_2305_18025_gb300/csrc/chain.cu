// Forward and backward potential recursions as blocked triangular solves: one
// kernel forms the inverses of the diagonal tiles, then one thread-block
// cluster per recursion runs the row tiles in order (the two clusters run
// concurrently).
//
// Forward  (Eq. our-forward-potential-recurrence, linear-space form):
//   y_0 = 1,  y_{r+1} = c_{r+1} * S_r,  S_r = sum_{w<=r} y_w g(w+1, r+1)
// Backward (Eq. backward-potential-recursion, linear-space form), with rows
// r = N-1-a and sources w = N-1-b so that it has the same lower-triangular
// shape:  Y_0 = mu_N = 1, S_r = B_{a+1} = sum_{w<=r} Y_w g(a+1, b+1),
//   Y_{r+1} = mu_a = c_a * S_r   (c_0 := 1 for the last row, Y_N = B_1).
// Both read  Y_{r+1} = c_r sum_{w<=r} H(w, r) Y_w  with the pair factors H of
// the recursion's own coordinates and c_r its row coefficient.
//
// Blocked form.  Row tile t (rows r = 32t + j) has the unknowns
// X^t_j = Y_{32t+1+j}; the previous tile's unknowns X^{t-1} are the sources
// 32t-31 .. 32t (X^{-1} = (0, ..., 0, Y_0)).  Then
//   X^t = b^t + L^t X^t,      L^t(j, i) = c_r H(32t+1+i, r)  for i < j,
//   b^t_j = c_r A^t_j + sum_i Dc^t(j, i) X^{t-1}_i,   Dc^t(j, i) = c_r H(32t-31+i, r),
// where A^t_j sums the sources before X^{t-1} (w <= 32t-32).  Hence
//   X^t = M^t b^t,   M^t = (I - L^t)^{-1} = sum_{k<32} (L^t)^k,
// a unit lower-triangular matrix with nonnegative entries (L^t is strictly
// lower triangular and nonnegative), so every sum below adds nonnegative
// terms: no cancellation anywhere.  M^t and Dc^t depend on the positions only;
// tile_inverse_kernel forms them for every tile at once, spread over the GPU,
// and the sequential part of a recursion is two 32 x 32 matrix-vector
// products per tile instead of 32 dependent steps.
//
// Cluster schedule.  GB300 facts behind it (measured): a cluster barrier, and
// a bulk copy in flight anywhere in the cluster, hold a period for ~2000
// cycles; a float64 FMA has a 64-cycle latency and the SM's float64 pipe
// retires ~1.7 lanes per clock, against ~19 for a 32 x 32 -> 64-bit integer
// multiply-add.  So nothing in the loop is a cluster barrier or a bulk copy:
//   * The lead CTA (cluster rank 0) runs tile t in period t with eight phase
//     warps, four rows each; a row's 32 sources are split over eight lanes
//     (four products per lane) and reduced by three shuffle levels.  Phase 1
//     forms b^t = c A^t + Dc^t X^{t-1}, phase 2 X^t = M^t b^t; both use 64-bit
//     integer mantissas (the xi format of chain_common.cuh): no float64
//     instruction on the sequential path.  A loader warp copies tile t+3's Dc
//     and M into shared memory once tile t is done (cp.async, counted on an
//     mbarrier); the export warp writes each finished tile of Y to global
//     memory and hands X^t to the bulk CTAs; another warp forms the prefix
//     sums C' (forward recursion).
//   * The O(N^2) bulk runs on the other CTAs of the cluster (seven, or
//     fifteen in the 16-CTA form used above N = 256): row tile T belongs to
//     CTA 1 + T mod NH, which keeps its rows' sums A in its own shared memory.
//     In period t each adds X^{t-1} to every row tile T >= t+1 it owns: one
//     warp per (row tile, quarter of 8 sources), 64-bit integer products of
//     the float64 factors (float32 products of BPIMD_MIXED32's float32
//     factors); the quarters are combined in a fixed order.  The owner of
//     tile t+1 takes that tile's quarters first and hands c A^{t+1} to the
//     lead as soon as they are done.
//   * Hand-offs are st.async stores into the receiving CTA's shared memory,
//     completed on its mbarriers (X^t in slot t mod XRING of each bulk CTA,
//     c A^t in slot t mod 2 of the lead); every wait is bounded.  Slot reuse
//     is safe without back-pressure: the lead reaches period t only after
//     c A of the last tile <= t of every bulk CTA, so a bulk CTA is at most NH
//     periods behind the X it is sent (XRING > NH), and c A^{t+2} needs X^t,
//     which the lead hands off after reading c A^t.
// Every value is an extended number m * 2^e (int32 exponent), so no exp or
// log is evaluated in the recursions; each recursion reads its own copy of
// the pair factors, laid out in its (source, row) coordinates, with coalesced
// loads.
#include <cooperative_groups.h>
#include <mutex>
#include <type_traits>

#include "chain_common.cuh"

namespace cg = cooperative_groups;

namespace bpimd {
namespace {

using namespace chain_detail;

constexpr int YRING = 128;       // Y values kept in the lead (4 tiles)
constexpr int LEAD_WARPS = 8;    // warps of the two phases
constexpr int EXPORT_WARP = 8;   // copies finished tiles of Y to global memory
constexpr int PREFIX_WARP = 9;   // prefix sums C' (forward recursion)
constexpr int LOADER_WARP = 10;  // copies the phase warps' operands of coming tiles
constexpr int TINV_THREADS = 1024;
// Dynamic shared memory the tile-inverse kernel asks for and does not use: more
// than half an SM's, so that no SM holds two of its issue-bound CTAs (32
// substitution chains each).  Measured: the recursions stage (tile inverses
// and clusters) fell from 63.0 to 61.2 us at N = 1024; the longest CTA is
// still ~2.5x the mean under ncu's cold caches.
constexpr int TINV_PAD_SMEM = 120 * 1024;
constexpr int OPBUF = 3;         // tiles of lead operands in shared memory: the current one and two ahead
constexpr int XRING = 16;        // tiles of X held by a bulk CTA: more than the 15 bulk CTAs of a cluster
constexpr int BAR_PHASE = 1;     // named barrier of the phase warps (phase 1 -> phase 2)
constexpr int BAR_TILE = 2;      // named barrier of the phase, export and loader warps (tile done)
constexpr int BAR_TILE_THREADS = (LEAD_WARPS + 2) * 32;
constexpr int BAR_CRIT = 3;      // named barrier of the four warps of a bulk CTA's critical row tile

// Shared memory of the lead CTA.
struct LeadSmem {
  // Dc and M of tile t in buffer t % OPBUF, copied by the loader warp; opbar[b]
  // completes when its copies into buffer b have landed
  unsigned long long Bk[OPBUF][2 * TILE2];
  int Be[OPBUF][2 * TILE2];
  unsigned long long opbar[OPBUF];
  unsigned long long cAm[2 * TILE];  // c A of tile t in slot t & 1, handed in by the tile's owner
  unsigned long long cabar[2];       // completion of those hand-offs
  unsigned long long never;          // an mbarrier nothing arrives on (BPIMD_FLAG_TEST_TIMEOUT)
  unsigned long long Ym[YRING];      // Y_v at v mod YRING (xi mantissas)
  unsigned long long bm[TILE];       // b of the current tile (phase 1 -> phase 2)
  double misc[4];                    // end of the forward recursion: C'[N], 1/(N y_N) mantissa
  long long nsum;                    // sum of the exponent parts n carried by y_N
  int cAe[2 * TILE];
  int Ye[YRING];
  int be[TILE];
  int misci[4];                      // 1/(N y_N) exponent
  int aborted;                       // a hand-off wait of this CTA expired
};

// Start of a bulk CTA's shared memory (the lead hands X^t in at these
// offsets): X^t in slot t mod XRING, X^{-1} = (0, ..., 0, Y_0) in slot XRING,
// and one mbarrier per ring slot.  The rows' sums A (local tile lt = T / NH),
// the quarter-tile partial sums of the current period and the rows'
// coefficients c follow.
struct HelperHead {
  unsigned long long Xm[XRING + 1][TILE];
  int Xe[XRING + 1][TILE];
  unsigned long long xbar[XRING];
  int aborted;
  int pad[3];
};

__host__ __device__ constexpr int helper_tiles(int NT, int NH) { return (NT + NH - 1) / NH; }

__host__ __device__ constexpr size_t helper_smem_bytes(int NT, int NH, bool RC) {
  return sizeof(HelperHead) +
         (size_t)helper_tiles(NT, NH) * TILE * (sizeof(unsigned long long) + sizeof(int)) * 6 +
         256 * sizeof(unsigned long long);
}

// First row tile >= t + 1 owned by bulk CTA h (tiles T with T mod NH == h);
// the CTA has work in period t while it is below NT.
__host__ __device__ constexpr int bulk_first_tile(int t, int h, int NH) {
  return (t + 1) + ((h - (t + 1) % NH) + NH) % NH;
}

// Row r's pair factors H(src, r) as stored, or recomputed from the endpoint
// copies (bit-identical), as c_r H in the K format.
template <int MODE, bool BWD, bool RC, bool PBC>
struct RowFactors {
  using M_t = typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type;
  RowEnds<MODE, BWD, PBC> re;
  int r;
  __device__ __forceinline__ void load(const Workspace &w, int row) {
    r = row;
    if (RC) re.load(w, row);
  }
  __device__ __forceinline__ void h(const Workspace &w, int src, const unsigned long long *T63, M_t &m,
                                    int &e) const {
    if constexpr (RC) {
      m = re.h(w, src, T63, e);
    } else {
      const size_t gi = hidx(src, r);
      m = __ldg((const M_t *)chain_gm<BWD>(w) + gi);
      e = __ldg(chain_ge<BWD>(w) + gi);
    }
  }
  __device__ __forceinline__ xk k(const Workspace &w, xd c, int src, const unsigned long long *T63) const {
    M_t m;
    int e;
    h(w, src, T63, m, e);
    return mul_mant<M_t>(c, m, e);
  }
};

// Base of tile t's blocks of one recursion: Dc at +0, M at +TILE2.
__device__ __forceinline__ size_t tile_block_base(const Workspace &w, bool bwd, int t) {
  return (size_t)((bwd ? w.NT : 0) + t) * 2 * TILE2;
}
// Layout of a 32 x 32 tile block, in the order the lead's phase warps read it:
// warp w (rows 4w .. 4w+3) lane l = 8 (j & 3) + g holds sources 4g .. 4g+3 of
// row j; a warp's mantissas are two planes of 16-byte pairs (sources 4g, 4g+1
// and 4g+2, 4g+3), its exponents one plane of 16-byte quads, so each read is
// one conflict-free 16-byte load per lane.  Entry (j, i) sits at mantissa
// index 2 (32 (2 (j/4) + (i/2)%2) + 8 (j%4) + i/4) + i%2 and exponent index
// 4 (32 (j/4) + 8 (j%4) + i/4) + i%4; blk_jk / blk_je give (j, i) of an index.
__device__ __forceinline__ int2 blk_jk(int x) {  // (j, i) of mantissa index x
  const int l = (x >> 1) & 31, z = x >> 6;
  return make_int2((z >> 1) * 4 + (l >> 3), (l & 7) * 4 + (z & 1) * 2 + (x & 1));
}
__device__ __forceinline__ int2 blk_je(int x) {  // (j, i) of exponent index x
  const int l = (x >> 2) & 31;
  return make_int2((x >> 7) * 4 + (l >> 3), (l & 7) * 4 + (x & 3));
}

// ---------------------------------------------------------- tile inverses
// One CTA per (tile, recursion), one warp per source column: thread (i, j)
// forms L(j, i) and Dc(j, i) of row j; then warp k forms column k of M by
// forward substitution, M(:, k) = e_k + L M(:, k): lane j holds M(j, k),
// and step s adds L(j, s) M(s, k) once M(s, k) is final (s >= k).
template <int MODE, bool BWD, bool RC, bool PBC>
__device__ void tile_inverse_body(const Workspace &w, int t, const unsigned long long *T63,
                                  unsigned long long (*Lk)[TILE + 1], int (*Le)[TILE + 1],
                                  unsigned long long (*Ok)[TILE + 1], int (*Oe)[TILE + 1]) {
  const int lane = threadIdx.x & 31, i = threadIdx.x >> 5;
  const int r0 = t * TILE, row = r0 + lane;
  xk L{1ull << 63, XZERO_E}, D{1ull << 63, XZERO_E};
  if (row < w.N) {
    const xd c = xnorm_int(chain_coef<BWD>(w, row));
    RowFactors<MODE, BWD, RC, PBC> f;
    f.load(w, row);
    if (i < lane) L = f.k(w, c, r0 + 1 + i, T63);
    if (r0 - 31 + i >= 0) D = f.k(w, c, r0 - 31 + i, T63);
  }
  Lk[i][lane] = L.m;
  Le[i][lane] = L.e;
  Ok[lane][i] = D.m;
  Oe[lane][i] = D.e;
  __syncthreads();
  const size_t base = tile_block_base(w, BWD, t);
  const int x = threadIdx.x;
  const int2 pk = blk_jk(x), pe = blk_je(x);
  w.bk[base + x] = Ok[pk.x][pk.y];  // Dc
  w.be[base + x] = Oe[pe.x][pe.y];
  __syncthreads();
  const int k = i;
  xi acc{1ull << 62, lane == k ? 0 : XZERO_E};
  for (int s = k; s < TILE - 1; ++s) {
    xi y;
    y.m = __shfl_sync(0xffffffffu, acc.m, s);
    y.e = __shfl_sync(0xffffffffu, acc.e, s);
    acc = xi_fma<false>(acc, Lk[s][lane], Le[s][lane], y);
  }
  Ok[lane][k] = acc.m << 1;  // the K format: the same value
  Oe[lane][k] = acc.e;
  __syncthreads();
  w.bk[base + TILE2 + x] = Ok[pk.x][pk.y];  // M
  w.be[base + TILE2 + x] = Oe[pe.x][pe.y];
}

template <int MODE, bool RC>
__global__ void __launch_bounds__(TINV_THREADS) tile_inverse_kernel(Workspace w) {
  __shared__ unsigned long long Lk[TILE][TILE + 1], Ok[TILE][TILE + 1];
  __shared__ int Le[TILE][TILE + 1], Oe[TILE][TILE + 1];
  __shared__ unsigned long long T63[256];
  if (RC) {
    pairg::table_init(T63);
    __syncthreads();
  }
  pdl_wait();
  pdl_trigger();  // the recursions wait for this grid's completion
  const int t = blockIdx.x;
  const bool bwd = blockIdx.y != 0;
  if (w.pbc) {
    if (bwd) tile_inverse_body<MODE, true, RC, true>(w, t, T63, Lk, Le, Ok, Oe);
    else tile_inverse_body<MODE, false, RC, true>(w, t, T63, Lk, Le, Ok, Oe);
  } else {
    if (bwd) tile_inverse_body<MODE, true, RC, false>(w, t, T63, Lk, Le, Ok, Oe);
    else tile_inverse_body<MODE, false, RC, false>(w, t, T63, Lk, Le, Ok, Oe);
  }
}

// ------------------------------------------------------------ recursions
// This lane's four entries (row 4 wid + lane/8, sources 4 (lane%8) .. +3) of
// a tile block in shared memory (the blk_k / blk_e layout).
__device__ __forceinline__ void load_row4(const unsigned long long *bk, const int *be, int wid, int lane,
                                          unsigned long long (&k)[4], int (&e)[4]) {
  const ulonglong2 a = *(const ulonglong2 *)(bk + (((wid * 2 + 0) * 32 + lane) << 1));
  const ulonglong2 b = *(const ulonglong2 *)(bk + (((wid * 2 + 1) * 32 + lane) << 1));
  const int4 q = *(const int4 *)(be + ((wid * 32 + lane) << 2));
  k[0] = a.x; k[1] = a.y; k[2] = b.x; k[3] = b.y;
  e[0] = q.x; e[1] = q.y; e[2] = q.z; e[3] = q.w;
}

// Reduce an xsum over the eight lanes of a row (lane bits 0..2).
__device__ __forceinline__ xsum row_reduce(xsum s) {
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    xsum u;
    u.s = __shfl_xor_sync(0xffffffffu, s.s, o);
    u.E = __shfl_xor_sync(0xffffffffu, s.E, o);
    s = xsum_add(s, u);
  }
  return s;
}

// Recompute mode: the 8 factors H(sb + i, r) of one bulk task (rows past N
// get extended zeros; sources below 0 meet X^{-1}'s zeros and read H(0, r)).
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
    for (int i = 0; i < 8; ++i) m[i] = re.h(w, max(sb + i, 0), T63, e[i]);
  } else {
    RowEnds<MODE, BWD, false> re;
    re.load(w, r);
#pragma unroll
    for (int i = 0; i < 8; ++i) m[i] = re.h(w, max(sb + i, 0), T63, e[i]);
  }
}

// MODE: precision form (the stored-factor kernels serve BPIMD_MIXED with the
// BPIMD_FP64 code: the same float64-mantissa layout); RC: recompute mode, H
// formed from the endpoint copies wherever it is used.
template <int MODE, bool BWD, int NHELP, bool RC>
__device__ void run_chain(const Workspace &w, unsigned char *smem_raw, double *V_B) {
  constexpr bool MIXED = MODE == BPIMD_MIXED32;  // float32 factors and bulk products
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const int N = w.N, NT = w.NT;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const M_t *gm = (const M_t *)chain_gm<BWD>(w);
  const int *ge = chain_ge<BWD>(w);
  double *gYm = BWD ? w.ybm : w.yfm;
  int *gYe = BWD ? w.ybe : w.yfe;

  if (rank == 0) {
    LeadSmem &sm = *(LeadSmem *)smem_raw;
    for (int v = tid; v < YRING; v += blockDim.x) { sm.Ym[v] = 1ull << 62; sm.Ye[v] = XZERO_E; }
    if (tid < 2 * TILE) { sm.cAm[tid] = 1ull << 62; sm.cAe[tid] = XZERO_E; }
    if (tid < 2) {
      mbar_init(smem_addr(&sm.cabar[tid]), 1);
      mbar_fence_init();
    }
    if (tid >= 32 && tid < 32 + OPBUF) mbar_init(smem_addr(&sm.opbar[tid - 32]), 32);  // one per loader lane
    if (tid == 64) mbar_init(smem_addr(&sm.never), 1);
    if (tid == 0) {
      sm.aborted = 0;
      sm.Ym[0] = 1ull << 62; sm.Ye[0] = 0;
    }
    // phase warps: rows j = 4 wid + (lane >> 3), sources 4g .. 4g+3 (g = lane & 7)
    const int g = lane & 7, jrow = 4 * wid + (lane >> 3);
    // loader warp: tile tt's Dc and M (24 KB, contiguous in both places) into
    // buffer tt % OPBUF, 16-byte copies, completion counted on opbar
    auto copy_tile = [&](int tt) {
      const int b = tt % OPBUF;
      const size_t base = tile_block_base(w, BWD, tt);
      for (int i = lane; i < TILE2; i += 32) cp_async16(smem_addr(sm.Bk[b] + 2 * i), w.bk + base + 2 * i);
      for (int i = lane; i < TILE2 / 2; i += 32) cp_async16(smem_addr(sm.Be[b] + 4 * i), w.be + base + 4 * i);
      cp_async_arrive(smem_addr(&sm.opbar[b]));
    };
    __syncthreads();  // the operand mbarriers are initialised
    // Everything above touches shared memory only, so it runs, and the cluster
    // barrier starts, while the tile inverses are still being formed; global
    // memory is accessed only after the wait for that grid.
    cluster_arrive();
    pdl_wait();
    if (tid == 0) {
      gYm[0] = 1.0; gYe[0] = 0;
      if (!BWD) w.C[0] = 0.0;
    }
    if (wid == LOADER_WARP)
      for (int tt = 0; tt < OPBUF && tt < NT; ++tt) copy_tile(tt);
    cluster_wait();  // every mbarrier of the cluster is initialised

    double carry = 0.0;    // prefix-sum warp (forward): running reduced prefix sum C'
    long long ncarry = 0;  // and the running sum of the exponent parts n
    if (wid < LEAD_WARPS) {
      // the error-path test: a wait that expires before the first tile
      if (!BWD && w.test_timeout) handoff_wait(smem_addr(&sm.never), 0, w.status, (volatile int *)&sm.aborted);
      for (int t = 0; t < NT; ++t) {
        const int buf = t % OPBUF;
        handoff_wait(smem_addr(&sm.opbar[buf]), (t / OPBUF) & 1, w.status, (volatile int *)&sm.aborted);
        unsigned long long Dk[4], Mk[4];
        int De[4], Me[4];
        load_row4(sm.Bk[buf], sm.Be[buf], wid, lane, Dk, De);
        load_row4(sm.Bk[buf] + TILE2, sm.Be[buf] + TILE2, wid, lane, Mk, Me);
        xi X[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int v = (t * TILE - 31 + 4 * g + q) & (YRING - 1);
          X[q] = xi{sm.Ym[v], sm.Ye[v]};
        }
        // phase 1: b_j = c_j A_j + sum_i Dc(j, i) X^{t-1}_i   (33 terms: S = 6).
        // The 32 Dc terms are summed and reduced while c A^t may still be on its
        // way from the tile's owner; c A^t (tile 0 has none: an extended zero)
        // joins the row sum after the reduction, so only one addition follows
        // its arrival.
        const xsum sd = row_reduce(xsum_dot<6, 4>(Dk, De, X, 0, 2 * XZERO_E));
        if (t >= 1) handoff_wait(smem_addr(&sm.cabar[t & 1]), ((t - 1) >> 1) & 1, w.status, (volatile int *)&sm.aborted);
        if (g == 0) {
          const xsum ca{sm.cAm[(t & 1) * TILE + jrow] >> 6, sm.cAe[(t & 1) * TILE + jrow]};
          const xi b = xsum_fin<6>(xsum_add(sd, ca));
          sm.bm[jrow] = b.m;
          sm.be[jrow] = b.e;
        }
        asm volatile("bar.sync %0, %1;" ::"n"(BAR_PHASE), "n"(LEAD_WARPS * 32) : "memory");
        // phase 2: X^t_j = sum_{i <= j} M(j, i) b_i   (32 terms: S = 5)
        xi B[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) B[q] = xi{sm.bm[4 * g + q], sm.be[4 * g + q]};
        const xsum s2 = row_reduce(xsum_dot<5, 4>(Mk, Me, B, 0, 2 * XZERO_E));
        // every lane of the row holds the same sum (the butterfly pairs the
        // same partial sums in every lane): lane g == 0 keeps X^t_j in the ring
        const xi x = xsum_fin<5>(s2);
        if (g == 0) {
          const int v = (t * TILE + 1 + jrow) & (YRING - 1);
          sm.Ym[v] = x.m;
          sm.Ye[v] = x.e;
        }
        asm volatile("bar.sync %0, %1;" ::"n"(BAR_TILE), "n"(BAR_TILE_THREADS) : "memory");
      }
    } else if (wid == EXPORT_WARP) {
      // off the phase warps, lane j takes row j of each finished tile t: Y to
      // global memory, and X^t to every bulk CTA that still has work in
      // period t+1 (slot t mod XRING; lane 0 adds the expected bytes)
      const HelperHead *hh0 = (const HelperHead *)smem_raw;  // offsets of the bulk CTAs' X slots
      for (int t = 0; t < NT; ++t) {
        asm volatile("bar.sync %0, %1;" ::"n"(BAR_TILE), "n"(BAR_TILE_THREADS) : "memory");
        const int v = t * TILE + lane + 1;
        const xi x{sm.Ym[v & (YRING - 1)], sm.Ye[v & (YRING - 1)]};
        if (!*(volatile int *)&sm.aborted) {
          const int slot = t % XRING;
          const unsigned lm = smem_addr(&hh0->Xm[slot][lane]), le = smem_addr(&hh0->Xe[slot][lane]),
                         lb = smem_addr(&hh0->xbar[slot]);
          for (int hh = 1; hh <= NHELP; ++hh) {
            if (bulk_first_tile(t + 1, hh - 1, NHELP) >= NT) continue;  // warp-uniform
            const unsigned rb = cluster_addr(lb, hh);
            st_async_u64(cluster_addr(lm, hh), x.m, rb);
            st_async_u32(cluster_addr(le, hh), (unsigned)x.e, rb);
            if (lane == 0) mbar_arrive_expect_remote(rb, TILE * (sizeof(unsigned long long) + sizeof(int)));
          }
        }
        if (v <= N) {
          const xd y = xi_to_xd(x);
          gYm[v] = y.m;
          gYe[v] = y.e;
        }
      }
    } else if (wid == LOADER_WARP) {
      // buffer t % OPBUF is free once tile t is done: copy tile t + OPBUF into it
      for (int t = 0; t < NT; ++t) {
        asm volatile("bar.sync %0, %1;" ::"n"(BAR_TILE), "n"(BAR_TILE_THREADS) : "memory");
        if (t + OPBUF < NT) copy_tile(t + OPBUF);
      }
    } else if (!BWD && wid == PREFIX_WARP) {
      for (int t = 0; t < NT; ++t) prefix_tile(w, t, carry, ncarry);
    }
    // every hand-off this CTA takes part in is complete: release the bulk CTAs
    cluster_arrive();
    pdl_trigger();  // the probability pass may launch during the epilogue
    if (!BWD) {
      // V^{[1,N]} = C'[N] - (ln(y_N) - n ln 2)/beta, normaliser 1/(N y_N), alpha_a = y_a/(N y_N)
      if (wid == PREFIX_WARP && lane == 0) { sm.misc[0] = carry; sm.nsum = ncarry; }
      __syncthreads();
      const xd yN = xi_to_xd(xi{sm.Ym[N & (YRING - 1)], sm.Ye[N & (YRING - 1)]});
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
    HelperHead &hd = *(HelperHead *)smem_raw;
    unsigned char *p = smem_raw + sizeof(HelperHead);
    const int lt_max = helper_tiles(NT, NHELP);
    const int nwarps = (int)(blockDim.x >> 5);
    unsigned long long *Am = (unsigned long long *)p; p += sizeof(unsigned long long) * lt_max * TILE;
    unsigned long long *Pm = (unsigned long long *)p; p += sizeof(unsigned long long) * 4 * lt_max * TILE;
    double *Cm = (double *)p; p += sizeof(double) * lt_max * TILE;
    int *Ae = (int *)p; p += sizeof(int) * lt_max * TILE;
    int *Pe = (int *)p; p += sizeof(int) * 4 * lt_max * TILE;
    int *Ce = (int *)p; p += sizeof(int) * lt_max * TILE;
    unsigned long long *T63 = (unsigned long long *)p;  // recompute mode
    const int h = (int)rank - 1;  // owns row tiles T with T mod NHELP == h
    auto first_tile = [&](int t) { return bulk_first_tile(t, h, NHELP); };
    auto units = [&](int t) {
      const int T0 = first_tile(t);
      return T0 < NT ? (NT - 1 - T0) / NHELP + 1 : 0;
    };
    // this warp's tasks in order: period t, task k (row tile first_tile(t) +
    // (k/4) NHELP, sources 32t-31 + 8 (k%4) .. +7), k = wid, wid + nwarps, ...
    // (units never grow with t: a warp without a task in period t has none later)
    auto advance = [&](int &t, int &k) {
      while (t < NT && k >= 4 * units(t)) {
        ++t;
        k = wid;
        if (t < NT && wid >= 4 * units(t)) t = NT;
      }
    };
    // stored factors of task (t, k): rows past N hold extended zeros; sources
    // below 0 meet X^{-1}'s zeros and read H(0, r)
    auto load_factors = [&](int t, int k, M_t(&m)[8], int(&e)[8]) {
      const int r = (first_tile(t) + (k >> 2) * NHELP) * TILE + lane;
      const int sb = t * TILE - 31 + 8 * (k & 3);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const size_t gi = hidx(max(sb + i, 0), r);
        m[i] = __ldg(gm + gi);
        e[i] = __ldg(ge + gi);
      }
    };
    if (tid < TILE) {  // X^{-1} = (0, ..., 0, Y_0)
      hd.Xm[XRING][tid] = 1ull << 62;
      hd.Xe[XRING][tid] = tid == TILE - 1 ? 0 : XZERO_E;
    }
    if (tid < XRING) {
      mbar_init(smem_addr(&hd.xbar[tid]), 1);
      mbar_fence_init();
    }
    if (tid == 0) hd.aborted = 0;
    if (RC) pairg::table_init(T63);  // from constant memory
    // as in the lead: the barrier starts before the wait for the tile inverses,
    // and global memory is read only after it
    cluster_arrive();
    pdl_wait();
    for (int q = tid; q < lt_max * TILE; q += blockDim.x) {
      Am[q] = 1ull << 62;
      Ae[q] = XZERO_E;
      const int r = ((q >> 5) * NHELP + h) * TILE + (q & 31);  // owned row of local tile q/32
      const xd c = r < N ? chain_coef<BWD>(w, r) : xd{1.0, XZERO_E};
      Cm[q] = c.m;
      Ce[q] = c.e;
    }
    int nt = 0, nk = wid;  // this warp's next task
    advance(nt, nk);
    M_t fm[8];             // its factors, loaded one task ahead (stored mode)
    int fe[8];
    if (!RC && nt < NT) load_factors(nt, nk, fm, fe);
    __syncthreads();  // the rows' sums and coefficients are initialised
    cluster_wait();   // every mbarrier of the cluster is initialised
    const LeadSmem *L0 = (const LeadSmem *)smem_raw;  // offsets of the lead's hand-off slots
    // unit u of period t: add the four quarter partials to the rows' sums A; the
    // owner of tile t+1 hands c A of the finished tile to the lead (one warp)
    auto combine = [&](int t, int T0, int u) {
      const int T = T0 + u * NHELP, lt = T / NHELP;
      xi acc{Am[lt * TILE + lane], Ae[lt * TILE + lane]};
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = xi_add(acc, xi{Pm[(4 * u + q) * TILE + lane], Pe[(4 * u + q) * TILE + lane]});
      Am[lt * TILE + lane] = acc.m;
      Ae[lt * TILE + lane] = acc.e;
      if (T == t + 1 && !*(volatile int *)&hd.aborted) {
        const int r = T * TILE + lane;
        const xi ca = (r < N) ? xi_mul(acc, xd{Cm[lt * TILE + lane], Ce[lt * TILE + lane]}) : xi{1ull << 62, XZERO_E};
        const int slot = (t + 1) & 1;
        const unsigned rb = cluster_addr(smem_addr(&L0->cabar[slot]), 0);
        st_async_u64(cluster_addr(smem_addr(&L0->cAm[slot * TILE + lane]), 0), ca.m, rb);
        st_async_u32(cluster_addr(smem_addr(&L0->cAe[slot * TILE + lane]), 0), (unsigned)ca.e, rb);
        if (lane == 0) mbar_arrive_expect_remote(rb, TILE * (sizeof(unsigned long long) + sizeof(int)));
      }
    };
    for (int t = 0; t < NT; ++t) {
      const int nunits = units(t);
      if (nunits == 0) break;  // and none later
      const int T0 = first_tile(t);
      const int xs = t == 0 ? XRING : (t - 1) % XRING;  // X^{t-1}
      if (t >= 1) handoff_wait(smem_addr(&hd.xbar[xs]), ((t - 1) / XRING) & 1, w.status, (volatile int *)&hd.aborted);
      const bool crit = T0 == t + 1;  // this CTA owns the tile the lead needs next
      const unsigned long long *Xm = hd.Xm[xs];
      const int *Xe = hd.Xe[xs];
      for (int k = wid; k < 4 * nunits; k += nwarps) {
        const int u = k >> 2, q = k & 3;
        const int r = (T0 + u * NHELP) * TILE + lane;
        const int sb = t * TILE - 31 + 8 * q;
        M_t m[8];
        int e[8];
        if (RC) {
          bulk_factors_rc<MODE, BWD>(w, r, sb, T63, m, e);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) { m[i] = fm[i]; e[i] = fe[i]; }
          nk += nwarps;
          advance(nt, nk);
          if (nt < NT) load_factors(nt, nk, fm, fe);
        }
        xi y[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) y[i] = xi{Xm[8 * q + i], Xe[8 * q + i]};
        xi part;
        if constexpr (MIXED) {
          float sacc = 0.0f;
          int E = XZERO_E;
#pragma unroll
          for (int i = 0; i < 8; ++i) fmerge(sacc, E, xi_mant_float(y[i]) * m[i], e[i] + y[i].e);
          part = xi_from_float(sacc, E);
        } else {
          unsigned long long kk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) kk[i] = mant53(m[i]) << 11;
          part = xsum_fin<3>(xsum_dot<3, 8>(kk, e, y, 0, 2 * XZERO_E));
        }
        Pm[k * TILE + lane] = part.m;
        Pe[k * TILE + lane] = part.e;
        if (crit && k < 4) {
          // the four quarters of the critical tile t+1 (tasks 0..3, the first
          // task of warps 0..3) are done: hand it off before the other tasks
          asm volatile("bar.sync %0, %1;" ::"n"(BAR_CRIT), "n"(4 * 32) : "memory");
          if (wid == 0) combine(t, T0, 0);
        }
      }
      __syncthreads();
      // combine the four quarters of each other owned row tile in a fixed order
      for (int u = wid + (crit ? 1 : 0); u < nunits; u += nwarps) combine(t, T0, u);
      __syncthreads();  // the partial sums are read: the next period may overwrite them
    }
    cluster_arrive();
  }
  // No CTA leaves while a hand-off into its shared memory may be in flight:
  // each arrived above once its own waits were over.  After an expired wait
  // a hand-off may still be on its way: give it time to land.
  cluster_wait();
  if (*(volatile int *)w.status & ST_TIMEOUT)
    for (int i = 0; i < 200; ++i) __nanosleep(1000);
}

// Cluster size CL (CTAs per recursion) is given at launch; blocks [0, CL) run
// the forward recursion, [CL, 2 CL) the backward one.
template <int MODE, int CL, bool RC>
__global__ void __launch_bounds__(CHAIN_THREADS, 1) chain_kernel(Workspace w, double *V_B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // run_chain waits for the preceding grid (griddepcontrol.wait) once its
  // shared-memory set-up is done, before its first global-memory access
  if (blockIdx.x < CL) run_chain<MODE, false, CL - 1, RC>(w, smem_raw, V_B);
  else run_chain<MODE, true, CL - 1, RC>(w, smem_raw, V_B);
}

constexpr size_t chain_smem_bytes(int N, int CL, bool RC) {
  const size_t lead = sizeof(LeadSmem);
  const size_t help = helper_smem_bytes((N + TILE - 1) / TILE, CL - 1, RC);
  return lead > help ? lead : help;
}
// the largest N of each mode: stored factors up to BPIMD_STORE_MAX_N
constexpr int chain_max_n(bool RC) { return RC ? CHAIN_MAX_N : BPIMD_STORE_MAX_N; }
static_assert(chain_smem_bytes(chain_max_n(true), CHAIN_CLUSTER, true) <= 227 * 1024 &&
                  chain_smem_bytes(chain_max_n(false), CHAIN_CLUSTER, false) <= 227 * 1024,
              "recursion state for the largest N must fit in shared memory");
constexpr int CHAIN_CLUSTER_LARGE = 16;
constexpr int LARGE_CLUSTER_MIN_NT = 9;  // N > 256: the bulk work would set the pace with 7 bulk CTAs

template <int MODE, bool RC>
cudaError_t launch_tile_inverse(const Workspace &w, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(w.NT, 2);
  cfg.blockDim = dim3(TINV_THREADS);
  cfg.dynamicSmemBytes = TINV_PAD_SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tile_inverse_kernel<MODE, RC>, w);
}

template <int MODE, int CL, bool RC>
cudaError_t launch_chain_cluster(const Workspace &w, double *V_B, cudaStream_t s) {
  cudaError_t e = launch_tile_inverse<MODE, RC>(w, s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * CL);
  cfg.blockDim = dim3(CHAIN_THREADS);
  cfg.dynamicSmemBytes = chain_smem_bytes(w.N, CL, RC);
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
static_assert(CHAIN_THREADS % 32 == 0 && CHAIN_THREADS / 32 > PREFIX_WARP && CHAIN_THREADS / 32 <= 32,
              "the lead needs its phase, export and prefix warps; a bulk CTA has at most 32 Y slots");

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
  const int bytes = (int)chain_smem_bytes(chain_max_n(RC), CL, RC);
  cudaError_t e =
      cudaFuncSetAttribute(chain_kernel<MODE, CL, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tile_inverse_kernel<MODE, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TINV_PAD_SMEM);
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
  cfg.dynamicSmemBytes = chain_smem_bytes(chain_max_n(false), CL, false);
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
  if (!w.blocks) return cudaErrorInvalidValue;  // no tile-inverse storage in this workspace
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
