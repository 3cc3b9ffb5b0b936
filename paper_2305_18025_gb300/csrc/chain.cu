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
// latency and a warp has one float64 instruction in flight at a time; a
// release/acquire hand-off between warps inside a step costs far more than
// the step itself; a cluster barrier costs ~360 cycles and a distributed
// shared-memory access ~215.  So the rows are processed in tiles of 32 and
//   * all intra-tile work stays in one warp of the lead CTA (cluster rank 0):
//     warp 0 runs the 32 dependent steps of row tile t.  Lane j holds
//     c_r * (partial row sum) of row 32t+j and the partial sum of row
//     32(t+1)+j.  A step is one float64 FMA on the current row (the
//     dependency chain: acc_j += K(i, j) y_i, exponents aligned with integer
//     operations on the double's bits), one FMA on the next tile's row (off
//     the chain), and a shuffle that broadcasts the new Y;
//   * twelve other lead warps (none on warp 0's sub-partition) stage, for
//     tile t+1, the block of H from source tile t+1 to the rows of tile t+2
//     and the diagonal block pre-scaled by c; one more lead warp of the
//     forward cluster forms the prefix sums C, one tile of 32 per period;
//   * the O(N^2) bulk runs on the seven other CTAs of the cluster: row tile T
//     belongs to CTA 1 + T mod 7, which keeps its rows' partial sums in its
//     own shared memory.  In period t each of them adds source tile t-1 to
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
// dependent steps and the tile hand-offs stay float64.
#include <cooperative_groups.h>
#include <type_traits>

#include "bpimd_internal.cuh"

namespace cg = cooperative_groups;

namespace bpimd {
namespace {

constexpr int NHELP = CHAIN_CLUSTER - 1;  // bulk CTAs per recursion
constexpr int YRING = 128;                // Y values kept in the lead (4 tiles)
constexpr int BLK = 32 * 33;              // padded 32 x 32 block in shared memory

__device__ __forceinline__ size_t hidx(int src, int row) {
  const int t = row >> 5, s = src >> 5;
  return ((size_t)(t * (t + 1) / 2 + s) << 10) + ((src & 31) << 5) + (row & 31);
}

// x * 2^k for k <= 0 by integer arithmetic on the exponent field (x >= 0 normal
// or zero); 0 when the result would leave the normal range.
__device__ __forceinline__ double scale_nonpos(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)(b >> 52);  // sign bit is 0
  return (ex + k <= 0) ? 0.0 : __longlong_as_double(b + ((long long)k << 52));
}

// acc + K * y, branch-free, for the dependency chain.  Operands are extended
// numbers whose mantissas are normal doubles in [1, 2^60) (an extended zero is
// carried as mantissa 1 with exponent XZERO_E, i.e. 2^-536870912).  Both
// operands are scaled by 2^k, k <= 0 clamped at -1000, by adding k to the
// exponent field of the high word: a clamped operand is below 2^-900 of the
// other and cannot change the float64 sum.  One float64 FMA, five integer ops.
__device__ __forceinline__ xd fma_chain(xd acc, double km, int ke, xd y) {
  const int pe = ke + y.e;
  const int E = max(acc.e, pe);
  const int k1 = max(pe - E, -1000), k2 = max(acc.e - E, -1000);
  const double ks = __hiloint2double(__double2hiint(km) + k1 * (1 << 20), __double2loint(km));
  const double as = __hiloint2double(__double2hiint(acc.m) + k2 * (1 << 20), __double2loint(acc.m));
  return xd{fma(ks, y.m, as), E};
}

// Explicit shared-memory loads (32-bit shared-window addresses).
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ double lds_f64(unsigned a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_f32(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int lds_s32(unsigned a) {
  int v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

// Normalise with integer ops only (m > 0 normal, or 0).
__device__ __forceinline__ xd xnorm_int(xd a) {
  const long long b = __double_as_longlong(a.m);
  if (b <= 0) return xd{0.0, XZERO_E};
  const int ex = (int)(b >> 52);
  return xd{__longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL), a.e + ex - 1023};
}

// a * b with integer normalisation (one float64 multiply).
__device__ __forceinline__ xd xmul_int(xd a, xd b) { return xnorm_int(xd{a.m * b.m, a.e + b.e}); }

// Round the significand of a positive normal double to a float in [1,2] with
// integer ops (no float64 conversion unit); the binary exponent is dropped.
__device__ __forceinline__ float mant_to_float(double m) {
  const long long b = __double_as_longlong(m);
  const long long frac = b & 0x000fffffffffffffLL;
  return __int_as_float((int)((frac + (1LL << 28)) >> 29) + 0x3f800000);
}

// Mantissa in [1,2) as a 53-bit integer (implicit bit set), from a double or a float.
__device__ __forceinline__ unsigned long long mant53(double m) {
  return ((unsigned long long)__double_as_longlong(m) & 0xFFFFFFFFFFFFFull) | (1ull << 52);
}
__device__ __forceinline__ unsigned long long mant53(float m) {
  return ((unsigned long long)((unsigned)__float_as_int(m) & 0x7FFFFFu) | 0x800000ull) << 29;
}

// c * h for extended numbers with mantissas in [1,2): the 53 x 53-bit mantissa
// product on the integer pipe (truncated to 52 fraction bits, error below one
// unit in the last place), so that staging issues no float64 instruction.
template <typename M_t>
__device__ __forceinline__ xd mul_mant(xd c, M_t hm, int he) {
  const unsigned long long hi = __umul64hi(mant53(c.m) << 11, mant53(hm) << 11);  // in [2^62, 2^64)
  const int sh = (int)(hi >> 63);
  const unsigned long long frac = (hi >> (10 + sh)) & 0xFFFFFFFFFFFFFull;
  return xd{__longlong_as_double((long long)(frac | 0x3FF0000000000000ull)), c.e + he + sh};
}

// A positive normal float (or 0) as a double, with integer operations.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned b = (unsigned)__float_as_int(f);
  if (b < 0x00800000u) return 0.0;
  return __longlong_as_double(((long long)((b >> 23) + 896) << 52) | ((long long)(b & 0x7FFFFFu) << 29));
}

// a + b for extended numbers with positive normal (or zero) mantissas: the
// smaller operand is aligned by integer arithmetic, then one float64 add.
__device__ __forceinline__ xd xadd_int(xd a, xd b) {
  const int E = max(a.e, b.e);
  return xd{scale_nonpos(a.m, max(a.e - E, -1100)) + scale_nonpos(b.m, max(b.e - E, -1100)), E};
}

// Online-max merge of a float partial sum (s * 2^E) with a term x * 2^e.
__device__ __forceinline__ void fmerge(float &s, int &E, float x, int e) {
  const int En = max(E, e);
  s = fmaf(x, pow2f_nonpos(e - En), s * pow2f_nonpos(E - En));
  E = En;
}

// Shared memory of the lead CTA.
struct LeadSmem {
  double Kdm[2 * BLK];  // c-scaled diagonal blocks (double buffer)
  double Hom[2 * BLK];  // H(source of tile t, row of tile t+1) (double buffer; MIXED: floats)
  double Ym[YRING];     // Y_v at v mod YRING
  double Am[2 * TILE];  // bulk row sums of the next tile, written by its owner
  double misc[4];       // end of the forward recursion: C[N], 1/(N y_N) mantissa
  int Kde[2 * BLK];
  int Hoe[2 * BLK];
  int Ye[YRING];
  int Ae[2 * TILE];
  int misci[4];         // 1/(N y_N) exponent
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

__host__ __device__ constexpr int helper_tiles(int NT) { return (NT + NHELP - 1) / NHELP; }

__host__ __device__ constexpr size_t helper_smem_bytes(int NT) {
  return (size_t)helper_tiles(NT) * TILE * (sizeof(double) + sizeof(int)) * 5 +
         (size_t)32 * 8 * (sizeof(double) + sizeof(int));
}

template <bool MIXED, bool BWD>
__device__ void run_chain(const Workspace &w, unsigned char *smem_raw, double *V_B) {
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const int N = w.N, NT = w.NT;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // H(src, row) in this recursion's own coordinates (both copies share the layout)
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const void *gm = BWD ? w.gbm : w.gm;
  const int *ge = BWD ? w.gbe : w.ge;
  auto coef = [&](int row) -> xd {
    if (!BWD) return xd{__ldg(w.ccm + row), __ldg(w.cce + row)};
    if (row >= N - 1) return xd{1.0, 0};
    return xd{__ldg(w.ccm + N - 2 - row), __ldg(w.cce + N - 2 - row)};
  };
  double *gYm = BWD ? w.ybm : w.yfm;
  int *gYe = BWD ? w.ybe : w.yfe;
  LeadSmem *lead_local = (LeadSmem *)smem_raw;
  // the lead's shared memory as seen from this CTA (distributed shared memory)
  LeadSmem *lead = cluster.map_shared_rank(lead_local, 0);

  if (rank == 0) {
    LeadSmem &sm = *lead_local;
    // Staging issues no float64 instruction (the SM's float64 pipe belongs to
    // the dependency chain).  Pairs outside src <= row < N hold the extended
    // zero 1 * 2^XZERO_E; loads are coalesced along rows and issued before use.
    // Staging warps are the lead's warps off warp 0's sub-partition (warp id
    // not a multiple of 4), numbered q = 0, 1, ...: q < 8 stage four rows each
    // of the diagonal block, 8 <= q < 12 eight rows each of the off-diagonal
    // block, q == 12 forms the prefix sums (forward recursion).
    // H(tt*32+i, (tt+1)*32+lane) for i in [i0, i0+8), as stored (float for MIXED)
    auto stage_offdiag = [&](int tt, int buf, int i0) {
      const int srcbase = tt * TILE, row = tt * TILE + TILE + lane;
      M_t *dm = (M_t *)(sm.Hom + buf * BLK);
      int *de = sm.Hoe + buf * BLK;
#pragma unroll
      for (int i = i0; i < i0 + 8; ++i) {
        const int src = srcbase + i;
        M_t m = (M_t)1.0;
        int e = XZERO_E;
        if (row < N) {
          const size_t gi = hidx(src, row);
          m = __ldg((const M_t *)gm + gi);
          e = __ldg(ge + gi);
        }
        dm[i * 33 + lane] = m;
        de[i * 33 + lane] = e;
      }
    };
    // the diagonal block of tile tt, K = c_row * H (float64 mantissas), rows
    // i in [i0, i0+4)
    auto stage_diag = [&](int tt, int buf, int i0) {
      const int r0 = tt * TILE, row = r0 + lane;
      double *dm = sm.Kdm + buf * BLK;
      int *de = sm.Kde + buf * BLK;
      const xd c = (row < N) ? xnorm_int(coef(row)) : xd{1.0, 0};
#pragma unroll
      for (int i = i0; i < i0 + 4; ++i) {
        const int src = r0 + i;
        M_t m = (M_t)1.0;
        int e = XZERO_E;
        if (row < N && src <= row) {
          const size_t gi = hidx(src, row);
          m = __ldg((const M_t *)gm + gi);
          e = __ldg(ge + gi);
        }
        const xd k = mul_mant<M_t>(c, m, e);
        dm[i * 33 + lane] = k.m;
        de[i * 33 + lane] = k.e;
      }
    };
    if (tid < 2 * TILE) { sm.Am[tid] = 0.0; sm.Ae[tid] = XZERO_E; }
    if (tid == 0) { sm.Ym[0] = 1.0; sm.Ye[0] = 0; gYm[0] = 1.0; gYe[0] = 0; }
    if (!BWD && tid == 0) w.C[0] = 0.0;
    const int q = (wid & 3) ? wid - (wid >> 2) - 1 : -1;  // staging index (-1: SMSP of warp 0)
    if (q >= 0 && q < 8) stage_diag(0, 0, 4 * q);
    if (q >= 8 && q < 12) stage_offdiag(0, 0, 8 * (q - 8));
    cluster.sync();

    xd nxt{1.0, XZERO_E};  // warp 0: partial sum of row 32(t+1)+lane over source tile t
    xd cnext{1.0, 0};      // warp 0: coefficient of its row in the coming tile
    if (wid == 0 && lane < N) cnext = coef(lane);
    double carry = 0.0;    // warp 3 (forward): running prefix sum
    for (int t = 0; t < NT; ++t) {
      const int r0 = t * TILE, buf = t & 1;
      if (wid == 0) {
        // ---------------------------------------------- dependent steps of tile t
        const int row = r0 + lane;
        xd acc{0.0, XZERO_E};
        const xd crow = cnext;
        if (row + TILE < N) cnext = coef(row + TILE);  // prefetch for tile t+1
        if (row < N) {
          acc = xadd_int(xd{sm.Am[buf * TILE + lane], sm.Ae[buf * TILE + lane]}, nxt);
          acc = xmul_int(xnorm_int(acc), crow);  // acc' = c_row * (sum over sources < r0)
        }
        xd ycur{sm.Ym[r0 & (YRING - 1)], sm.Ye[r0 & (YRING - 1)]};
        const double *Kdm = sm.Kdm + buf * BLK, *Hom = sm.Hom + buf * BLK;
        const int *Kde = sm.Kde + buf * BLK, *Hoe = sm.Hoe + buf * BLK;
        if (__double_as_longlong(acc.m) <= 0) acc = xd{1.0, XZERO_E};
        nxt = xd{1.0, XZERO_E};
        float nsum = 0.0f;  // MIXED: the next tile's partial sum in float32
        int nexp = XZERO_E;
        // 32 steps, no branches and no stores: rows past N and finished rows see
        // extended zeros in the staged blocks, and row j's accumulator is final
        // after step j (later steps add at most 2^-1000 of it).  Block entries of
        // step i+1 are loaded (explicit ld.shared) before step i's shuffle.
        const unsigned aKm = smem_addr(Kdm + lane), aKe = smem_addr(Kde + lane), aHe = smem_addr(Hoe + lane);
        const unsigned aHm = MIXED ? smem_addr((const float *)Hom + lane) : smem_addr(Hom + lane);
        double km = lds_f64(aKm), hm = MIXED ? 0.0 : lds_f64(aHm);
        float hf = MIXED ? lds_f32(aHm) : 0.0f;
        int ke = lds_s32(aKe), he = lds_s32(aHe);
#pragma unroll
        for (int i = 0; i < TILE; ++i) {
          double km1 = 0.0, hm1 = 0.0;
          float hf1 = 0.0f;
          int ke1 = 0, he1 = 0;
          if (i + 1 < TILE) {
            km1 = lds_f64(aKm + (i + 1) * 33 * 8);
            if (MIXED) hf1 = lds_f32(aHm + (i + 1) * 33 * 4);
            else hm1 = lds_f64(aHm + (i + 1) * 33 * 8);
            ke1 = lds_s32(aKe + (i + 1) * 33 * 4);
            he1 = lds_s32(aHe + (i + 1) * 33 * 4);
          }
          acc = fma_chain(acc, km, ke, ycur);  // the dependency chain
          // next tile's rows, off the chain (MIXED: float32, no float64 pipe)
          // (ycur.m is a positive normal double, not necessarily in [1,2))
          if (MIXED)
            fmerge(nsum, nexp, mant_to_float(ycur.m) * hf,
                   he + ycur.e + (int)(__double_as_longlong(ycur.m) >> 52) - 1023);
          else nxt = fma_chain(nxt, hm, he, ycur);
          ycur.m = __shfl_sync(0xffffffffu, acc.m, i);
          ycur.e = __shfl_sync(0xffffffffu, acc.e, i);
          km = km1; hm = hm1; hf = hf1; ke = ke1; he = he1;
        }
        if (MIXED) nxt = xd{f2d_int(nsum), nexp};
        if (row < N) {  // Y_{row+1} = final accumulator of row `row`
          const xd yn = xnorm_int(acc);
          sm.Ym[(row + 1) & (YRING - 1)] = yn.m;
          sm.Ye[(row + 1) & (YRING - 1)] = yn.e;
          gYm[row + 1] = yn.m;
          gYe[row + 1] = yn.e;
        }
        nxt = xnorm_int(nxt);
      } else if (q >= 0 && q < 8) {
        if (t + 1 < NT) stage_diag(t + 1, buf ^ 1, 4 * q);
      } else if (q >= 8 && q < 12) {
        if (t + 1 < NT) stage_offdiag(t + 1, buf ^ 1, 8 * (q - 8));
      } else if (!BWD && q == 12) {
        // prefix sums C[i+1] = sum_{q<=i} (E_int_q + link_q), one tile per period
        const int i = r0 + lane;
        double v = (i < N) ? (__ldg(w.Eint + i) + __ldg(w.link + i)) : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const double u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        if (i < N) w.C[i + 1] = carry + v;
        carry += __shfl_sync(0xffffffffu, v, 31);
      }
      cluster.sync();
    }
    if (!BWD) {
      // V^{[1,N]} = C[N] - ln(y_N)/beta, normaliser 1/(N y_N), alpha_a = y_a/(N y_N)
      if (q == 12 && lane == 0) sm.misc[0] = carry;
      __syncthreads();
      if (tid == 0) {
        const xd yN{sm.Ym[N & (YRING - 1)], sm.Ye[N & (YRING - 1)]};
        const double VB = sm.misc[0] - xlog(yN) / w.beta;
        w.scal[0] = VB;
        if (V_B) *V_B = VB;
        const xd inv = xnorm(1.0 / (yN.m * (double)N), -yN.e);
        w.scal[1] = inv.m;
        w.scal_i[0] = inv.e;
        sm.misc[1] = inv.m;
        sm.misci[0] = inv.e;
        if (!isfinite(VB)) atomicOr(w.status, ST_NONFINITE);
      }
      __syncthreads();
      const xd inv{sm.misc[1], sm.misci[0]};
      for (int a = tid; a < N; a += blockDim.x) {
        const xd al = xmul(xd{gYm[a], gYe[a]}, inv);
        if (MIXED) ((float *)w.alm)[a] = (float)al.m;
        else ((double *)w.alm)[a] = al.m;
        w.ale[a] = al.e;
      }
    }
  } else {
    // ------------------------------------------------------------ bulk CTA
    HelperSmem hs;
    unsigned char *p = smem_raw;
    const int lt_max = helper_tiles(NT);
    hs.Am = (double *)p; p += sizeof(double) * lt_max * TILE;
    hs.Pm = (double *)p; p += sizeof(double) * 4 * lt_max * TILE;
    hs.Yd = (double *)p; p += sizeof(double) * 32 * 8;
    hs.Ae = (int *)p; p += sizeof(int) * lt_max * TILE;
    hs.Pe = (int *)p; p += sizeof(int) * 4 * lt_max * TILE;
    hs.Yx = (int *)p;
    const int h = (int)rank - 1;  // owns row tiles T with T mod NHELP == h
    const int nwarps = (int)(blockDim.x >> 5);
    for (int q = tid; q < lt_max * TILE; q += blockDim.x) { hs.Am[q] = 0.0; hs.Ae[q] = XZERO_E; }
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
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              m[i] = __ldg((const float *)gm + gbase + i * 32);
              e[i] = __ldg(ge + gbase + i * 32);
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
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              m[i] = __ldg((const double *)gm + gbase + i * 32);
              e[i] = __ldg(ge + gbase + i * 32) + Yx[i];
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

template <bool MIXED>
__global__ void __cluster_dims__(CHAIN_CLUSTER, 1, 1) __launch_bounds__(CHAIN_THREADS, 1)
    chain_kernel(Workspace w, double *V_B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (blockIdx.x < CHAIN_CLUSTER) run_chain<MIXED, false>(w, smem_raw, V_B);
  else run_chain<MIXED, true>(w, smem_raw, V_B);
}

constexpr size_t chain_smem_bytes(int N) {
  const size_t lead = sizeof(LeadSmem);
  const size_t help = helper_smem_bytes((N + TILE - 1) / TILE);
  return lead > help ? lead : help;
}
static_assert(chain_smem_bytes(CHAIN_MAX_N) <= 227 * 1024, "recursion state for the largest N must fit in shared memory");
static_assert(CHAIN_THREADS % 32 == 0 && CHAIN_THREADS / 32 >= 18 && CHAIN_THREADS / 32 <= 32,
              "the lead needs 13 staging warps off warp 0's sub-partition; a bulk CTA has at most 32 Y slots");

}  // namespace

// Raise the dynamic shared-memory limit of both chain kernels to the maximum
// once per process and device (a host call that must not sit between the
// launches of an evaluation).
cudaError_t prepare_chains() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  const int bytes = (int)chain_smem_bytes(CHAIN_MAX_N);
  e = cudaFuncSetAttribute(chain_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chain_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

cudaError_t launch_chains(const Workspace &w, double *V_B, cudaStream_t s) {
  cudaError_t e = prepare_chains();
  if (e != cudaSuccess) return e;
  const size_t bytes = chain_smem_bytes(w.N);
  if (w.mixed) chain_kernel<true><<<2 * CHAIN_CLUSTER, CHAIN_THREADS, bytes, s>>>(w, V_B);
  else chain_kernel<false><<<2 * CHAIN_CLUSTER, CHAIN_THREADS, bytes, s>>>(w, V_B);
  return cudaGetLastError();
}

}  // namespace bpimd
