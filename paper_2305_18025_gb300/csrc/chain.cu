// Forward and backward potential recursions (one CTA each, run concurrently).
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
// the step itself.  So all intra-tile work stays in one warp:
//   * warp 0 runs the 32 dependent steps of row tile t.  Lane j holds
//     c_r * (partial row sum) of row 32t+j and the partial sum of row
//     32(t+1)+j.  A step is one float64 FMA on the current row (the dependency
//     chain: acc_j += K(i, j) y_i, exponents aligned with integer operations
//     on the double's bits), one FMA on the next tile's row (off the chain),
//     and a shuffle that broadcasts the new Y;
//   * warps 1 and 2 stage, for tile t+1, the block of H from source tile t+1
//     to the rows of tile t+2 and the diagonal block pre-scaled by c;
//   * bulk warps (never on warp 0's sub-partition) add source tile t-1 to the
//     rows of tiles >= t+1; tiles only meet at __syncthreads.
// Each recursion reads H from a copy of the pair factors laid out in its own
// (row, source) coordinates, so all its block loads are coalesced.
// Every value is an extended number m * 2^e (int32 exponent), so no exp/log
// sits on the dependency chain.  MIXED: the bulk products are summed in
// float32 per 32-source tile and added to the float64 row accumulator; the
// dependent steps and the tile hand-offs stay float64.
#include "bpimd_internal.cuh"

namespace bpimd {
namespace {


template <bool MIXED>
struct GView {
  const void *gm;
  const int *ge;
  __device__ __forceinline__ static size_t idx(int a, int b) {
    const int t = b >> 5, s = a >> 5;
    return ((size_t)(t * (t + 1) / 2 + s) << 10) + ((a & 31) << 5) + (b & 31);
  }
  __device__ __forceinline__ double m(size_t i) const {
    return MIXED ? (double)((const float *)gm)[i] : ((const double *)gm)[i];
  }
  __device__ __forceinline__ float mf(size_t i) const {
    return MIXED ? ((const float *)gm)[i] : (float)((const double *)gm)[i];
  }
  __device__ __forceinline__ int e(size_t i) const { return ge[i]; }
};

// x * 2^k for k <= 0 by integer arithmetic on the exponent field (x >= 0 normal
// or zero); 0 when the result would leave the normal range.
__device__ __forceinline__ double scale_nonpos(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)(b >> 52);  // sign bit is 0
  return (ex + k <= 0) ? 0.0 : __longlong_as_double(b + ((long long)k << 52));
}

// acc + K * y with K = (km, ke) normalised (or an extended zero), y normalised,
// acc any positive mantissa: one float64 FMA.
__device__ __forceinline__ xd fma_x(xd acc, double km, int ke, xd y) {
  const int pe = ke + y.e;
  const int E = max(acc.e, pe);
  return xd{fma(scale_nonpos(km, pe - E), y.m, scale_nonpos(acc.m, acc.e - E)), E};
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

// Round a mantissa in [1,2) to float with integer ops (no float64 conversion unit).
__device__ __forceinline__ float mant_to_float(double m) {
  const long long b = __double_as_longlong(m);
  const long long frac = b & 0x000fffffffffffffLL;
  return __int_as_float((int)((frac + (1LL << 28)) >> 29) + 0x3f800000);
}

struct ChainSmem {
  double *Ym;  // [N+1] Y mantissas
  int *Ye;     // [N+1]
  double *Am;  // [N] bulk row sums (sources of tiles <= t-1 for rows of tile t+1)
  int *Ae;
  double *Kdm;  // [2][32][33] c-scaled diagonal blocks (double buffer)
  int *Kde;
  double *Hom;  // [2][32][33] H(source of tile t, row of tile t+1) (double buffer)
  int *Hoe;
};

template <bool MIXED, bool BWD>
__device__ void run_chain(const Workspace &w, ChainSmem sm) {
  const int N = w.N, NT = w.NT;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // H(src, row) in this recursion's own coordinates (both copies share the layout)
  const void *gm = BWD ? w.gbm : w.gm;
  const int *ge = BWD ? w.gbe : w.ge;
  auto hidx = [](int src, int row) -> size_t { return GView<MIXED>::idx(src, row); };
  auto hm_ld = [&](size_t gi) -> double {
    return MIXED ? (double)__ldg((const float *)gm + gi) : __ldg((const double *)gm + gi);
  };
  auto coef = [&](int row) -> xd {
    if (!BWD) return xd{__ldg(w.ccm + row), __ldg(w.cce + row)};
    if (row >= N - 1) return xd{1.0, 0};
    return xd{__ldg(w.ccm + N - 2 - row), __ldg(w.cce + N - 2 - row)};
  };
  double *gYm = BWD ? w.ybm : w.yfm;
  int *gYe = BWD ? w.ybe : w.yfe;
  // roles: warp 0 = dependency chain; warps 1, 2 = staging of the next tile's
  // blocks; bulk = every other warp not on warp 0's sub-partition (id % 4 != 0)
  auto bulk_warp = [](int q) { return q > 2 && (q & 3) != 0; };
  const bool is_bulk = bulk_warp(wid);
  int nbulk = 0, bulk_rank = 0;
  for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
    if (bulk_warp(q)) { if (q < wid) ++bulk_rank; ++nbulk; }

  // Load H(srcbase+i, rowbase+lane), i = 0..31, into dm/de[i*33+lane] (one warp,
  // loads coalesced along rows, all issued before use).  Pairs outside
  // src <= row < N hold the extended zero 1 * 2^XZERO_E.
  auto load_block = [&](int srcbase, int rowbase, double *dm, int *de) {
    const int row = rowbase + lane;
#pragma unroll 16
    for (int i = 0; i < TILE; ++i) {
      const int src = srcbase + i;
      double m = 1.0;
      int e = XZERO_E;
      if (row < N && src <= row) {
        const size_t gi = hidx(src, row);
        m = hm_ld(gi);
        e = __ldg(ge + gi);
      }
      dm[i * 33 + lane] = m;
      de[i * 33 + lane] = e;
    }
  };
  // warp 1: H from source tile tt to the rows of tile tt+1 (raw)
  auto stage_offdiag = [&](int tt, int buf) {
    load_block(tt * TILE, tt * TILE + TILE, sm.Hom + buf * 32 * 33, sm.Hoe + buf * 32 * 33);
  };
  // warp 2: the diagonal block of tile tt, pre-scaled by the row coefficient c
  auto stage_diag = [&](int tt, int buf) {
    const int r0 = tt * TILE, row = r0 + lane;
    double *dm = sm.Kdm + buf * 32 * 33;
    int *de = sm.Kde + buf * 32 * 33;
    load_block(r0, r0, dm, de);
    const xd c = (row < N) ? xnorm_int(coef(row)) : xd{1.0, 0};
#pragma unroll 8
    for (int i = 0; i < TILE; ++i) {
      const xd k = xmul_int(c, xd{dm[i * 33 + lane], de[i * 33 + lane]});
      dm[i * 33 + lane] = k.m;
      de[i * 33 + lane] = k.e;
    }
  };

  for (int r = tid; r < N; r += blockDim.x) { sm.Am[r] = 0.0; sm.Ae[r] = XZERO_E; }
  if (tid == 0) { sm.Ym[0] = 1.0; sm.Ye[0] = 0; }
  xd nxt{1.0, XZERO_E};  // warp 0: partial sum of row 32(t+1)+lane over source tile t
  if (wid == 1) stage_offdiag(0, 0);
  if (wid == 2) stage_diag(0, 0);
  __syncthreads();

  for (int t = 0; t < NT; ++t) {
    const int r0 = t * TILE, buf = t & 1;
    if (wid == 0) {
      // ------------------------------------------------ dependent steps of tile t
      const int row = r0 + lane;
      xd acc{0.0, XZERO_E};
      if (row < N) {
        acc = xadd_raw(xd{sm.Am[row], sm.Ae[row]}, nxt);
        acc = xmul_int(xnorm(acc.m, acc.e), coef(row));  // acc' = c_row * (sum over sources < r0)
      }
      xd ycur{sm.Ym[r0], sm.Ye[r0]};
      const double *Kdm = sm.Kdm + buf * 32 * 33, *Hom = sm.Hom + buf * 32 * 33;
      const int *Kde = sm.Kde + buf * 32 * 33, *Hoe = sm.Hoe + buf * 32 * 33;
      if (!(acc.m > 0.0)) acc = xd{1.0, XZERO_E};
      nxt = xd{1.0, XZERO_E};
      // 32 steps, no branches and no stores: rows past N and finished rows see
      // extended zeros in the staged blocks, and row j's accumulator is final
      // after step j (later steps add at most 2^-1000 of it).  Block entries of
      // step i+1 are loaded (explicit ld.shared) before step i's shuffle.
      const unsigned aKm = smem_addr(Kdm + lane), aHm = smem_addr(Hom + lane);
      const unsigned aKe = smem_addr(Kde + lane), aHe = smem_addr(Hoe + lane);
      double km = lds_f64(aKm), hm = lds_f64(aHm);
      int ke = lds_s32(aKe), he = lds_s32(aHe);
#pragma unroll
      for (int i = 0; i < TILE; ++i) {
        double km1 = 0.0, hm1 = 0.0;
        int ke1 = 0, he1 = 0;
        if (i + 1 < TILE) {
          km1 = lds_f64(aKm + (i + 1) * 33 * 8);
          hm1 = lds_f64(aHm + (i + 1) * 33 * 8);
          ke1 = lds_s32(aKe + (i + 1) * 33 * 4);
          he1 = lds_s32(aHe + (i + 1) * 33 * 4);
        }
        acc = fma_chain(acc, km, ke, ycur);  // the dependency chain
        nxt = fma_chain(nxt, hm, he, ycur);  // next tile's rows, off the chain
        ycur.m = __shfl_sync(0xffffffffu, acc.m, i);
        ycur.e = __shfl_sync(0xffffffffu, acc.e, i);
        km = km1; hm = hm1; ke = ke1; he = he1;
      }
      if (row < N) {  // Y_{row+1} = final accumulator of row `row`
        const xd yn = xnorm_int(acc);
        sm.Ym[row + 1] = yn.m;
        sm.Ye[row + 1] = yn.e;
      }
      nxt = xnorm_int(nxt);
    } else if (wid == 1) {
      if (t + 1 < NT) stage_offdiag(t + 1, buf ^ 1);
    } else if (wid == 2) {
      if (t + 1 < NT) stage_diag(t + 1, buf ^ 1);
    } else if (is_bulk && t >= 1) {
      // ------------------------------ bulk: source tile t-1 -> rows of tiles >= t+1
      // thread per row; loads coalesced along rows
      const int srcbase = r0 - TILE;
      const int bthreads = nbulk * 32;
      for (int r = r0 + TILE + bulk_rank * 32 + lane; r < N; r += bthreads) {
        xd acc{sm.Am[r], sm.Ae[r]};
        if (MIXED) {
          // one pass with a running maximum exponent (rescale on increase)
          float sacc = 0.0f;
          int E = XZERO_E;
#pragma unroll 8
          for (int i = 0; i < TILE; ++i) {
            const int src = srcbase + i;
            const size_t gi = hidx(src, r);
            const float m = __ldg((const float *)gm + gi);
            const int e = __ldg(ge + gi) + sm.Ye[src];
            const int En = max(E, e);
            sacc = fmaf(mant_to_float(sm.Ym[src]) * m, pow2f_nonpos(e - En), sacc * pow2f_nonpos(E - En));
            E = En;
          }
          acc = xadd_raw(acc, xd{(double)sacc, E});
        } else {
          // float64: an integer pass for the maximum exponent, then one FMA per term
          int E = XZERO_E;
#pragma unroll 16
          for (int i = 0; i < TILE; ++i) E = max(E, sm.Ye[srcbase + i] + __ldg(ge + hidx(srcbase + i, r)));
          double sacc = 0.0;
#pragma unroll 16
          for (int i = 0; i < TILE; ++i) {
            const int src = srcbase + i;
            const size_t gi = hidx(src, r);
            sacc = fma(scale_nonpos(__ldg((const double *)gm + gi), sm.Ye[src] + __ldg(ge + gi) - E), sm.Ym[src],
                       sacc);
          }
          acc = xadd_raw(acc, xd{sacc, E});
        }
        acc = xnorm(acc.m, acc.e);
        sm.Am[r] = acc.m;
        sm.Ae[r] = acc.e;
      }
    }
    __syncthreads();
  }
  for (int v = tid; v <= N; v += blockDim.x) { gYm[v] = sm.Ym[v]; gYe[v] = sm.Ye[v]; }
}

template <bool MIXED>
__global__ void __launch_bounds__(CHAIN_THREADS, 1) chain_kernel(Workspace w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = w.N;
  ChainSmem sm;
  unsigned char *p = smem_raw;
  sm.Ym = (double *)p; p += sizeof(double) * (N + 1);
  sm.Am = (double *)p; p += sizeof(double) * N;
  sm.Kdm = (double *)p; p += sizeof(double) * 2 * 32 * 33;
  sm.Hom = (double *)p; p += sizeof(double) * 2 * 32 * 33;
  sm.Ye = (int *)p; p += sizeof(int) * (N + 1);
  sm.Ae = (int *)p; p += sizeof(int) * N;
  sm.Kde = (int *)p; p += sizeof(int) * 2 * 32 * 33;
  sm.Hoe = (int *)p; p += sizeof(int) * 2 * 32 * 33;
  if (blockIdx.x == 0) run_chain<MIXED, false>(w, sm);
  else run_chain<MIXED, true>(w, sm);
}

constexpr size_t chain_smem_bytes(int N) {
  return sizeof(double) * ((size_t)(N + 1) + N + 4 * 32 * 33) + sizeof(int) * ((size_t)(N + 1) + N + 4 * 32 * 33);
}
static_assert(chain_smem_bytes(CHAIN_MAX_N) <= 227 * 1024, "recursion state for the largest N must fit in shared memory");

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

cudaError_t launch_chains(const Workspace &w, cudaStream_t s) {
  cudaError_t e = prepare_chains();
  if (e != cudaSuccess) return e;
  const size_t bytes = chain_smem_bytes(w.N);
  if (w.mixed) chain_kernel<true><<<2, CHAIN_THREADS, bytes, s>>>(w);
  else chain_kernel<false><<<2, CHAIN_THREADS, bytes, s>>>(w);
  return cudaGetLastError();
}

}  // namespace bpimd
