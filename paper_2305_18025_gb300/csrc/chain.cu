// Forward and backward potential recursions (one CTA each, run concurrently).
//
// Forward  (Eq. our-forward-potential-recurrence, linear-space form):
//   y_0 = 1,  y_{r+1} = c_{r+1} * S_r,  S_r = sum_{w<=r} y_w g(w+1, r+1)
// Backward (Eq. backward-potential-recursion, linear-space form), with rows
// r = N-1-a and sources w = N-1-b so that it has the same lower-triangular
// shape:  Y_0 = mu_N = 1, S_r = B_{a+1} = sum_{w<=r} Y_w g(a+1, b+1),
//   Y_{r+1} = mu_a = c_a * S_r   (c_0 := 1 for the last row, Y_N = B_1).
// Both are lower-triangular solves with the matrix of pair factors g.
//
// Schedule (rows in tiles of 32):
//   phase a (all warps)   : rows of tile t += contributions of source tile t-1;
//                           the diagonal 32x32 block of g is staged in smem.
//   phase b (concurrently): warp 0 runs the 32 dependent steps of tile t
//                           (lane j holds row 32t+j; each step adds the newest
//                           y to every later row and finalises one row);
//                           warps 1..31 add source tile t-1 to all rows of
//                           tiles >= t+1.
// Every value is an extended number (mantissa * 2^exponent), so a step is a
// multiply-add; no exp/log is on the dependency chain.
// MIXED: the bulk tile products are summed in float32 per 32-source tile and
// then added to the float64 row accumulator; the dependent steps stay float64.
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

struct ChainSmem {
  double *Ym;
  int *Ye;
  float *Y32;  // float copy of the mantissas (MIXED bulk)
  double *Am;
  int *Ae;
  double *Dm;  // [32][33]
  int *De;     // [32][33]
};

template <bool MIXED, bool BWD>
__device__ void run_chain(const Workspace &w, ChainSmem sm) {
  const int N = w.N;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  GView<MIXED> G{w.gm, w.ge};
  // H(src, row) for this direction
  auto hidx = [&](int src, int row) -> size_t {
    return BWD ? GView<MIXED>::idx(N - 1 - row, N - 1 - src) : GView<MIXED>::idx(src, row);
  };
  auto coef = [&](int row) -> xd {
    if (!BWD) return xd{w.ccm[row], w.cce[row]};
    if (row >= N - 1) return xd{1.0, 0};
    return xd{w.ccm[N - 2 - row], w.cce[N - 2 - row]};
  };
  double *gYm = BWD ? w.ybm : w.yfm;
  int *gYe = BWD ? w.ybe : w.yfe;
  double *gSm = BWD ? w.sbm : w.sfm;
  int *gSe = BWD ? w.sbe : w.sfe;

  for (int r = tid; r < N; r += blockDim.x) { sm.Am[r] = 0.0; sm.Ae[r] = XZERO_E; }
  if (tid == 0) { sm.Ym[0] = 1.0; sm.Ye[0] = 0; sm.Y32[0] = 1.0f; }
  __syncthreads();

  const int NT = w.NT;
  for (int t = 0; t < NT; ++t) {
    const int r0 = t * TILE;
    // ---------------- phase a: critical update of tile t with source tile t-1
    if (t >= 1) {
      const int r = r0 + wid;
      if (r < N) {
        const int src = r0 - TILE + lane;
        const size_t gi = hidx(src, r);
        if (MIXED) {
          float pm = sm.Y32[src] * G.mf(gi);
          int pe = sm.Ye[src] + G.e(gi);
          int E = pe;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
          float v = pm * pow2f_nonpos(pe - E);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) {
            xd a = xadd_raw(xd{sm.Am[r], sm.Ae[r]}, xd{(double)v, E});
            a = xnorm(a.m, a.e);
            sm.Am[r] = a.m; sm.Ae[r] = a.e;
          }
        } else {
          double pm = sm.Ym[src] * G.m(gi);
          int pe = sm.Ye[src] + G.e(gi);
          int E = pe;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
          double v = pm * pow2_nonpos(pe - E);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) {
            xd a = xadd_raw(xd{sm.Am[r], sm.Ae[r]}, xd{v, E});
            a = xnorm(a.m, a.e);
            sm.Am[r] = a.m; sm.Ae[r] = a.e;
          }
        }
      }
    }
    {  // stage the diagonal block: D[i][j] = H(r0+i, r0+j) for i <= j
      const int src = r0 + wid, row = r0 + lane;
      double dm = 0.0;
      int de = XZERO_E;
      if (row < N && src <= row) {
        const size_t gi = hidx(src, row);
        dm = G.m(gi);
        de = G.e(gi);
      }
      sm.Dm[wid * 33 + lane] = dm;
      sm.De[wid * 33 + lane] = de;
    }
    __syncthreads();
    // ---------------- phase b
    if (wid == 0) {
      const int row = r0 + lane;
      xd acc = (row < N) ? xd{sm.Am[row], sm.Ae[row]} : xd{0.0, XZERO_E};
      xd ycur{sm.Ym[r0], sm.Ye[r0]};
      for (int i = 0; i < TILE; ++i) {
        const int r = r0 + i;
        if (r >= N) break;
        if (lane >= i) acc = xmuladd_raw(acc, ycur, sm.Dm[i * 33 + lane], sm.De[i * 33 + lane]);
        xd ynew{0.0, 0};
        if (lane == i) {
          const xd S = xnorm(acc.m, acc.e);
          ynew = xmul(S, coef(r));
          sm.Ym[r + 1] = ynew.m;
          sm.Ye[r + 1] = ynew.e;
          sm.Y32[r + 1] = (float)ynew.m;
          gSm[r] = S.m;
          gSe[r] = S.e;
        }
        ycur.m = __shfl_sync(0xffffffffu, ynew.m, i);
        ycur.e = __shfl_sync(0xffffffffu, ynew.e, i);
      }
    } else if (t >= 1) {
      // bulk: rows of tiles >= t+1 += source tile t-1
      const int srcbase = r0 - TILE;
      for (int r = r0 + TILE + (tid - 32); r < N; r += blockDim.x - 32) {
        xd acc{sm.Am[r], sm.Ae[r]};
        if (MIXED) {
          float s = 0.0f;
          int E = XZERO_E;
#pragma unroll 8
          for (int i = 0; i < TILE; ++i) {
            const int src = srcbase + i;
            const size_t gi = hidx(src, r);
            const float pm = sm.Y32[src] * G.mf(gi);
            const int pe = sm.Ye[src] + G.e(gi);
            const int En = max(E, pe);
            s = fmaf(pm, pow2f_nonpos(pe - En), s * pow2f_nonpos(E - En));
            E = En;
          }
          acc = xadd_raw(acc, xd{(double)s, E});
        } else {
#pragma unroll 8
          for (int i = 0; i < TILE; ++i) {
            const int src = srcbase + i;
            const size_t gi = hidx(src, r);
            acc = xmuladd_raw(acc, xd{sm.Ym[src], sm.Ye[src]}, G.m(gi), G.e(gi));
          }
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
  sm.Dm = (double *)p; p += sizeof(double) * 32 * 33;
  sm.Ye = (int *)p; p += sizeof(int) * (N + 1);
  sm.Ae = (int *)p; p += sizeof(int) * N;
  sm.De = (int *)p; p += sizeof(int) * 32 * 33;
  sm.Y32 = (float *)p;
  if (blockIdx.x == 0) run_chain<MIXED, false>(w, sm);
  else run_chain<MIXED, true>(w, sm);
}

size_t chain_smem_bytes(int N) {
  return sizeof(double) * ((size_t)(N + 1) + N + 32 * 33) + sizeof(int) * ((size_t)(N + 1) + N + 32 * 33)
         + sizeof(float) * (size_t)(N + 1);
}

}  // namespace

cudaError_t launch_chains(const Workspace &w, cudaStream_t s) {
  const size_t bytes = chain_smem_bytes(w.N);
  cudaError_t e;
  if (w.mixed) {
    e = cudaFuncSetAttribute(chain_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    chain_kernel<true><<<2, CHAIN_THREADS, bytes, s>>>(w);
  } else {
    e = cudaFuncSetAttribute(chain_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    chain_kernel<false><<<2, CHAIN_THREADS, bytes, s>>>(w);
  }
  return cudaGetLastError();
}

}  // namespace bpimd
