// Pair Boltzmann factors and diagnostic potentials.
//
// gmat: g(u,v) = exp(-beta (1/2) m w_P^2 (r_v^P - r_u^1)^2) for every u <= v --
// the closing-spring factor of the cycle energy E^{[u,v]} (Eq. e-recurrence-step,
// last term) -- stored once per evaluation as an extended number 2^x =
// mantissa(2^frac(x)) * 2^floor(x), x = -beta (1/2)k |d|^2 log2(e).
// FP64: float64 difference, square and exp2.  MIXED: difference of the
// float32 high/low parts of the positions, float32 square, hardware
// ex2.approx.  The potentials V^{[1,v]}, V^{[u,N]} for diagnostics are
// computed on demand by diag_potentials_kernel.
#include <type_traits>

#include "bpimd_internal.cuh"

namespace bpimd {
namespace {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// block index -> (t, s) with s <= t, blk = t(t+1)/2 + s
// (float32 estimate of the triangular root, corrected with integer tests:
// no float64 instruction)
__device__ __forceinline__ void block_coords(int blk, int &t, int &s) {
  int tt = (int)((sqrtf(8.0f * (float)blk + 1.0f) - 1.0f) * 0.5f);
  while ((tt + 1) * (tt + 2) / 2 <= blk) ++tt;
  while (tt * (tt + 1) / 2 > blk) --tt;
  t = tt;
  s = blk - tt * (tt + 1) / 2;
}

// g for one pair from the bead-P position of b and the bead-1 position of a:
// returns the mantissa (float or double) and sets the exponent.
template <bool MIXED>
__device__ __forceinline__ double pair_factor(const Workspace &w, double cx, int a, int b, int &e) {
  if (MIXED) {
    float fx, fy, fz;
    if (w.pbc) {  // minimum image from the fixed-point copies
      const uint4 ub = *(const uint4 *)(w.RPs + 8 * (size_t)b), ua = *(const uint4 *)(w.R1s + 8 * (size_t)a);
      fx = fixdiff(ub.x, ua.x, w.Lscale);
      fy = fixdiff(ub.y, ua.y, w.Lscale);
      fz = fixdiff(ub.z, ua.z, w.Lscale);
    } else {
      const float4 bh = *(const float4 *)(w.RPs + 8 * (size_t)b), bl = *(const float4 *)(w.RPs + 8 * (size_t)b + 4);
      const float4 ah = *(const float4 *)(w.R1s + 8 * (size_t)a), al = *(const float4 *)(w.R1s + 8 * (size_t)a + 4);
      fx = (bh.x - ah.x) + (bl.x - al.x);
      fy = (bh.y - ah.y) + (bl.y - al.y);
      fz = (bh.z - ah.z) + (bl.z - al.z);
    }
    // exponents below -2^28 stand for zero (keeps every exponent sum in int32)
    const float x = fmaxf((float)cx * fmaf(fx, fx, fmaf(fy, fy, fz * fz)), -268435456.0f);
    const float n = floorf(x);
    float mm = ex2_approx(x - n);  // in [1, 2]
    e = (int)n;
    if (mm >= 2.0f) { mm *= 0.5f; e += 1; }
    return mm;
  } else {
    const double dx = mimage(w, w.RP[4 * b] - w.R1[4 * a]), dy = mimage(w, w.RP[4 * b + 1] - w.R1[4 * a + 1]),
                 dz = mimage(w, w.RP[4 * b + 2] - w.R1[4 * a + 2]);
    // exponents below -2^28 stand for zero (keeps every exponent sum in int32)
    const double x = fmax(cx * fma(dx, dx, fma(dy, dy, dz * dz)), -268435456.0);
    const double n = floor(x);
    const xd g = xnorm(exp2(x - n), (int)n);
    e = g.e;
    return g.m;
  }
}

// One pass over the forward blocks (a = s*32+i, b = t*32+j): each valid pair
// a <= b < N is evaluated once and stored in both copies -- the forward one
// directly (coalesced along b), the backward one (row r = N-1-a, source
// w = N-1-b) after a transpose through shared memory, so that those stores
// are coalesced along r.  Entries outside a <= b < N are never written here
// (gmat_padding_kernel fills them once).
// One block of g (all threads of the CTA; Tm/Te: 32 x 33 shared tiles).
template <bool MIXED>
__device__ __forceinline__ void gmat_block(const Workspace &w, int blk,
                                           typename std::conditional<MIXED, float, double>::type *Tm, int *Te) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const double cx = -w.beta * w.half_k * LOG2E;
  const int N = w.N;
  M_t *gm = (M_t *)w.gm, *gbm = (M_t *)w.gbm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int t, s;
  block_coords(blk, t, s);
  {
    const int b = t * TILE + lane;
    for (int i = warp; i < TILE; i += 8) {
      const int a = s * TILE + i;
      if (b < N && a <= b) {
        int e;
        const M_t m = (M_t)pair_factor<MIXED>(w, cx, a, b, e);
        const size_t idx = (size_t)blk * TILE2 + i * TILE + lane;
        gm[idx] = m;
        w.ge[idx] = e;
        Tm[i * 33 + lane] = m;
        Te[i * 33 + lane] = e;
      }
    }
  }
  __syncthreads();
  {
    const int a = s * TILE + lane, r = N - 1 - a;
    for (int jj = warp; jj < TILE; jj += 8) {
      const int b = t * TILE + jj;
      if (b < N && a <= b) {
        const int src = N - 1 - b;
        const int T = r >> 5, S = src >> 5;
        const size_t idx = ((size_t)(T * (T + 1) / 2 + S) << 10) + ((src & 31) << 5) + (r & 31);
        gbm[idx] = Tm[lane * 33 + jj];
        w.gbe[idx] = Te[lane * 33 + jj];
      }
    }
  }
  __syncthreads();
}

template <bool MIXED>
__global__ void __launch_bounds__(256) gmat_kernel(Workspace w) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  __shared__ M_t Tm[TILE * 33];
  __shared__ int Te[TILE * 33];
  for (int blk = blockIdx.x; blk < w.NB; blk += gridDim.x) gmat_block<MIXED>(w, blk, Tm, Te);
}

// Replica batch: entry k of tab is (replica, block).
template <bool MIXED>
__global__ void __launch_bounds__(256) gmat_batched(const Workspace *__restrict__ ws, const int2 *__restrict__ tab,
                                                    int ntab) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  __shared__ M_t Tm[TILE * 33];
  __shared__ int Te[TILE * 33];
  for (int k = blockIdx.x; k < ntab; k += gridDim.x) {
    const int2 e = tab[k];
    gmat_block<MIXED>(ws[e.x], e.y, Tm, Te);
  }
}

// Entries outside lo <= col < N of either copy of one block (the upper part
// of diagonal blocks and the rows past N of the last tile): mantissa 1 with
// exponent XZERO_E, an extended zero.  They depend only on N.
template <bool MIXED>
__device__ __forceinline__ void gmat_padding_block(const Workspace &w, int blk) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  int t, s;
  block_coords(blk, t, s);
  const int j = threadIdx.x & 31, col = t * TILE + j;
  for (int i = threadIdx.x >> 5; i < TILE; i += 8) {
    const int lo = s * TILE + i;
    if (col >= w.N || lo > col) {
      const size_t idx = (size_t)blk * TILE2 + i * TILE + j;
      ((M_t *)w.gm)[idx] = (M_t)1.0;
      w.ge[idx] = XZERO_E;
      ((M_t *)w.gbm)[idx] = (M_t)1.0;
      w.gbe[idx] = XZERO_E;
    }
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(256) gmat_padding_kernel(Workspace w) {
  for (int blk = blockIdx.x; blk < w.NB; blk += gridDim.x) gmat_padding_block<MIXED>(w, blk);
}

template <bool MIXED>
__global__ void __launch_bounds__(256) gmat_padding_batched(const Workspace *__restrict__ ws,
                                                            const int2 *__restrict__ tab, int ntab) {
  for (int k = blockIdx.x; k < ntab; k += gridDim.x) {
    const int2 e = tab[k];
    gmat_padding_block<MIXED>(ws[e.x], e.y);
  }
}

// Diagnostic potentials of the last evaluation (on demand):
//   V^{[1,v]} = C[v] - ln(y_v)/beta,  V^{[u,N]} = C[N] - C[u-1] - ln(B_u / N)/beta.
__global__ void diag_potentials_kernel(Workspace w, double *Vf, double *Vb) {
  const int N = w.N;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= N; v += gridDim.x * blockDim.x) {
    Vf[v] = (v == 0) ? 0.0 : w.C[v] - xlog(xd{w.yfm[v], w.yfe[v]}) / w.beta;
    if (v < N) {  // u = v+1, particle a = v
      const xd B = backward_row_sum(w, v);
      Vb[v] = w.C[N] - w.C[v] - (xlog(B) - log((double)N)) / w.beta;
    } else {
      Vb[N] = 0.0;
    }
  }
}

}  // namespace

cudaError_t launch_diag_potentials(const Workspace &w, double *Vf, double *Vb, cudaStream_t s) {
  diag_potentials_kernel<<<(w.N + 256) / 256, 256, 0, s>>>(w, Vf, Vb);
  return cudaGetLastError();
}

cudaError_t launch_gmat(const Workspace &w, cudaStream_t s) {
  const int sms = sm_count();
  const int grid = w.NB < sms * 8 ? w.NB : sms * 8;
  if (w.mixed) gmat_kernel<true><<<grid, 256, 0, s>>>(w);
  else gmat_kernel<false><<<grid, 256, 0, s>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_gmat_padding(const Workspace &w, cudaStream_t s) {
  const int sms = sm_count();
  const int grid = w.NB < sms * 8 ? w.NB : sms * 8;
  if (w.mixed) gmat_padding_kernel<true><<<grid, 256, 0, s>>>(w);
  else gmat_padding_kernel<false><<<grid, 256, 0, s>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_gmat_batched(const Workspace *ws, const int2 *tab, int ntab, bool mixed, bool padding,
                                int blocks_per_sm, cudaStream_t s) {
  if (ntab <= 0) return cudaSuccess;
  const int sms = sm_count();
  const int cap = sms * (blocks_per_sm > 0 ? blocks_per_sm : 8);
  const int grid = ntab < cap ? ntab : cap;
  if (padding) {
    if (mixed) gmat_padding_batched<true><<<grid, 256, 0, s>>>(ws, tab, ntab);
    else gmat_padding_batched<false><<<grid, 256, 0, s>>>(ws, tab, ntab);
  } else {
    if (mixed) gmat_batched<true><<<grid, 256, 0, s>>>(ws, tab, ntab);
    else gmat_batched<false><<<grid, 256, 0, s>>>(ws, tab, ntab);
  }
  return cudaGetLastError();
}

}  // namespace bpimd
