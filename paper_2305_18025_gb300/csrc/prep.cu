// Pair Boltzmann factors and the scalar epilogue.
//
// gmat: g(u,v) = exp(-beta (1/2) m w_P^2 (r_v^P - r_u^1)^2) for every u <= v --
// the closing-spring factor of the cycle energy E^{[u,v]} (Eq. e-recurrence-step,
// last term) -- stored once per evaluation as an extended number 2^x =
// mantissa(2^frac(x)) * 2^floor(x), x = -beta (1/2)k |d|^2 log2(e).
// FP64: float64 difference, square and exp2.  MIXED: float64 difference
// rounded to float32, float32 square, hardware ex2.approx.
//
// scalars: prefix sums C[l] (FP64), V^{[1,N]} = C[N] - ln(y_N)/beta and the
// probability normaliser 1/(N y_N).  The potentials V^{[1,v]}, V^{[u,N]} for
// diagnostics are computed on demand by diag_potentials_kernel.
#include "bpimd_internal.cuh"

namespace bpimd {
namespace {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// block index -> (t, s) with s <= t, blk = t(t+1)/2 + s
__device__ __forceinline__ void block_coords(int blk, int &t, int &s) {
  int tt = (int)((sqrt(8.0 * blk + 1.0) - 1.0) * 0.5);
  while ((tt + 1) * (tt + 2) / 2 <= blk) ++tt;
  while (tt * (tt + 1) / 2 > blk) --tt;
  t = tt;
  s = blk - tt * (tt + 1) / 2;
}

// Blocks 0..NB-1 fill the forward copy (a = s*32+i, b = t*32+j); blocks
// NB..2NB-1 fill the backward copy in its own coordinates (source w = s*32+i,
// row r = t*32+j, i.e. a = N-1-r, b = N-1-w).  Invalid pairs (outside a <= b < N)
// are stored as mantissa 1 with exponent XZERO_E (an extended zero).
template <bool MIXED>
__global__ void __launch_bounds__(256) gmat_kernel(Workspace w) {
  const double cx = -w.beta * w.half_k * LOG2E;
  const int N = w.N;
  for (int gblk = blockIdx.x; gblk < 2 * w.NB; gblk += gridDim.x) {
    const bool bwd = gblk >= w.NB;
    const int blk = bwd ? gblk - w.NB : gblk;
    int t, s;
    block_coords(blk, t, s);
    void *gm = bwd ? w.gbm : w.gm;
    int *ge = bwd ? w.gbe : w.ge;
    const int j = threadIdx.x & 31;
    const int col = t * TILE + j;  // b (forward) or r (backward)
    for (int i = threadIdx.x >> 5; i < TILE; i += 8) {
      const int lo = s * TILE + i;  // a (forward) or w (backward)
      const size_t idx = (size_t)blk * TILE2 + i * TILE + j;
      if (col >= N || lo > col) {
        if (MIXED) ((float *)gm)[idx] = 1.0f; else ((double *)gm)[idx] = 1.0;
        ge[idx] = XZERO_E;
        continue;
      }
      const int a = bwd ? N - 1 - col : lo, b = bwd ? N - 1 - lo : col;
      const double dx = w.RP[4 * b] - w.R1[4 * a], dy = w.RP[4 * b + 1] - w.R1[4 * a + 1],
                   dz = w.RP[4 * b + 2] - w.R1[4 * a + 2];
      if (MIXED) {
        const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
        // exponents below -2^28 stand for zero (keeps every exponent sum in int32)
        const float x = fmaxf((float)cx * fmaf(fx, fx, fmaf(fy, fy, fz * fz)), -268435456.0f);
        const float n = floorf(x);
        float mm = ex2_approx(x - n);  // in [1, 2]
        int e = (int)n;
        if (mm >= 2.0f) { mm *= 0.5f; e += 1; }
        ((float *)gm)[idx] = mm;
        ge[idx] = e;
      } else {
        // exponents below -2^28 stand for zero (keeps every exponent sum in int32)
        const double x = fmax(cx * fma(dx, dx, fma(dy, dy, dz * dz)), -268435456.0);
        const double n = floor(x);
        xd g = xnorm(exp2(x - n), (int)n);
        ((double *)gm)[idx] = g.m;
        ge[idx] = g.e;
      }
    }
  }
}

// Single CTA: prefix sums, V_B, normaliser.
__global__ void __launch_bounds__(1024) scalars_kernel(Workspace w, double *V_B) {
  __shared__ double warp_tot[32];
  __shared__ double carry;
  const int N = w.N;
  if (threadIdx.x == 0) { carry = 0.0; w.C[0] = 0.0; }
  __syncthreads();
  // inclusive scan of A_i = E_int_i + link_i, C[i+1] = sum_{t<=i} A_t
  for (int base = 0; base < N; base += blockDim.x) {
    const int i = base + threadIdx.x;
    double v = (i < N) ? (w.Eint[i] + w.link[i]) : 0.0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      double u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
      double tsum = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0.0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        double u = __shfl_up_sync(0xffffffffu, tsum, o);
        if (lane >= o) tsum += u;
      }
      warp_tot[lane] = tsum;  // inclusive
    }
    __syncthreads();
    const double prefix = carry + (wid > 0 ? warp_tot[wid - 1] : 0.0);
    if (i < N) w.C[i + 1] = prefix + v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = prefix + v;
    __syncthreads();
  }
  // V_B and the normaliser 1/(N y_N)
  const xd yN{w.yfm[N], w.yfe[N]};
  if (threadIdx.x == 0) {
    const double CN = w.C[N];
    const double VB = CN - xlog(yN) / w.beta;
    w.scal[0] = VB;
    if (V_B) *V_B = VB;
    xd inv = xnorm(1.0 / (yN.m * (double)N), -yN.e);
    w.scal[1] = inv.m;
    w.scal_i[0] = inv.e;
    if (!isfinite(VB)) atomicOr(w.status, ST_NONFINITE);
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
  const int grid = 2 * w.NB < sms * 8 ? 2 * w.NB : sms * 8;
  if (w.mixed) gmat_kernel<true><<<grid, 256, 0, s>>>(w);
  else gmat_kernel<false><<<grid, 256, 0, s>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_scalars(const Workspace &w, double *V_B, cudaStream_t s) {
  scalars_kernel<<<1, 1024, 0, s>>>(w, V_B);
  return cudaGetLastError();
}

}  // namespace bpimd
