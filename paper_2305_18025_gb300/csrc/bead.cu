// Bead pass: one read of the positions per evaluation.
//
// Per particle l (one warp for the bead sums, then one lane for the rest):
//   E_int^{(l)} = (1/2) m w_P^2 sum_{j=1}^{P-1} (r_l^{j+1} - r_l^j)^2     (Eq. e-interior)
//   link_l      = (1/2) m w_P^2 (r_l^P - r_{l+1}^1)^2, 0 for l = N       (spring of Eq. e-recurrence-step)
//   interior forces -m w_P^2 (2 r_l^j - r_l^{j+1} - r_l^{j-1}), j=2..P-1  (Eq. intermediate-bead-force)
//   copies of r_l^1 and r_l^P (MIXED: also as float32 high/low parts), and
//   the coefficient c_l = exp(beta link_l)/l of the linear-space recursions,
//   as an extended number.
// FP64: everything in float64.  MIXED: bead differences formed in float64,
// rounded to float32; squares, warp sums and interior forces in float32;
// E_int and link widened to float64.
#include "bpimd_internal.cuh"

namespace bpimd {
namespace {

constexpr int BEAD_WARPS = BEAD_BLOCK_PARTICLES;  // particles per block (one warp each)

// Particles l0 .. l0+7 of one system (all threads of the block).
template <bool MIXED>
__device__ __forceinline__ void bead_pass_body(const Workspace &w, const double *__restrict__ pos,
                                               double *__restrict__ F, int l0) {
  __shared__ double eint_s[BEAD_WARPS];
  __shared__ int finite_s[BEAD_WARPS];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int P = w.P;
  const double k = w.k;
  // phase 1: one warp per particle -- interior springs and interior forces
  {
    const int l = l0 + wp;
    bool finite = true;
    double s64 = 0.0;
    float s32 = 0.0f;
    if (l < w.N) {
      const double *p = pos + (size_t)l * P * 3;
      double *f = F + (size_t)l * P * 3;
      for (int j = lane; j < P; j += 32) {
        const double x = p[3 * j], y = p[3 * j + 1], z = p[3 * j + 2];
        finite &= isfinite(x) && isfinite(y) && isfinite(z);
        if (j + 1 < P) {
          const double dx = mimage(w, p[3 * j + 3] - x), dy = mimage(w, p[3 * j + 4] - y),
                       dz = mimage(w, p[3 * j + 5] - z);
          if (MIXED) {
            const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
            s32 = fmaf(fx, fx, fmaf(fy, fy, fmaf(fz, fz, s32)));
          } else {
            s64 = fma(dx, dx, fma(dy, dy, fma(dz, dz, s64)));
          }
        }
        if (j >= 1 && j + 1 < P) {  // interior bead (0-based 1..P-2)
          const double ax = mimage(w, x - p[3 * j + 3]), ay = mimage(w, y - p[3 * j + 4]),
                       az = mimage(w, z - p[3 * j + 5]);
          const double bx = mimage(w, x - p[3 * j - 3]), by = mimage(w, y - p[3 * j - 2]),
                       bz = mimage(w, z - p[3 * j - 1]);
          if (MIXED) {
            const float kf = (float)k;
            f[3 * j] = (double)(-kf * ((float)ax + (float)bx));
            f[3 * j + 1] = (double)(-kf * ((float)ay + (float)by));
            f[3 * j + 2] = (double)(-kf * ((float)az + (float)bz));
          } else {
            f[3 * j] = -k * (ax + bx);
            f[3 * j + 1] = -k * (ay + by);
            f[3 * j + 2] = -k * (az + bz);
          }
        }
      }
    }
    if (MIXED) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s32 += __shfl_xor_sync(0xffffffffu, s32, o);
      s64 = (double)s32;
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, o);
    }
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) { eint_s[wp] = w.half_k * s64; finite_s[wp] = finite; }
  }
  __syncthreads();
  // phase 2: one lane per particle -- links, endpoint copies and the
  // coefficients c, 1/c (the float64 transcendentals run once per 8 particles)
  if (wp == 0 && lane < BEAD_WARPS) {
    const int l = l0 + lane;
    if (l < w.N) {
      if (!finite_s[lane]) atomicOr(w.status, ST_NONFINITE);
      const double *b1 = pos + (size_t)l * P * 3, *bP = b1 + 3 * (P - 1);
      double lk = 0.0;
      if (l + 1 < w.N) {
        const double *n1 = b1 + 3 * P;  // bead 1 of particle l+1
        const double dx = mimage(w, bP[0] - n1[0]), dy = mimage(w, bP[1] - n1[1]),
                     dz = mimage(w, bP[2] - n1[2]);
        if (MIXED) {
          const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
          lk = w.half_k * (double)fmaf(fx, fx, fmaf(fy, fy, fz * fz));
        } else {
          lk = w.half_k * fma(dx, dx, fma(dy, dy, dz * dz));
        }
      }
      w.Eint[l] = eint_s[lane];
      w.link[l] = lk;
      double *r1 = w.R1 + 4 * (size_t)l, *rp = w.RP + 4 * (size_t)l;
      r1[0] = b1[0]; r1[1] = b1[1]; r1[2] = b1[2]; r1[3] = 0.0;
      rp[0] = bP[0]; rp[1] = bP[1]; rp[2] = bP[2]; rp[3] = 0.0;
      if (MIXED && w.pbc) {  // fixed-point fractions of the box
        unsigned *u1 = (unsigned *)(w.R1s + 8 * (size_t)l), *uP = (unsigned *)(w.RPs + 8 * (size_t)l);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double f1 = b1[c] * w.invL - floor(b1[c] * w.invL), fP = bP[c] * w.invL - floor(bP[c] * w.invL);
          u1[c] = (unsigned)fmin(f1 * 4294967296.0, 4294967295.0);
          uP[c] = (unsigned)fmin(fP * 4294967296.0, 4294967295.0);
        }
        u1[3] = 0u; uP[3] = 0u;
      } else if (MIXED) {  // float32 high + low parts (x = hi + lo to ~2^-48 relative)
        float *s1 = w.R1s + 8 * (size_t)l, *sp = w.RPs + 8 * (size_t)l;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float h1 = (float)b1[c], hP = (float)bP[c];
          s1[c] = h1; s1[4 + c] = (float)(b1[c] - (double)h1);
          sp[c] = hP; sp[4 + c] = (float)(bP[c] - (double)hP);
        }
        s1[3] = 0.0f; s1[7] = 0.0f; sp[3] = 0.0f; sp[7] = 0.0f;
      }
      // c_{l+1} = exp(beta link_l) / (l+1) = 2^x, x = beta link_l log2(e) - log2(l+1)
      // |x| is clamped to 2^28 so that exponent sums stay in int32
      const double x = fmin(fmax(w.beta * lk * LOG2E - log2((double)(l + 1)), -268435456.0), 268435456.0);
      const double n = floor(x);
      const xd c = xnorm(exp2(x - n), (int)n);
      w.ccm[l] = c.m;
      w.cce[l] = c.e;
      const double ni = floor(-x);
      const xd ic = xnorm(exp2(-x - ni), (int)ni);
      w.icm[l] = ic.m;
      w.ice[l] = ic.e;
    }
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(32 * BEAD_WARPS) bead_pass_kernel(Workspace w, const double *__restrict__ pos,
                                                                    double *__restrict__ F) {
  bead_pass_body<MIXED>(w, pos, F, blockIdx.x * BEAD_WARPS);
}

// Replica batch: block k handles particles tab[k].y.. of replica tab[k].x,
// whose positions and forces start at element off[replica] of the packed arrays.
template <bool MIXED>
__global__ void __launch_bounds__(32 * BEAD_WARPS) bead_pass_batched(const Workspace *__restrict__ ws,
                                                                     const int2 *__restrict__ tab,
                                                                     const long long *__restrict__ off,
                                                                     const double *__restrict__ pos,
                                                                     double *__restrict__ F) {
  const int2 e = tab[blockIdx.x];
  bead_pass_body<MIXED>(ws[e.x], pos + off[e.x], F + off[e.x], e.y);
}

}  // namespace

cudaError_t launch_bead_pass(const Workspace &w, const double *pos, double *F, cudaStream_t s) {
  dim3 grid((w.N + BEAD_WARPS - 1) / BEAD_WARPS), block(32 * BEAD_WARPS);
  if (w.mixed) bead_pass_kernel<true><<<grid, block, 0, s>>>(w, pos, F);
  else bead_pass_kernel<false><<<grid, block, 0, s>>>(w, pos, F);
  return cudaGetLastError();
}

cudaError_t launch_bead_pass_batched(const Workspace *ws, const int2 *tab, int ntab, const long long *off,
                                     bool mixed, const double *pos, double *F, cudaStream_t s) {
  if (ntab <= 0) return cudaSuccess;
  if (mixed) bead_pass_batched<true><<<ntab, 32 * BEAD_WARPS, 0, s>>>(ws, tab, off, pos, F);
  else bead_pass_batched<false><<<ntab, 32 * BEAD_WARPS, 0, s>>>(ws, tab, off, pos, F);
  return cudaGetLastError();
}

}  // namespace bpimd
