// Connection probabilities fused with the exterior-bead forces.
//
//   Pr[l -> u] (u <= l) = y_{u-1} g(u,l) mu_l / (N y_N)     (Eq. close-cycle-probability)
//   Pr[l -> l+1]        = 1 - y_l B_{l+1} / (N y_N)          (Eq. direct-link-probability)
//   Pr[l -> u]          = 0 for u > l+1                      (Lemma zero-connection-probability)
// The N x N matrix is never stored: each 32x32 block of the lower triangle is
// generated from the stored pair factors g and reduced on the spot into
//   row l    : sum_u Pr[l->u],  sum_u Pr[l->u] (r_l^P - r_u^1)    (bead P of l)
//   column u : sum_l Pr[l->u],  sum_l Pr[l->u] (r_u^1 - r_l^P)    (bead 1 of u)
// partial sums per block (deterministic, no atomics).  The finalise pass adds
// the partials of each particle in a fixed order, adds the direct-link term and
// forms (Eq. force-on-1-sum-neighbors, Eq. force-on-P-sum-neighbors)
//   F_l^P = -m w_P^2 [ (sum_u Pr[l->u]) (r_l^P - r_l^{P-1}) + sum_u Pr[l->u] (r_l^P - r_u^1) ]
//   F_l^1 = -m w_P^2 [ (sum_l' Pr[l'->l]) (r_l^1 - r_l^2) + sum_l' Pr[l'->l] (r_l^1 - r_l'^P) ]
// i.e. the per-neighbour sums of the paper distributed over their terms.
// MIXED: block-local products and sums in float32, combination in float64.
#include "bpimd_internal.cuh"

namespace bpimd {
namespace {

__device__ __forceinline__ void block_coords_f(int blk, int &t, int &s) {
  int tt = (int)((sqrt(8.0 * blk + 1.0) - 1.0) * 0.5);
  while ((tt + 1) * (tt + 2) / 2 <= blk) ++tt;
  while (tt * (tt + 1) / 2 > blk) --tt;
  t = tt;
  s = blk - tt * (tt + 1) / 2;
}

__device__ __forceinline__ xd alpha_of(const Workspace &w, int a) {
  // y_a / (N y_N)
  return xmul(xd{w.yfm[a], w.yfe[a]}, xd{w.scal[1], w.scal_i[0]});
}
__device__ __forceinline__ xd mu_of(const Workspace &w, int b) {
  const int r = w.N - 1 - b;  // backward row index of mu_b (0-based mu~_b = Yb[N-1-b])
  return xd{w.ybm[r], w.ybe[r]};
}

template <bool MIXED>
__global__ void __launch_bounds__(256) prob_force_kernel(Workspace w) {
  __shared__ double red[8][32][4];
  for (int blk = blockIdx.x; blk < w.NB; blk += gridDim.x) {
    int t, s;
    block_coords_f(blk, t, s);
    const int j = threadIdx.x & 31, i0 = threadIdx.x >> 5;
    const int b = t * TILE + j;
    const bool bvalid = b < w.N;
    xd mub{0.0, XZERO_E};
    double bx = 0, by = 0, bz = 0;
    if (bvalid) {
      mub = mu_of(w, b);
      bx = w.RP[4 * b]; by = w.RP[4 * b + 1]; bz = w.RP[4 * b + 2];
    }
    double rs = 0, rx = 0, ry = 0, rz = 0;  // row partials (thread's 4 entries)
    float frs = 0, frx = 0, fry = 0, frz = 0;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int i = i0 + 8 * kk;
      const int a = s * TILE + i;
      const size_t gi = (size_t)blk * TILE2 + i * TILE + j;
      const bool valid = bvalid && a <= b;
      double cs = 0, cx = 0, cy = 0, cz = 0;
      float fcs = 0, fcx = 0, fcy = 0, fcz = 0;
      if (valid) {
        const xd al = alpha_of(w, a);
        const double dx = bx - w.R1[4 * a], dy = by - w.R1[4 * a + 1], dz = bz - w.R1[4 * a + 2];
        if (MIXED) {
          const float gmf = ((const float *)w.gm)[gi];
          const int e = al.e + mub.e + w.ge[gi];
          float M = (float)al.m * (float)mub.m * gmf;
          M = (e < -150) ? 0.0f : (e > 0 ? M * (float)(1 << min(e, 2)) : M * pow2f_nonpos(e));
          const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
          frs += M; frx += M * fx; fry += M * fy; frz += M * fz;
          fcs = M; fcx = -M * fx; fcy = -M * fy; fcz = -M * fz;
        } else {
          const double gmd = ((const double *)w.gm)[gi];
          const double M = xtod(xd{al.m * mub.m * gmd, al.e + mub.e + w.ge[gi]});
          rs += M; rx = fma(M, dx, rx); ry = fma(M, dy, ry); rz = fma(M, dz, rz);
          cs = M; cx = -M * dx; cy = -M * dy; cz = -M * dz;
        }
      }
      // column a: reduce over the 32 lanes (b)
      if (MIXED) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fcs += __shfl_xor_sync(0xffffffffu, fcs, o);
          fcx += __shfl_xor_sync(0xffffffffu, fcx, o);
          fcy += __shfl_xor_sync(0xffffffffu, fcy, o);
          fcz += __shfl_xor_sync(0xffffffffu, fcz, o);
        }
        cs = fcs; cx = fcx; cy = fcy; cz = fcz;
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          cs += __shfl_xor_sync(0xffffffffu, cs, o);
          cx += __shfl_xor_sync(0xffffffffu, cx, o);
          cy += __shfl_xor_sync(0xffffffffu, cy, o);
          cz += __shfl_xor_sync(0xffffffffu, cz, o);
        }
      }
      if (j == 0) {
        double *cp = w.colpart + ((size_t)blk * TILE + i) * 4;
        cp[0] = cs; cp[1] = cx; cp[2] = cy; cp[3] = cz;
      }
    }
    if (MIXED) { rs = frs; rx = frx; ry = fry; rz = frz; }
    red[i0][j][0] = rs; red[i0][j][1] = rx; red[i0][j][2] = ry; red[i0][j][3] = rz;
    __syncthreads();
    if (threadIdx.x < 128) {
      const int jj = threadIdx.x >> 2, q = threadIdx.x & 3;
      double acc = 0.0;
#pragma unroll
      for (int g = 0; g < 8; ++g) acc += red[g][jj][q];
      w.rowpart[((size_t)blk * TILE + jj) * 4 + q] = acc;
    }
    __syncthreads();
  }
}

// Pr[l -> l+1] = 1 - y_l B_{l+1} / (N y_N); in 0-based particle index p (row p,
// column p+1) this is 1 - y[p+1] B(p+1) / (N y_N) with B(a) the backward row sum
// of particle a.
__device__ __forceinline__ double direct_link_prob(const Workspace &w, int p) {
  const xd y{w.yfm[p + 1], w.yfe[p + 1]};
  const xd B = backward_row_sum(w, p + 1);
  const double q = xtod(xmul(xmul(y, B), xd{w.scal[1], w.scal_i[0]}));
  return 1.0 - q;
}

__global__ void __launch_bounds__(256) force_finalize_kernel(Workspace w, const double *__restrict__ pos,
                                                             double *__restrict__ F) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= w.N) return;
  const int N = w.N, P = w.P, NT = w.NT;
  const double *r1 = w.R1 + 4 * (size_t)p, *rp = w.RP + 4 * (size_t)p;
  // row p (bead P of particle p)
  double rs = 0, rx = 0, ry = 0, rz = 0;
  {
    const int t = p >> 5, j = p & 31;
    for (int s = 0; s <= t; ++s) {
      const double *q = w.rowpart + ((size_t)(t * (t + 1) / 2 + s) * TILE + j) * 4;
      rs += q[0]; rx += q[1]; ry += q[2]; rz += q[3];
    }
    if (p + 1 < N) {
      const double M = direct_link_prob(w, p);
      const double *n1 = w.R1 + 4 * (size_t)(p + 1);
      rs += M;
      rx = fma(M, rp[0] - n1[0], rx); ry = fma(M, rp[1] - n1[1], ry); rz = fma(M, rp[2] - n1[2], rz);
    }
  }
  // column p (bead 1 of particle p)
  double cs = 0, cx = 0, cy = 0, cz = 0;
  {
    const int s = p >> 5, i = p & 31;
    for (int t = s; t < NT; ++t) {
      const double *q = w.colpart + ((size_t)(t * (t + 1) / 2 + s) * TILE + i) * 4;
      cs += q[0]; cx += q[1]; cy += q[2]; cz += q[3];
    }
    if (p >= 1) {
      const double M = direct_link_prob(w, p - 1);
      const double *pP = w.RP + 4 * (size_t)(p - 1);
      cs += M;
      cx = fma(M, r1[0] - pP[0], cx); cy = fma(M, r1[1] - pP[1], cy); cz = fma(M, r1[2] - pP[2], cz);
    }
  }
  const double k = w.k;
  const double *bead = pos + (size_t)p * P * 3;
  const double *nbP = bead + 3 * (P - 2);  // bead P-1 (1-based) next to bead P
  const double *nb1 = bead + 3;            // bead 2 (1-based) next to bead 1
  double *fP = F + ((size_t)p * P + (P - 1)) * 3;
  double *f1 = F + (size_t)p * P * 3;
  fP[0] = -k * fma(rs, rp[0] - nbP[0], rx);
  fP[1] = -k * fma(rs, rp[1] - nbP[1], ry);
  fP[2] = -k * fma(rs, rp[2] - nbP[2], rz);
  f1[0] = -k * fma(cs, r1[0] - nb1[0], cx);
  f1[1] = -k * fma(cs, r1[1] - nb1[1], cy);
  f1[2] = -k * fma(cs, r1[2] - nb1[2], cz);
  if (!(isfinite(fP[0]) && isfinite(fP[1]) && isfinite(fP[2]) && isfinite(f1[0]) && isfinite(f1[1]) &&
        isfinite(f1[2])))
    atomicOr(w.status, ST_NONFINITE);
}

__global__ void dense_prob_kernel(Workspace w, double *M) {
  const size_t NN = (size_t)w.N * w.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx / w.N), a = (int)(idx % w.N);  // row l = b, column l' = a
    double v = 0.0;
    if (a <= b) {
      const int t = b >> 5, s = a >> 5;
      const size_t gi = ((size_t)(t * (t + 1) / 2 + s) << 10) + ((a & 31) << 5) + (b & 31);
      const double gmd = w.mixed ? (double)((const float *)w.gm)[gi] : ((const double *)w.gm)[gi];
      const xd al = alpha_of(w, a), mu = mu_of(w, b);
      v = xtod(xd{al.m * mu.m * gmd, al.e + mu.e + w.ge[gi]});
    } else if (a == b + 1) {
      v = direct_link_prob(w, b);
    }
    M[idx] = v;
  }
}

}  // namespace

cudaError_t launch_prob_blocks(const Workspace &w, cudaStream_t s) {
  const int sms = sm_count();
  const int grid = w.NB < sms * 8 ? w.NB : sms * 8;
  if (w.mixed) prob_force_kernel<true><<<grid, 256, 0, s>>>(w);
  else prob_force_kernel<false><<<grid, 256, 0, s>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_force_finalize(const Workspace &w, const double *pos, double *F, cudaStream_t s) {
  force_finalize_kernel<<<(w.N + 255) / 256, 256, 0, s>>>(w, pos, F);
  return cudaGetLastError();
}

cudaError_t launch_dense_probabilities(const Workspace &w, double *M, cudaStream_t s) {
  dense_prob_kernel<<<1024, 256, 0, s>>>(w, M);
  return cudaGetLastError();
}

}  // namespace bpimd
