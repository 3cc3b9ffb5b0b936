// Connection probabilities fused with the exterior-bead forces.
//
//   Pr[l -> u] (u <= l) = y_{u-1} g(u,l) mu_l / (N y_N)     (Eq. close-cycle-probability)
//   Pr[l -> l+1]        = 1 - y_l B_{l+1} / (N y_N)          (Eq. direct-link-probability)
//   Pr[l -> u]          = 0 for u > l+1                      (Lemma zero-connection-probability)
// The N x N matrix is never stored: each 32x32 block of the lower triangle is
// generated from the stored pair factors g and reduced on the spot into
//   row l    : sum_u Pr[l->u],  sum_u Pr[l->u] (r_l^P - r_u^1)    (bead P of l)
//   column u : sum_l Pr[l->u],  sum_l Pr[l->u] (r_u^1 - r_l^P)    (bead 1 of u)
// partial sums per block.  Each block then counts itself in its row tile and
// its column tile (an atomic counter per tile); the block that completes a
// tile adds that tile's partials in a fixed block order (so the result does
// not depend on which block finishes last), adds the direct-link term and
// forms (Eq. force-on-1-sum-neighbors, Eq. force-on-P-sum-neighbors)
//   F_l^P = -m w_P^2 [ (sum_u Pr[l->u]) (r_l^P - r_l^{P-1}) + sum_u Pr[l->u] (r_l^P - r_u^1) ]
//   F_l^1 = -m w_P^2 [ (sum_l' Pr[l'->l]) (r_l^1 - r_l^2) + sum_l' Pr[l'->l] (r_l^1 - r_l'^P) ]
// i.e. the per-neighbour sums of the paper distributed over their terms.
// Precision forms: FP64 in float64 throughout.  MIXED (prob_block_mixed):
// Pr from 64-bit integer mantissa products, products with the float32 bead
// differences and all sums as compensated float32 pairs.  MIXED32: bead
// differences from float32 high/low parts, block-local products and sums in
// float32, the combination across blocks with float32 TwoSum compensation.
#include <type_traits>

#include "bpimd_internal.cuh"
#include "pairg.cuh"

namespace bpimd {
namespace {

// (float32 estimate of the triangular root, corrected with integer tests:
// no float64 instruction)
__device__ __forceinline__ void block_coords_f(int blk, int &t, int &s) {
  int tt = (int)((sqrtf(8.0f * (float)blk + 1.0f) - 1.0f) * 0.5f);
  while ((tt + 1) * (tt + 2) / 2 <= blk) ++tt;
  while (tt * (tt + 1) / 2 > blk) --tt;
  t = tt;
  s = blk - tt * (tt + 1) / 2;
}

__device__ __forceinline__ xd alpha_of(const Workspace &w, int a) {
  // y_a / (N y_N), stored by the forward recursion
  return xd{w.mixed ? (double)((const float *)w.alm)[a] : ((const double *)w.alm)[a], w.ale[a]};
}
__device__ __forceinline__ xd mu_of(const Workspace &w, int b) {
  const int r = w.N - 1 - b;  // backward row index of mu_b (0-based mu~_b = Yb[N-1-b])
  return xd{w.ybm[r], w.ybe[r]};
}

// Sum of float32 block partials, in the given order, to float64 accuracy on
// the float32 pipe: Knuth's TwoSum splits every addition into its rounded sum
// and exact rounding error, and the errors are carried alongside (float64
// additions would queue on the SM's slow float64 pipe: 16 per thread here).
struct fsum2 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v, bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
  }
  __device__ __forceinline__ void add2(float h, float l) {  // an unevaluated sum h + l
    add(h);
    c += l;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// 2^e as a double for e in the normal range (0 below it), built from the bits.
__device__ __forceinline__ double pow2_normal(int e) {
  return e < -1022 ? 0.0 : __longlong_as_double((long long)(min(e, 1023) + 1023) << 52);
}

// Pr[p -> p+1] = 1 - y_{p+1} B_{p+2} / (N y_N) (0-based p; Eq.
// direct-link-probability) with B_{p+2} = Yb[N-p-1] / c_{p+1}: one mantissa
// product and quotient in float64, the exponents summed as integers.
__device__ __forceinline__ double direct_link_fast(const Workspace &w, int p) {
  const double ym = w.yfm[p + 1], bm = w.ybm[w.N - p - 1], cm = w.ccm[p], zm = w.scal[1];
  const int e = w.yfe[p + 1] + w.ybe[w.N - p - 1] - w.cce[p] + w.scal_i[0];
  return 1.0 - ((ym * bm) * zm / cm) * pow2_normal(e);
}

template <bool PBC>
__device__ __forceinline__ double img(const Workspace &w, double d) {
  return PBC ? d - w.L * rint(d * w.invL) : d;
}

// Bead P of the 32 particles of row tile t: sum the row partials of blocks
// (t, 0..t) in that order, add the direct link, form F_l^P.  Run by the last
// block of the tile to finish; all 256 threads call it.  The finishing warp's
// loads are issued before the partial sums.
// Kinds of block partials: float64, float32, or an unevaluated float32 pair
// (high, low) written by the MIXED pass.
constexpr int PK_F64 = 0, PK_F32 = 1, PK_FF = 2;

template <int PK, bool PBC>
__device__ void finalize_rows(const Workspace &w, int t, const double *__restrict__ pos, double *__restrict__ F,
                              double (*fin)[9]) {
  const int q = threadIdx.x & 3, jj = (threadIdx.x >> 2) & 31, half = threadIdx.x >> 7;
  const int p = t * TILE + threadIdx.x;
  const bool mine = threadIdx.x < TILE && p < w.N;
  double M = 0.0, rp[3] = {0, 0, 0}, n1[3] = {0, 0, 0}, nb[3] = {0, 0, 0};
  if (mine) {
    const double *r = w.RP + 4 * (size_t)p, *nbP = pos + ((size_t)p * w.P + (w.P - 2)) * 3;  // bead P-1 (1-based)
#pragma unroll
    for (int c = 0; c < 3; ++c) { rp[c] = r[c]; nb[c] = nbP[c]; }
    if (p + 1 < w.N) {
      const double *n = w.R1 + 4 * (size_t)(p + 1);
#pragma unroll
      for (int c = 0; c < 3; ++c) n1[c] = n[c];
    }
  }
  const size_t base = (size_t)t * (t + 1) / 2;
  using P_t = typename std::conditional<PK == PK_F64, double, typename std::conditional<PK == PK_F32, float, float2>::type>::type;
  const P_t *part = (const P_t *)w.rowpart;
  double acc = 0.0;
  fsum2 f;
  // partials in chunks of 8 per thread, all loads of a chunk issued first;
  // the direct link's float64 chain runs while the first chunk is in flight
  for (int s0 = half; s0 <= t; s0 += 16) {
    P_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {  // index clamped into the tile: a valid address even if the load is speculated
      const int k = min(s0 + 2 * u, t);
      v[u] = (s0 + 2 * u <= t) ? __ldcg(part + ((base + k) * TILE + jj) * 4 + q) : P_t{};
    }
    if (s0 == half && mine && p + 1 < w.N) M = direct_link_fast(w, p);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if constexpr (PK == PK_F32) f.add(v[u]);
      else if constexpr (PK == PK_FF) f.add2(v[u].x, v[u].y);
      else acc += v[u];
    }
  }
  fin[jj][q + 4 * half] = PK == PK_F64 ? acc : f.value();
  __syncthreads();
  if (mine) {
    const double *fr = fin[threadIdx.x];
    double rs = fr[0] + fr[4] + M, r3[3] = {fr[1] + fr[5], fr[2] + fr[6], fr[3] + fr[7]};
    const double k = w.k;
    double *fP = F + ((size_t)p * w.P + (w.P - 1)) * 3;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double rc = fma(M, img<PBC>(w, rp[c] - n1[c]), r3[c]);
      fP[c] = -k * fma(rs, img<PBC>(w, rp[c] - nb[c]), rc);
      ok &= isfinite(fP[c]);
    }
    if (!ok) atomicOr(w.status, ST_NONFINITE);
  }
  if (threadIdx.x == 0) w.rowcnt[t] = 0;  // ready for the next evaluation
  __syncthreads();
}

// Bead 1 of the 32 particles of column tile s: blocks (s..NT-1, s) in order.
template <int PK, bool PBC>
__device__ void finalize_cols(const Workspace &w, int s, const double *__restrict__ pos, double *__restrict__ F,
                              double (*fin)[9]) {
  const int q = threadIdx.x & 3, ii = (threadIdx.x >> 2) & 31, half = threadIdx.x >> 7;
  const int p = s * TILE + threadIdx.x;
  const bool mine = threadIdx.x < TILE && p < w.N;
  double M = 0.0, r1[3] = {0, 0, 0}, pP[3] = {0, 0, 0}, nb[3] = {0, 0, 0};
  if (mine) {
    const double *r = w.R1 + 4 * (size_t)p, *nb1 = pos + ((size_t)p * w.P + 1) * 3;  // bead 2 (1-based)
#pragma unroll
    for (int c = 0; c < 3; ++c) { r1[c] = r[c]; nb[c] = nb1[c]; }
    if (p >= 1) {
      const double *n = w.RP + 4 * (size_t)(p - 1);
#pragma unroll
      for (int c = 0; c < 3; ++c) pP[c] = n[c];
    }
  }
  using P_t = typename std::conditional<PK == PK_F64, double, typename std::conditional<PK == PK_F32, float, float2>::type>::type;
  const P_t *part = (const P_t *)w.colpart;
  double acc = 0.0;
  fsum2 f;
  for (int t0 = s + half; t0 < w.NT; t0 += 16) {
    P_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = min(t0 + 2 * u, w.NT - 1);  // clamped into the tile: a valid address even if speculated
      v[u] = (t0 + 2 * u < w.NT) ? __ldcg(part + (((size_t)t * (t + 1) / 2 + s) * TILE + ii) * 4 + q) : P_t{};
    }
    if (t0 == s + half && mine && p >= 1) M = direct_link_fast(w, p - 1);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if constexpr (PK == PK_F32) f.add(v[u]);
      else if constexpr (PK == PK_FF) f.add2(v[u].x, v[u].y);
      else acc += v[u];
    }
  }
  fin[ii][q + 4 * half] = PK == PK_F64 ? acc : f.value();
  __syncthreads();
  if (mine) {
    const double *fc = fin[threadIdx.x];
    double cs = fc[0] + fc[4] + M, c3[3] = {fc[1] + fc[5], fc[2] + fc[6], fc[3] + fc[7]};
    const double k = w.k;
    double *f1 = F + (size_t)p * w.P * 3;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double cc = fma(M, img<PBC>(w, r1[c] - pP[c]), c3[c]);
      f1[c] = -k * fma(cs, img<PBC>(w, r1[c] - nb[c]), cc);
      ok &= isfinite(f1[c]);
    }
    if (!ok) atomicOr(w.status, ST_NONFINITE);
  }
  if (threadIdx.x == 0) w.colcnt[s] = 0;
  __syncthreads();
}

// One 32 x 32 block of the lower triangle (all 256 threads of the CTA).
// MIXED keeps the block partials in float32 (each is a float32 sum already).
template <bool MIXED, bool PBC>
__device__ __forceinline__ void prob_block(const Workspace &w, int blk, const double *__restrict__ pos,
                                           double *__restrict__ F,
                                           typename std::conditional<MIXED, float, double>::type (*red)[32][4],
                                           double (*fin)[9], int *last) {
  using P_t = typename std::conditional<MIXED, float, double>::type;
  {
    int t, s;
    block_coords_f(blk, t, s);
    const int j = threadIdx.x & 31, i0 = threadIdx.x >> 5;
    const int b = t * TILE + j;
    const bool bvalid = b < w.N;
    xd mub{0.0, XZERO_E};
    double bx = 0, by = 0, bz = 0;
    float4 bh = make_float4(0.f, 0.f, 0.f, 0.f), bl = bh;
    if (bvalid) {
      mub = mu_of(w, b);
      if (MIXED) {
        bh = *(const float4 *)(w.RPs + 8 * (size_t)b);
        bl = *(const float4 *)(w.RPs + 8 * (size_t)b + 4);
      } else {
        bx = w.RP[4 * b]; by = w.RP[4 * b + 1]; bz = w.RP[4 * b + 2];
      }
    }
    const float mubf = (float)mub.m;
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
        if (MIXED) {
          float fx, fy, fz;
          if (PBC) {  // minimum image from the fixed-point copies (bh holds RP's bits)
            const uint4 ua = *(const uint4 *)(w.R1s + 8 * (size_t)a);
            fx = fixdiff(__float_as_uint(bh.x), ua.x, w.Lscale);
            fy = fixdiff(__float_as_uint(bh.y), ua.y, w.Lscale);
            fz = fixdiff(__float_as_uint(bh.z), ua.z, w.Lscale);
          } else {
            const float4 ah = *(const float4 *)(w.R1s + 8 * (size_t)a);
            const float4 al4 = *(const float4 *)(w.R1s + 8 * (size_t)a + 4);
            fx = (bh.x - ah.x) + (bl.x - al4.x);
            fy = (bh.y - ah.y) + (bl.y - al4.y);
            fz = (bh.z - ah.z) + (bl.z - al4.z);
          }
          const float gmf = ((const float *)w.gm)[gi];
          const int e = ((const int *)w.ale)[a] + mub.e + w.ge[gi];
          float M = ((const float *)w.alm)[a] * mubf * gmf;
          M = (e < -150) ? 0.0f : (e > 0 ? M * (float)(1 << min(e, 2)) : M * pow2f_nonpos(e));
          frs += M; frx += M * fx; fry += M * fy; frz += M * fz;
          fcs = M; fcx = -M * fx; fcy = -M * fy; fcz = -M * fz;
        } else {
          const double dx = img<PBC>(w, bx - w.R1[4 * a]), dy = img<PBC>(w, by - w.R1[4 * a + 1]),
                       dz = img<PBC>(w, bz - w.R1[4 * a + 2]);
          const double gmd = ((const double *)w.gm)[gi];
          // alpha mu g with its exponent applied as an integer-built power of two
          const double M = (((const double *)w.alm)[a] * mub.m * gmd) * pow2_normal(w.ale[a] + mub.e + w.ge[gi]);
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
        P_t *cp = (P_t *)w.colpart + ((size_t)blk * TILE + i) * 4;
        if (MIXED) { cp[0] = fcs; cp[1] = fcx; cp[2] = fcy; cp[3] = fcz; }
        else { cp[0] = (P_t)cs; cp[1] = (P_t)cx; cp[2] = (P_t)cy; cp[3] = (P_t)cz; }
      }
    }
    if (MIXED) {
      red[i0][j][0] = frs; red[i0][j][1] = frx; red[i0][j][2] = fry; red[i0][j][3] = frz;
    } else {
      red[i0][j][0] = (P_t)rs; red[i0][j][1] = (P_t)rx; red[i0][j][2] = (P_t)ry; red[i0][j][3] = (P_t)rz;
    }
    __syncthreads();
    if (threadIdx.x < 128) {
      const int jj = threadIdx.x >> 2, q = threadIdx.x & 3;
      P_t acc = 0;
#pragma unroll
      for (int g = 0; g < 8; ++g) acc += red[g][jj][q];
      ((P_t *)w.rowpart)[((size_t)blk * TILE + jj) * 4 + q] = acc;
    }
    // publish this block's partials, then count it in its row and column tile;
    // the block that completes a tile forms that tile's forces (no waiting)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      last[0] = atomicAdd(w.rowcnt + t, 1) == t;             // blocks (t, 0..t)
      last[1] = atomicAdd(w.colcnt + s, 1) == w.NT - 1 - s;  // blocks (s..NT-1, s)
    }
    __syncthreads();
    const bool last_row = last[0], last_col = last[1];
    if (last_row || last_col) __threadfence();
    if (last_row) finalize_rows<MIXED ? PK_F32 : PK_F64, PBC>(w, t, pos, F, fin);
    if (last_col) finalize_cols<MIXED ? PK_F32 : PK_F64, PBC>(w, s, pos, F, fin);
  }
}

// Exterior-bead forces of one row tile (bead P) or column tile (bead 1) from
// complete sums fin[j][0..3] + fin[j][4..7] = (sum Pr, sum Pr (r - r')), used
// by the recompute pass (the same formulas as the tile finalisers above).
template <bool PBC>
__device__ void finish_rows(const Workspace &w, int t, const double *__restrict__ pos, double *__restrict__ F,
                            double (*fin)[9]) {
  const int p = t * TILE + threadIdx.x;
  if (threadIdx.x >= TILE || p >= w.N) return;
  const double *r = w.RP + 4 * (size_t)p, *nbP = pos + ((size_t)p * w.P + (w.P - 2)) * 3;  // bead P-1
  const double M = (p + 1 < w.N) ? direct_link_fast(w, p) : 0.0;
  const double *fr = fin[threadIdx.x];
  const double rs = fr[0] + fr[4] + M;
  double *fP = F + ((size_t)p * w.P + (w.P - 1)) * 3;
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double n1 = (p + 1 < w.N) ? w.R1[4 * (size_t)(p + 1) + c] : 0.0;
    const double rc = fma(M, img<PBC>(w, r[c] - n1), fr[1 + c] + fr[5 + c]);
    fP[c] = -w.k * fma(rs, img<PBC>(w, r[c] - nbP[c]), rc);
    ok &= isfinite(fP[c]);
  }
  if (!ok) atomicOr(w.status, ST_NONFINITE);
}
template <bool PBC>
__device__ void finish_cols(const Workspace &w, int s, const double *__restrict__ pos, double *__restrict__ F,
                            double (*fin)[9]) {
  const int p = s * TILE + threadIdx.x;
  if (threadIdx.x >= TILE || p >= w.N) return;
  const double *r = w.R1 + 4 * (size_t)p, *nb1 = pos + ((size_t)p * w.P + 1) * 3;  // bead 2
  const double M = (p >= 1) ? direct_link_fast(w, p - 1) : 0.0;
  const double *fc = fin[threadIdx.x];
  const double cs = fc[0] + fc[4] + M;
  double *f1 = F + (size_t)p * w.P * 3;
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double pP = (p >= 1) ? w.RP[4 * (size_t)(p - 1) + c] : 0.0;
    const double cc = fma(M, img<PBC>(w, r[c] - pP), fc[1 + c] + fc[5 + c]);
    f1[c] = -w.k * fma(cs, img<PBC>(w, r[c] - nb1[c]), cc);
    ok &= isfinite(f1[c]);
  }
  if (!ok) atomicOr(w.status, ST_NONFINITE);
}

// ----------------------------------------------------------- MIXED (config 3)
// Unevaluated sums h + l of two float32 numbers (|l| <= ulp(h)/2 after
// renormalisation): about 46 significant bits on the float32 pipe.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = a.h + b.h, bb = s - a.h;
  const float e = ((a.h - (s - bb)) + (b.h - bb)) + (a.l + b.l);
  const float h = s + e;
  return ff{h, e - (h - s)};
}
// a * d with a float32 d; a.h * d is exact by FMA (TwoProd)
__device__ __forceinline__ ff ff_mul(ff a, float d) {
  const float p = a.h * d;
  const float e = fmaf(a.h, d, -p) + a.l * d;
  const float h = p + e;
  return ff{h, e - (h - p)};
}

// Pr = alpha mu g of one pair from three extended numbers with double
// mantissas in [1, 2): the mantissa products on the integer pipe (64-bit
// truncations, 2^-62 relative), the exponents added as integers; returned as
// an unevaluated float32 pair (the mantissa cut at 2^-46), 0 below 2^-126.
__device__ __forceinline__ ff prob_ff(unsigned long long am, int e_am, double gm, int ge) {
  // am = (alpha mantissa)(mu mantissa) normalised to [2^63, 2^64), value am/2^63 2^e_am
  const unsigned long long gg = (((unsigned long long)__double_as_longlong(gm) & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11;
  unsigned long long pr = __umul64hi(am, gg);  // in [2^62, 2^64)
  const int sh = (int)(pr >> 63) ^ 1;
  pr <<= sh;
  const int E = e_am + ge + 1 - sh;  // Pr = (pr / 2^63) 2^E
  if (E < -126) return ff{0.0f, 0.0f};
  const float h = __uint_as_float((unsigned)((E + 127) << 23) | (unsigned)((pr >> 40) & 0x7FFFFFu));
  const float t = __uint_as_float(0x4B000000u | (unsigned)((pr >> 17) & 0x7FFFFFu)) - 8388608.0f;  // next 23 bits
  const float sc = (E - 46 >= -126) ? __uint_as_float((unsigned)((E - 46 + 127) << 23)) : 0.0f;
  return ff{h, t * sc};
}

// One 32 x 32 block of the lower triangle in the MIXED form (all 256
// threads).  Thread (i0 = warp, j = lane) forms the pairs (a = 32 s + i0 + 8 k,
// b = 32 t + j), k = 0..3: Pr and Pr (r_b^P - r_a^1) (float32 bead
// differences) as float32 pairs into the shared tile V[value][i][j]; then
// 128 threads sum the 32 rows b over their sources and 128 threads the 32
// columns a over their rows, in a fixed order, as float32 pairs.
template <bool PBC>
__device__ __forceinline__ void prob_block_mixed(const Workspace &w, int blk, const double *__restrict__ pos,
                                                 double *__restrict__ F, float (*V)[2][TILE][33], double (*fin)[9],
                                                 int *last) {
  int t, s;
  block_coords_f(blk, t, s);
  const int j = threadIdx.x & 31, i0 = threadIdx.x >> 5;
  const int b = t * TILE + j;
  const bool bvalid = b < w.N;
  unsigned long long mum = 0;
  int mue = 0;
  float4 bh = make_float4(0.f, 0.f, 0.f, 0.f), bl = bh;
  if (bvalid) {
    const xd mub = mu_of(w, b);
    mum = (((unsigned long long)__double_as_longlong(mub.m) & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11;
    mue = mub.e;
    bh = *(const float4 *)(w.RPs + 8 * (size_t)b);
    bl = *(const float4 *)(w.RPs + 8 * (size_t)b + 4);
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int i = i0 + 8 * kk;
    const int a = s * TILE + i;
    ff pr{0.0f, 0.0f}, px{0.0f, 0.0f}, py{0.0f, 0.0f}, pz{0.0f, 0.0f};
    if (bvalid && a <= b) {
      float fx, fy, fz;
      if (PBC) {  // minimum image from the fixed-point copies (bh holds RP's bits)
        const uint4 ua = *(const uint4 *)(w.R1s + 8 * (size_t)a);
        fx = fixdiff(__float_as_uint(bh.x), ua.x, w.Lscale);
        fy = fixdiff(__float_as_uint(bh.y), ua.y, w.Lscale);
        fz = fixdiff(__float_as_uint(bh.z), ua.z, w.Lscale);
      } else {
        const float4 ah = *(const float4 *)(w.R1s + 8 * (size_t)a);
        const float4 al4 = *(const float4 *)(w.R1s + 8 * (size_t)a + 4);
        fx = (bh.x - ah.x) + (bl.x - al4.x);
        fy = (bh.y - ah.y) + (bl.y - al4.y);
        fz = (bh.z - ah.z) + (bl.z - al4.z);
      }
      const size_t gi = (size_t)blk * TILE2 + i * TILE + j;
      const double alm = ((const double *)w.alm)[a];
      const unsigned long long aa = (((unsigned long long)__double_as_longlong(alm) & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11;
      unsigned long long am = __umul64hi(aa, mum);  // in [2^62, 2^64)
      const int sh = (int)(am >> 63) ^ 1;
      am <<= sh;
      pr = prob_ff(am, w.ale[a] + mue + 1 - sh, ((const double *)w.gm)[gi], w.ge[gi]);
      px = ff_mul(pr, fx);
      py = ff_mul(pr, fy);
      pz = ff_mul(pr, fz);
    }
    V[0][0][i][j] = pr.h; V[0][1][i][j] = pr.l;
    V[1][0][i][j] = px.h; V[1][1][i][j] = px.l;
    V[2][0][i][j] = py.h; V[2][1][i][j] = py.l;
    V[3][0][i][j] = pz.h; V[3][1][i][j] = pz.l;
  }
  __syncthreads();
  {
    const int q = (threadIdx.x >> 5) & 3, r = threadIdx.x & 31;
    ff acc{0.0f, 0.0f};
    if (threadIdx.x < 128) {  // row r (particle b = 32 t + r): sum over the sources i
#pragma unroll 8
      for (int i = 0; i < TILE; ++i) acc = ff_add(acc, ff{V[q][0][i][r], V[q][1][i][r]});
      ((float2 *)w.rowpart)[((size_t)blk * TILE + r) * 4 + q] = make_float2(acc.h, acc.l);
    } else {  // column r (particle a = 32 s + r): sum over the rows j; bead-1 sums carry r_a^1 - r_b^P
#pragma unroll 8
      for (int jj = 0; jj < TILE; ++jj) acc = ff_add(acc, ff{V[q][0][r][jj], V[q][1][r][jj]});
      const float sg = q == 0 ? 1.0f : -1.0f;
      ((float2 *)w.colpart)[((size_t)blk * TILE + r) * 4 + q] = make_float2(sg * acc.h, sg * acc.l);
    }
  }
  // publish this block's partials, then count it in its row and column tile;
  // the block that completes a tile forms that tile's forces (no waiting)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last[0] = atomicAdd(w.rowcnt + t, 1) == t;             // blocks (t, 0..t)
    last[1] = atomicAdd(w.colcnt + s, 1) == w.NT - 1 - s;  // blocks (s..NT-1, s)
  }
  __syncthreads();
  const bool last_row = last[0], last_col = last[1];
  if (last_row || last_col) __threadfence();
  if (last_row) finalize_rows<PK_FF, PBC>(w, t, pos, F, fin);
  if (last_col) finalize_cols<PK_FF, PBC>(w, s, pos, F, fin);
}

__global__ void __launch_bounds__(256, 4) prob_force_kernel_mixed(Workspace w, const double *__restrict__ pos,
                                                               double *__restrict__ F) {
  __shared__ float V[4][2][TILE][33];
  __shared__ double fin[32][9];
  __shared__ int last[2];
  pdl_wait();
  for (int blk = blockIdx.x; blk < w.NB; blk += gridDim.x) {
    if (w.pbc) prob_block_mixed<true>(w, blk, pos, F, V, fin, last);
    else prob_block_mixed<false>(w, blk, pos, F, V, fin, last);
    __syncthreads();  // V is rewritten by the next block
  }
  pdl_trigger();
}

__global__ void __launch_bounds__(256, 4) prob_force_batched_mixed(const Workspace *__restrict__ ws,
                                                                const int2 *__restrict__ tab, int ntab,
                                                                const long long *__restrict__ off,
                                                                const double *__restrict__ pos,
                                                                double *__restrict__ F) {
  __shared__ float V[4][2][TILE][33];
  __shared__ double fin[32][9];
  __shared__ int last[2];
  pdl_wait();
  for (int k = blockIdx.x; k < ntab; k += gridDim.x) {
    const int2 e = tab[k];
    if (ws[e.x].pbc) prob_block_mixed<true>(ws[e.x], e.y, pos + off[e.x], F + off[e.x], V, fin, last);
    else prob_block_mixed<false>(ws[e.x], e.y, pos + off[e.x], F + off[e.x], V, fin, last);
    __syncthreads();
  }
  pdl_trigger();
}

// ------------------------------------------------- recompute mode (no table)
// Probabilities and exterior forces by whole tiles: work item 2k is row tile
// NT-1-k (all its source tiles), item 2k+1 column tile k (all its row tiles),
// so that the items come in decreasing size.  A row item forms Pr[b -> a] for
// its 32 rows b (lanes) and every source a (8 warps, 4 sources each per 32x32
// block), with g recomputed from the endpoint copies, and accumulates the row
// sums in registers; the column items do the same for the 32 columns.  Every
// pair is formed twice (once per item kind) and nothing O(N^2) is stored; the
// sums are combined across warps in a fixed order (deterministic).
// Accumulators: float64 (FP64) or compensated float32 pairs (mixed forms).
template <int MODE>
struct PAcc {
  using T = typename std::conditional<MODE == BPIMD_FP64, double, ff>::type;
  T s, x, y, z;
  __device__ __forceinline__ void zero() {
    if constexpr (MODE == BPIMD_FP64) s = x = y = z = 0.0;
    else s = x = y = z = ff{0.0f, 0.0f};
  }
};

// Pr(a, b) for the recompute items: alpha_a, mu_b and g as extended numbers.
template <int MODE>
__device__ __forceinline__ typename PAcc<MODE>::T prob_rc(const Workspace &w, int a, xd mu, double gm, int ge) {
  if constexpr (MODE == BPIMD_FP64) {
    return (((const double *)w.alm)[a] * mu.m * gm) * pow2_normal(w.ale[a] + mu.e + ge);
  } else if constexpr (MODE == BPIMD_MIXED) {
    const unsigned long long aa =
        (((unsigned long long)__double_as_longlong(((const double *)w.alm)[a]) & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11;
    const unsigned long long mm = (((unsigned long long)__double_as_longlong(mu.m) & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11;
    unsigned long long am = __umul64hi(aa, mm);
    const int sh = (int)(am >> 63) ^ 1;
    am <<= sh;
    return prob_ff(am, w.ale[a] + mu.e + 1 - sh, gm, ge);
  } else {
    const int e = w.ale[a] + mu.e + ge;
    float M = ((const float *)w.alm)[a] * (float)mu.m * (float)gm;
    M = (e < -150) ? 0.0f : (e > 0 ? M * (float)(1 << min(e, 2)) : M * pow2f_nonpos(e));
    return ff{M, 0.0f};
  }
}

template <int MODE, typename D3>
__device__ __forceinline__ void acc_add(PAcc<MODE> &A, typename PAcc<MODE>::T pr, D3 d, float sign) {
  if constexpr (MODE == BPIMD_FP64) {
    A.s += pr;
    A.x = fma(sign * pr, d.x, A.x);
    A.y = fma(sign * pr, d.y, A.y);
    A.z = fma(sign * pr, d.z, A.z);
  } else {
    A.s = ff_add(A.s, pr);
    A.x = ff_add(A.x, ff_mul(pr, sign * d.x));
    A.y = ff_add(A.y, ff_mul(pr, sign * d.y));
    A.z = ff_add(A.z, ff_mul(pr, sign * d.z));
  }
}

template <int MODE>
__device__ __forceinline__ double acc_val(typename PAcc<MODE>::T v) {
  if constexpr (MODE == BPIMD_FP64) return v;
  else return (double)v.h + (double)v.l;
}

// One work item of the recompute pass (all 256 threads).  red: [8][32][4]
// per-warp sums; fin as in the tile finalisers.
template <int MODE, bool PBC>
__device__ void prob_item_rc(const Workspace &w, int item, const double *__restrict__ pos, double *__restrict__ F,
                             const unsigned long long *T63, double (*red)[32][4], double (*fin)[9]) {
  using EP = pairg::EndPt<MODE != BPIMD_FP64, PBC>;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const bool row_item = !(item & 1);
  const int tile = row_item ? w.NT - 1 - (item >> 1) : (item >> 1);
  const int me = tile * TILE + lane;  // this lane's particle (row b or column a)
  PAcc<MODE> A;
  A.zero();
  if (me < w.N) {
    const EP mine = pairg::load_end<MODE != BPIMD_FP64, PBC>(w, me, row_item);  // bead P of b, or bead 1 of a
    const xd mub = row_item ? mu_of(w, me) : xd{0.0, 0};
    const int t0 = row_item ? 0 : tile, t1 = row_item ? tile : w.NT - 1;
    for (int o = t0; o <= t1; ++o) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int other = o * TILE + wp + 8 * kk;  // source a (row item) or row b (column item)
        const int a = row_item ? other : me, b = row_item ? me : other;
        if (a <= b && b < w.N) {
          const EP oth = pairg::load_end<MODE != BPIMD_FP64, PBC>(w, other, !row_item);
          const EP &eb = row_item ? mine : oth, &ea = row_item ? oth : mine;
          int ge;
          const double gm = (double)pairg::g_of<MODE, PBC>(w, eb, ea, w.cx, T63, ge);
          const auto pr = prob_rc<MODE>(w, a, row_item ? mub : mu_of(w, b), gm, ge);
          // row b: Pr (r_b^P - r_a^1); column a: Pr (r_a^1 - r_b^P)
          acc_add<MODE>(A, pr, pairg::diff3(w, eb, ea), row_item ? 1.0f : -1.0f);
        }
      }
    }
  }
  red[wp][lane][0] = acc_val<MODE>(A.s);
  red[wp][lane][1] = acc_val<MODE>(A.x);
  red[wp][lane][2] = acc_val<MODE>(A.y);
  red[wp][lane][3] = acc_val<MODE>(A.z);
  __syncthreads();
  if (threadIdx.x < 128) {  // fixed-order sum over the 8 warps, into the finalisers' layout
    const int jj = threadIdx.x >> 2, q = threadIdx.x & 3;
    double v = 0.0;
#pragma unroll
    for (int g = 0; g < 8; ++g) v += red[g][jj][q];
    fin[jj][q] = v;
    fin[jj][q + 4] = 0.0;
  }
  __syncthreads();
  if (row_item) finish_rows<PBC>(w, tile, pos, F, fin);
  else finish_cols<PBC>(w, tile, pos, F, fin);
  __syncthreads();
}

template <int MODE>
__global__ void __launch_bounds__(256) prob_rc_kernel(Workspace w, const double *__restrict__ pos,
                                                      double *__restrict__ F) {
  __shared__ double red[8][32][4];
  __shared__ double fin[32][9];
  __shared__ unsigned long long T63[256];
  if (MODE != BPIMD_MIXED32) pairg::table_init(T63);
  __syncthreads();
  pdl_wait();
  for (int item = blockIdx.x; item < 2 * w.NT; item += gridDim.x) {
    if (w.pbc) prob_item_rc<MODE, true>(w, item, pos, F, T63, red, fin);
    else prob_item_rc<MODE, false>(w, item, pos, F, T63, red, fin);
  }
  pdl_trigger();
}

template <bool MIXED>
__global__ void __launch_bounds__(256, 4) prob_force_kernel(Workspace w, const double *__restrict__ pos,
                                                         double *__restrict__ F) {
  using P_t = typename std::conditional<MIXED, float, double>::type;
  __shared__ P_t red[8][32][4];
  __shared__ double fin[32][9];
  __shared__ int last[2];
  pdl_wait();
  for (int blk = blockIdx.x; blk < w.NB; blk += gridDim.x) {
    if (w.pbc) prob_block<MIXED, true>(w, blk, pos, F, red, fin, last);
    else prob_block<MIXED, false>(w, blk, pos, F, red, fin, last);
  }
  pdl_trigger();
}

// Replica batch: entry k of tab is (replica, block); positions and forces of
// replica r start at element off[r] of the packed arrays.
template <bool MIXED>
__global__ void __launch_bounds__(256, 4) prob_force_batched(const Workspace *__restrict__ ws,
                                                          const int2 *__restrict__ tab, int ntab,
                                                          const long long *__restrict__ off,
                                                          const double *__restrict__ pos, double *__restrict__ F) {
  using P_t = typename std::conditional<MIXED, float, double>::type;
  __shared__ P_t red[8][32][4];
  __shared__ double fin[32][9];
  __shared__ int last[2];
  pdl_wait();  // launched as a programmatic dependent of the recursions: their epilogue must be complete
  for (int k = blockIdx.x; k < ntab; k += gridDim.x) {
    const int2 e = tab[k];
    if (ws[e.x].pbc) prob_block<MIXED, true>(ws[e.x], e.y, pos + off[e.x], F + off[e.x], red, fin, last);
    else prob_block<MIXED, false>(ws[e.x], e.y, pos + off[e.x], F + off[e.x], red, fin, last);
  }
  pdl_trigger();
}

// Expected exterior-spring energy over representative permutations, per block
// of the lower triangle: (1/2) m w_P^2 sum_{a<=b in block} Pr[b -> a] |r_b^P - r_a^1|^2
// (the direct links l -> l+1 are added by the caller).  Float64 throughout;
// run once per molecular-dynamics call, for the primitive energy estimator.
// All threads of the block call it; thread 0 gets the sum.
__device__ double spring_block(const Workspace &w, int blk, double *red) {
  int t, s;
  block_coords_f(blk, t, s);
  double acc = 0.0;
  for (int e = threadIdx.x; e < TILE2; e += blockDim.x) {
    const int a = s * TILE + (e >> 5), b = t * TILE + (e & 31);
    if (b < w.N && a <= b) {
      const size_t gi = (size_t)blk * TILE2 + e;
      const xd g = w.recomp ? pairg::g_runtime(w, a, b)
                            : xd{w.mixed ? (double)((const float *)w.gm)[gi] : ((const double *)w.gm)[gi], w.ge[gi]};
      const xd al = alpha_of(w, a), mu = mu_of(w, b);
      const double M = xtod(xd{al.m * mu.m * g.m, al.e + mu.e + g.e});
      const double dx = mimage(w, w.RP[4 * b] - w.R1[4 * a]), dy = mimage(w, w.RP[4 * b + 1] - w.R1[4 * a + 1]),
                   dz = mimage(w, w.RP[4 * b + 2] - w.R1[4 * a + 2]);
      acc += M * (dx * dx + dy * dy + dz * dz);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  double sum = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += red[q];
  __syncthreads();
  return w.half_k * sum;
}

__global__ void __launch_bounds__(256) spring_expect_kernel(Workspace w, double *part) {
  __shared__ double red[8];
  for (int blk = blockIdx.x; blk < w.NB; blk += gridDim.x) {
    const double v = spring_block(w, blk, red);
    if (threadIdx.x == 0) part[blk] = v;
  }
}

// Replica batch: entry k of tab is (replica, block); part[k] as above.
__global__ void __launch_bounds__(256) spring_expect_batched(const Workspace *__restrict__ ws,
                                                             const int2 *__restrict__ tab, int ntab, double *part) {
  __shared__ double red[8];
  for (int k = blockIdx.x; k < ntab; k += gridDim.x) {
    const int2 e = tab[k];
    const double v = spring_block(ws[e.x], e.y, red);
    if (threadIdx.x == 0) part[k] = v;
  }
}

__global__ void dense_prob_kernel(Workspace w, double *M) {
  const size_t NN = (size_t)w.N * w.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx / w.N), a = (int)(idx % w.N);  // row l = b, column l' = a
    double v = 0.0;
    if (a <= b) {
      const int t = b >> 5, s = a >> 5;
      const size_t gi = ((size_t)(t * (t + 1) / 2 + s) << 10) + ((a & 31) << 5) + (b & 31);
      const xd g = w.recomp ? pairg::g_runtime(w, a, b)
                            : xd{w.mixed ? (double)((const float *)w.gm)[gi] : ((const double *)w.gm)[gi], w.ge[gi]};
      const xd al = alpha_of(w, a), mu = mu_of(w, b);
      v = xtod(xd{al.m * mu.m * g.m, al.e + mu.e + g.e});
    } else if (a == b + 1) {
      v = direct_link_prob(w, b);
    }
    M[idx] = v;
  }
}

}  // namespace

cudaError_t launch_prob_forces(const Workspace &w, const double *pos, double *F, cudaStream_t s) {
  const int sms = sm_count();
  cudaError_t e;
  if (w.recomp) {
    const int items = 2 * w.NT, grid_rc = items < sms * 4 ? items : sms * 4;
    switch (w.mode) {
      case BPIMD_FP64: e = launch_pdl(prob_rc_kernel<BPIMD_FP64>, grid_rc, 256, 0, s, w, pos, F); break;
      case BPIMD_MIXED: e = launch_pdl(prob_rc_kernel<BPIMD_MIXED>, grid_rc, 256, 0, s, w, pos, F); break;
      default: e = launch_pdl(prob_rc_kernel<BPIMD_MIXED32>, grid_rc, 256, 0, s, w, pos, F); break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  const int grid = w.NB < sms * 8 ? w.NB : sms * 8;
  switch (w.mode) {
    case BPIMD_FP64: e = launch_pdl(prob_force_kernel<false>, grid, 256, 0, s, w, pos, F); break;
    case BPIMD_MIXED: e = launch_pdl(prob_force_kernel_mixed, grid, 256, 0, s, w, pos, F); break;
    default: e = launch_pdl(prob_force_kernel<true>, grid, 256, 0, s, w, pos, F); break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_spring_expectation(const Workspace &w, double *part, cudaStream_t s) {
  const int sms = sm_count();
  const int grid = w.NB < sms * 4 ? w.NB : sms * 4;
  spring_expect_kernel<<<grid, 256, 0, s>>>(w, part);
  return cudaGetLastError();
}

cudaError_t launch_spring_expectation_batched(const Workspace *ws, const int2 *tab, int ntab, double *part,
                                             cudaStream_t s) {
  if (ntab <= 0) return cudaSuccess;
  const int sms = sm_count();
  const int grid = ntab < sms * 4 ? ntab : sms * 4;
  spring_expect_batched<<<grid, 256, 0, s>>>(ws, tab, ntab, part);
  return cudaGetLastError();
}

cudaError_t launch_dense_probabilities(const Workspace &w, double *M, cudaStream_t s) {
  dense_prob_kernel<<<1024, 256, 0, s>>>(w, M);
  return cudaGetLastError();
}

cudaError_t launch_prob_forces_batched(const Workspace *ws, const int2 *tab, int ntab, const long long *off,
                                      int mode, const double *pos, double *F, int blocks_per_sm, cudaStream_t s) {
  if (ntab <= 0) return cudaSuccess;
  const int sms = sm_count();
  const int cap = sms * (blocks_per_sm > 0 ? blocks_per_sm : 8);
  const int grid = ntab < cap ? ntab : cap;
  cudaError_t e;
  switch (mode) {
    case BPIMD_FP64: e = launch_pdl(prob_force_batched<false>, grid, 256, 0, s, ws, tab, ntab, off, pos, F); break;
    case BPIMD_MIXED: e = launch_pdl(prob_force_batched_mixed, grid, 256, 0, s, ws, tab, ntab, off, pos, F); break;
    default: e = launch_pdl(prob_force_batched<true>, grid, 256, 0, s, ws, tab, ntab, off, pos, F); break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace bpimd
