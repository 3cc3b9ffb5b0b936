// Preparation of one evaluation: the bead pass and the pair Boltzmann
// factors, in one launch (the first blocks take the bead pass, the rest the
// pair factors; the pair-factor blocks read the two endpoint beads they need
// straight from the positions, so neither part waits for the other).
//
// Bead pass, per particle l (one warp for the bead sums, then one lane for the rest):
//   E_int^{(l)} = (1/2) m w_P^2 sum_{j=1}^{P-1} (r_l^{j+1} - r_l^j)^2     (Eq. e-interior)
//   link_l      = (1/2) m w_P^2 (r_l^P - r_{l+1}^1)^2, 0 for l = N       (spring of Eq. e-recurrence-step)
//   interior forces -m w_P^2 (2 r_l^j - r_l^{j+1} - r_l^{j-1}), j=2..P-1  (Eq. intermediate-bead-force)
//   copies of r_l^1 and r_l^P for the probability pass (MIXED: also as
//   float32 high/low parts, or 32-bit fixed point in a box), and the
//   coefficient c_l = exp(beta link_l)/l of the linear-space recursions, as
//   an extended number.
// FP64: everything in float64.  MIXED: bead differences formed in float64,
// rounded to float32; squares, warp sums and interior forces in float32;
// E_int and link widened to float64.
//
// Pair factors: g(u,v) = exp(-beta (1/2) m w_P^2 (r_v^P - r_u^1)^2) for every
// u <= v -- the closing-spring factor of the cycle energy E^{[u,v]} (Eq.
// e-recurrence-step, last term) -- stored once per evaluation as an extended
// number 2^x = mantissa(2^frac(x)) * 2^floor(x), x = -beta (1/2)k |d|^2 log2(e).
// FP64: float64 difference and square; 2^x by the integer-pipe fixed-point
// method of pow2_fixed.cuh on the exact product of the square and the
// constant.  MIXED: difference of the float32 high/low parts (or fixed-point
// copies) of the positions, float32 square, the same integer method on the
// exact float32 x float64 product (MIXED32: hardware ex2.approx).  The potentials V^{[1,v]}, V^{[u,N]} for
// diagnostics are computed on demand by diag_potentials_kernel.
#include <type_traits>

#include "bpimd_internal.cuh"
#include "pairg.cuh"

namespace bpimd {
namespace {

constexpr int BEAD_WARPS = BEAD_BLOCK_PARTICLES;  // particles per block (one warp each)
static_assert(32 * BEAD_WARPS == 256, "bead-pass and pair-factor blocks share one launch shape");

// Non-finite test on the exponent bits (integer instructions only).
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// Phase 1 of the bead pass for one particle (one warp).  The particle's
// [P][3] row is contiguous: each chunk of 32 beads (and the first bead of the
// next chunk) is staged into the warp's shared buffer with coalesced 16-byte
// loads (8-byte loads where the row is not 16-byte aligned, i.e. odd P and odd
// particle index).  Lane j then forms the spring vector d_j = r^{j+1} - r^j
// (minimum image in a box) once; the interior force on bead j is
// k (d_j - d_{j-1}), with d_{j-1} taken from the neighbouring lane (lane 0
// from lane 31 of the previous chunk).  Adds sum |d_j|^2 to s32 (MIXED) or s64
// (FP64).
constexpr int STAGE_DOUBLES = 3 * 33 + 1;  // 33 beads, padded to a 16-byte multiple
template <bool MIXED, bool PBC>
__device__ __forceinline__ void bead_springs(const Workspace &w, const double *__restrict__ p,
                                             double *__restrict__ f, int lane, bool &finite, float &s32,
                                             double &s64, double *__restrict__ stage) {
  using D_t = typename std::conditional<MIXED, float, double>::type;
  const int P = w.P;
  const D_t kk = (D_t)w.k;
  D_t cx = 0, cy = 0, cz = 0;  // d_{j0-1} carried from the previous chunk
  const bool aligned = (((uintptr_t)p) & 15) == 0;  // warp-uniform
  for (int j0 = 0; j0 < P; j0 += 32) {
    const int nd = 3 * min(33, P - j0);  // doubles of beads j0 .. j0+32 that exist
    const double *src = p + 3 * j0;      // 16-byte aligned with p (3 * 32 doubles per chunk)
    __syncwarp();                        // the previous chunk's reads of the buffer are done
    if (aligned) {
      for (int i = lane; i < nd / 2; i += 32) ((double2 *)stage)[i] = __ldg((const double2 *)src + i);
      if ((nd & 1) && lane == 0) stage[nd - 1] = __ldg(src + nd - 1);
    } else {
      for (int i = lane; i < nd; i += 32) stage[i] = __ldg(src + i);
    }
    __syncwarp();
    const int j = j0 + lane;
    double dx = 0.0, dy = 0.0, dz = 0.0;
    if (j < P) {
      const double x = stage[3 * lane], y = stage[3 * lane + 1], z = stage[3 * lane + 2];
      finite &= finite_bits(x) && finite_bits(y) && finite_bits(z);
      if (j + 1 < P) {
        dx = stage[3 * lane + 3] - x;
        dy = stage[3 * lane + 4] - y;
        dz = stage[3 * lane + 5] - z;
        if (PBC) { dx = mimage(w, dx); dy = mimage(w, dy); dz = mimage(w, dz); }
      }
    }
    const D_t ex = (D_t)dx, ey = (D_t)dy, ez = (D_t)dz;
    if (MIXED) s32 = fmaf((float)ex, (float)ex, fmaf((float)ey, (float)ey, fmaf((float)ez, (float)ez, s32)));
    else s64 = fma(dx, dx, fma(dy, dy, fma(dz, dz, s64)));
    D_t qx = __shfl_up_sync(0xffffffffu, ex, 1), qy = __shfl_up_sync(0xffffffffu, ey, 1),
        qz = __shfl_up_sync(0xffffffffu, ez, 1);
    if (lane == 0) { qx = cx; qy = cy; qz = cz; }
    if (j >= 1 && j + 1 < P) {  // interior bead (0-based 1..P-2)
      f[3 * j] = (double)(kk * (ex - qx));
      f[3 * j + 1] = (double)(kk * (ey - qy));
      f[3 * j + 2] = (double)(kk * (ez - qz));
    }
    cx = __shfl_sync(0xffffffffu, ex, 31);
    cy = __shfl_sync(0xffffffffu, ey, 31);
    cz = __shfl_sync(0xffffffffu, ez, 31);
  }
}

// Particles l0 .. l0+7 of one system (all threads of the block).  MIXED:
// the float32 bead pass of both mixed forms.
template <bool MIXED>
__device__ __forceinline__ void bead_pass_body(const Workspace &w, const double *__restrict__ pos,
                                               double *__restrict__ F, int l0) {
  __shared__ double eint_s[BEAD_WARPS];
  __shared__ int finite_s[BEAD_WARPS];
  __shared__ __align__(16) double stage_s[BEAD_WARPS][STAGE_DOUBLES];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int P = w.P;
  // phase 1: one warp per particle -- interior springs and interior forces
  {
    const int l = l0 + wp;
    bool finite = true;
    double s64 = 0.0;
    float s32 = 0.0f;
    if (l < w.N) {  // warp-uniform
      const double *p = pos + (size_t)l * P * 3;
      double *f = F + (size_t)l * P * 3;
      if (w.pbc) bead_springs<MIXED, true>(w, p, f, lane, finite, s32, s64, stage_s[wp]);
      else bead_springs<MIXED, false>(w, p, f, lane, finite, s32, s64, stage_s[wp]);
    }
    if (MIXED) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s32 += __shfl_xor_sync(0xffffffffu, s32, o);
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, o);
    }
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
      eint_s[wp] = w.half_k * (MIXED ? (double)s32 : s64);
      finite_s[wp] = finite;
    }
  }
  __syncthreads();
  // phase 2: one lane per particle -- links, endpoint copies and the
  // coefficient c (the float64 transcendentals run once per 8 particles)
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
        *(uint4 *)(w.R1s + 8 * (size_t)l) =
            make_uint4(to_fixed(b1[0], w.invL32), to_fixed(b1[1], w.invL32), to_fixed(b1[2], w.invL32), 0u);
        *(uint4 *)(w.RPs + 8 * (size_t)l) =
            make_uint4(to_fixed(bP[0], w.invL32), to_fixed(bP[1], w.invL32), to_fixed(bP[2], w.invL32), 0u);
      } else if (MIXED) {  // float32 high + low parts
        float h1[3], l1[3], hP[3], lP[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          split_hi_lo(b1[c], h1[c], l1[c]);
          split_hi_lo(bP[c], hP[c], lP[c]);
        }
        float4 *s1 = (float4 *)(w.R1s + 8 * (size_t)l), *sp = (float4 *)(w.RPs + 8 * (size_t)l);
        s1[0] = make_float4(h1[0], h1[1], h1[2], 0.0f);
        s1[1] = make_float4(l1[0], l1[1], l1[2], 0.0f);
        sp[0] = make_float4(hP[0], hP[1], hP[2], 0.0f);
        sp[1] = make_float4(lP[0], lP[1], lP[2], 0.0f);
      }
      // c_{l+1} = exp(beta link_l) / (l+1) = 2^f 2^n / (l+1) with
      // x = beta link_l log2(e) = n + f, n integer, f in [0, 1).  x is formed
      // as an unevaluated double-double sum (exact products by FMA, log2(e) to
      // 106 bits), so f is accurate to a float64 rounding however large x is.
      // The integer part n goes into c's exponent and nowhere else: the
      // recursions' exponents carry sum n, and the reduced prefix sums
      //   C'[v] = sum_{i<=v} (E_int^(i) + link_i - n_i ln2/beta)
      //         = sum_{i<=v} (E_int^(i) + f_i ln2/beta)
      // exclude it, so V = C' - (ln y - (sum n) ln 2)/beta is formed from
      // numbers of the size of V itself (no cancellation against the open
      // chain's link energies).  x is clamped to 2^28 so that exponent sums
      // stay in int32.
      int n = 0;
      double f = 0.0;
      {
        const double p = w.beta * lk, pe = fma(w.beta, lk, -p);
        double xh = p * LOG2E;
        double xl = fma(p, LOG2E, -xh) + fma(pe, LOG2E, p * LOG2E_LO);
        if (xh >= 268435456.0) { xh = 268435456.0; xl = 0.0; }
        double nf = floor(xh);
        if (nf == xh && xl < 0.0) nf -= 1.0;
        n = (int)nf;
        f = (xh - nf) + xl;
      }
      const xd c = xnorm(exp2(f) / (double)(l + 1), n);
      w.ccm[l] = c.m;
      w.cce[l] = c.e;
      w.nexp[l] = n;
      w.Ap[l] = eint_s[lane] + f * (LN2 / w.beta);
    }
  }
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

// Endpoint beads of one block of g, staged in shared memory: side 0 holds
// bead P of the 32 particles b of row tile t, side 1 bead 1 of the 32
// particles a of source tile s.  FP64: x, y, z as doubles.  MIXED and
// MIXED32: float32 high parts then low parts (8 floats), or in a box the
// 32-bit fixed-point fractions of L (4 words); the same conversions as the
// bead pass's copies.
struct EndTiles {
  double v[2][TILE][4];
};

template <bool B32>
__device__ __forceinline__ void stage_endpoints(const Workspace &w, const double *__restrict__ pos, int t, int s,
                                                EndTiles &E) {
  if (threadIdx.x < 2 * TILE) {
    const int side = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = (side ? s : t) * TILE + lane;
    double x = 0.0, y = 0.0, z = 0.0;
    if (q < w.N) {
      const double *p = pos + ((size_t)q * w.P + (side ? 0 : w.P - 1)) * 3;
      x = p[0]; y = p[1]; z = p[2];
    }
    double *d = E.v[side][lane];
    if (!B32) {
      d[0] = x; d[1] = y; d[2] = z;
    } else if (w.pbc) {
      *(uint4 *)d = make_uint4(to_fixed(x, w.invL32), to_fixed(y, w.invL32), to_fixed(z, w.invL32), 0u);
    } else {
      float hx, lx, hy, ly, hz, lz;
      split_hi_lo(x, hx, lx);
      split_hi_lo(y, hy, ly);
      split_hi_lo(z, hz, lz);
      ((float4 *)d)[0] = make_float4(hx, hy, hz, 0.0f);
      ((float4 *)d)[1] = make_float4(lx, ly, lz, 0.0f);
    }
  }
  __syncthreads();
}

// g for one pair from the staged bead-P position of b (slot j of side 0) and
// bead-1 position of a (slot i of side 1): returns the mantissa (float for
// MIXED32, else double in [1, 2)) and sets the exponent (pairg.cuh; the
// recompute mode forms the same bits from the bead pass's copies).
template <int MODE, bool PBC>
__device__ __forceinline__ double pair_factor(const Workspace &w, double cx, const EndTiles &E, int i, int j,
                                              int &e, const unsigned long long *T63) {
  using EP = pairg::EndPt<MODE != BPIMD_FP64, PBC>;
  EP rb, ra;
  if constexpr (MODE == BPIMD_FP64) {
    rb = EP{E.v[0][j][0], E.v[0][j][1], E.v[0][j][2]};
    ra = EP{E.v[1][i][0], E.v[1][i][1], E.v[1][i][2]};
  } else if constexpr (PBC) {
    rb.u = *(const uint4 *)E.v[0][j];
    ra.u = *(const uint4 *)E.v[1][i];
  } else {
    rb.h = ((const float4 *)E.v[0][j])[0];
    rb.l = ((const float4 *)E.v[0][j])[1];
    ra.h = ((const float4 *)E.v[1][i])[0];
    ra.l = ((const float4 *)E.v[1][i])[1];
  }
  return (double)pairg::g_of<MODE, PBC>(w, rb, ra, cx, T63, e);
}

// One pass over the forward blocks (a = s*32+i, b = t*32+j): each valid pair
// a <= b < N is evaluated once and stored in both copies -- the forward one
// directly (coalesced along b), the backward one (row r = N-1-a, source
// w = N-1-b) after a transpose through shared memory, so that those stores
// are coalesced along r.  Entries outside a <= b < N are never written here
// (gmat_padding_kernel fills them once).
// One block of g (all threads of the CTA; Tm/Te: 32 x 33 shared tiles).
template <int MODE, bool PBC>
__device__ __forceinline__ void gmat_block(const Workspace &w, const double *__restrict__ pos, int blk,
                                           typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type *Tm,
                                           int *Te, EndTiles &E, const unsigned long long *T63) {
  using M_t = typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type;
  const double cx = w.cx;
  const int N = w.N;
  M_t *gm = (M_t *)w.gm, *gbm = (M_t *)w.gbm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int t, s;
  block_coords(blk, t, s);
  stage_endpoints<MODE != BPIMD_FP64>(w, pos, t, s, E);
  {
    const int b = t * TILE + lane;
    for (int i = warp; i < TILE; i += 8) {
      const int a = s * TILE + i;
      if (b < N && a <= b) {
        int e;
        const M_t m = (M_t)pair_factor<MODE, PBC>(w, cx, E, i, lane, e, T63);
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

// One evaluation's preparation: blocks 0..nbead-1 run the bead pass (8
// particles each), the others stride over the blocks of g.  MODE is the
// precision form (BPIMD_FP64, BPIMD_MIXED, BPIMD_MIXED32).
template <int MODE>
__global__ void __launch_bounds__(256) prep_kernel(Workspace w, const double *__restrict__ pos,
                                                   double *__restrict__ F, int nbead) {
  using M_t = typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type;
  __shared__ M_t Tm[TILE * 33];
  __shared__ int Te[TILE * 33];
  __shared__ EndTiles E;
  __shared__ unsigned long long T63[256];
  if (MODE != BPIMD_MIXED32) pairg::table_init(T63);  // published by gmat_block's first barrier
  pdl_wait();
  if ((int)blockIdx.x < nbead) {
    bead_pass_body<MODE != BPIMD_FP64>(w, pos, F, blockIdx.x * BEAD_WARPS);
  } else {
    for (int blk = blockIdx.x - nbead; blk < w.NB; blk += gridDim.x - nbead) {
      if (w.pbc) gmat_block<MODE, true>(w, pos, blk, Tm, Te, E, T63);
      else gmat_block<MODE, false>(w, pos, blk, Tm, Te, E, T63);
    }
  }
  pdl_trigger();
}

// Replica batch: bead_tab[k] = (replica, first particle), blk_tab[k] =
// (replica, block of g); positions and forces of replica r start at element
// off[r] of the packed arrays.
template <int MODE>
__global__ void __launch_bounds__(256) prep_batched(const Workspace *__restrict__ ws,
                                                    const int2 *__restrict__ bead_tab, int nbead,
                                                    const int2 *__restrict__ blk_tab, int nblk,
                                                    const long long *__restrict__ off,
                                                    const double *__restrict__ pos, double *__restrict__ F) {
  using M_t = typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type;
  __shared__ M_t Tm[TILE * 33];
  __shared__ int Te[TILE * 33];
  __shared__ EndTiles E;
  __shared__ unsigned long long T63[256];
  if (MODE != BPIMD_MIXED32) pairg::table_init(T63);  // published by gmat_block's first barrier
  pdl_wait();
  if ((int)blockIdx.x < nbead) {
    const int2 e = bead_tab[blockIdx.x];
    bead_pass_body<MODE != BPIMD_FP64>(ws[e.x], pos + off[e.x], F + off[e.x], e.y);
  } else {
    for (int k = blockIdx.x - nbead; k < nblk; k += gridDim.x - nbead) {
      const int2 e = blk_tab[k];
      if (ws[e.x].pbc) gmat_block<MODE, true>(ws[e.x], pos + off[e.x], e.y, Tm, Te, E, T63);
      else gmat_block<MODE, false>(ws[e.x], pos + off[e.x], e.y, Tm, Te, E, T63);
    }
  }
  pdl_trigger();
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

// Diagnostic potentials of the last evaluation (on demand), from the reduced
// prefix sums of Ap and the exponent parts n (see the bead pass):
//   V^{[1,v]} = C'[v] - (ln y_v - N_v ln 2)/beta,                 N_v = sum_{q<v} n_q
//   V^{[u,N]} = (C'[N] - C'[u-1]) - (ln(B_u/N) - (N_N - N_{u-1}) ln 2)/beta
// (0-based particle a = u-1).  One block: every thread sums a chunk of Ap in
// double-double, thread 0 scans the chunk sums, and each thread walks its
// chunk again, so that suffix sums C'[N] - C'[a] are as accurate as prefix sums.
__device__ __forceinline__ void dd_add(double &ah, double &al, double bh, double bl) {
  const double s = ah + bh, bb = s - ah;
  const double e = ((ah - (s - bb)) + (bh - bb)) + (al + bl);
  ah = s + e;
  al = e - (ah - s);
}

__device__ __forceinline__ double reduced_pot(double ch, double cl, xd y, long long n, double beta, double lnN) {
  const double k = (double)((long long)y.e - n);
  const double t = fma(k, LN2, fma(k, LN2_LO, log(y.m) - lnN));
  return (ch - t / beta) + cl;
}

constexpr int DIAG_THREADS = 1024;

__global__ void __launch_bounds__(DIAG_THREADS) diag_potentials_kernel(Workspace w, double *Vf, double *Vb) {
  __shared__ double sh[DIAG_THREADS], sl[DIAG_THREADS];
  __shared__ long long sn[DIAG_THREADS];
  __shared__ double tot[2];
  __shared__ long long ntot;
  const int N = w.N, tid = threadIdx.x;
  const int ch = (N + DIAG_THREADS - 1) / DIAG_THREADS;
  const int lo = min(N, tid * ch), hi = min(N, lo + ch);
  double a = 0.0, b = 0.0;
  long long n = 0;
  for (int i = lo; i < hi; ++i) {
    dd_add(a, b, w.Ap[i], 0.0);
    n += w.nexp[i];
  }
  sh[tid] = a;
  sl[tid] = b;
  sn[tid] = n;
  __syncthreads();
  if (tid == 0) {  // exclusive scan of the chunk sums
    double ca = 0.0, cb = 0.0;
    long long cn = 0;
    for (int k = 0; k < DIAG_THREADS; ++k) {
      const double ta = sh[k], tb = sl[k];
      const long long tn = sn[k];
      sh[k] = ca;
      sl[k] = cb;
      sn[k] = cn;
      dd_add(ca, cb, ta, tb);
      cn += tn;
    }
    tot[0] = ca;
    tot[1] = cb;
    ntot = cn;
  }
  __syncthreads();
  double pa = sh[tid], pb = sl[tid];
  long long pn = sn[tid];
  const double lnN = log((double)N);
  for (int v = lo; v < hi; ++v) {  // pa + pb = C'[v], pn = N_v
    Vf[v] = (v == 0) ? 0.0 : reduced_pot(pa, pb, xd{w.yfm[v], w.yfe[v]}, pn, w.beta, 0.0);
    double sa = tot[0], sb = tot[1];
    dd_add(sa, sb, -pa, -pb);  // C'[N] - C'[v]
    Vb[v] = reduced_pot(sa, sb, backward_row_sum(w, v), ntot - pn, w.beta, lnN);
    dd_add(pa, pb, w.Ap[v], 0.0);
    pn += w.nexp[v];
  }
  if (tid == 0) {
    Vf[N] = reduced_pot(tot[0], tot[1], xd{w.yfm[N], w.yfe[N]}, ntot, w.beta, 0.0);
    Vb[N] = 0.0;
  }
}

}  // namespace

cudaError_t launch_diag_potentials(const Workspace &w, double *Vf, double *Vb, cudaStream_t s) {
  diag_potentials_kernel<<<1, DIAG_THREADS, 0, s>>>(w, Vf, Vb);
  return cudaGetLastError();
}

cudaError_t launch_prep(const Workspace &w, const double *pos, double *F, cudaStream_t s) {
  const int nbead = (w.N + BEAD_WARPS - 1) / BEAD_WARPS;
  const int cap = sm_count() * 8;
  const int grid = nbead + (w.recomp ? 0 : (w.NB < cap ? w.NB : cap));  // recompute mode: bead pass only
  switch (w.mode) {
    case BPIMD_FP64: return launch_pdl(prep_kernel<BPIMD_FP64>, grid, 256, 0, s, w, pos, F, nbead);
    case BPIMD_MIXED: return launch_pdl(prep_kernel<BPIMD_MIXED>, grid, 256, 0, s, w, pos, F, nbead);
    default: return launch_pdl(prep_kernel<BPIMD_MIXED32>, grid, 256, 0, s, w, pos, F, nbead);
  }
}

cudaError_t launch_gmat_padding(const Workspace &w, cudaStream_t s) {
  const int sms = sm_count();
  const int grid = w.NB < sms * 8 ? w.NB : sms * 8;
  if (w.mixed) gmat_padding_kernel<true><<<grid, 256, 0, s>>>(w);
  else gmat_padding_kernel<false><<<grid, 256, 0, s>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_prep_batched(const Workspace *ws, const int2 *bead_tab, int nbead, const int2 *blk_tab,
                                int nblk, const long long *off, int mode, const double *pos, double *F,
                                int blocks_per_sm, cudaStream_t s) {
  if (nbead <= 0 && nblk <= 0) return cudaSuccess;
  const int cap = sm_count() * (blocks_per_sm > 0 ? blocks_per_sm : 8);
  const int grid = nbead + (nblk < cap ? nblk : cap);
  switch (mode) {
    case BPIMD_FP64:
      return launch_pdl(prep_batched<BPIMD_FP64>, grid, 256, 0, s, ws, bead_tab, nbead, blk_tab, nblk, off, pos, F);
    case BPIMD_MIXED:
      return launch_pdl(prep_batched<BPIMD_MIXED>, grid, 256, 0, s, ws, bead_tab, nbead, blk_tab, nblk, off, pos, F);
    default:
      return launch_pdl(prep_batched<BPIMD_MIXED32>, grid, 256, 0, s, ws, bead_tab, nbead, blk_tab, nblk, off, pos,
                        F);
  }
}

cudaError_t launch_gmat_padding_batched(const Workspace *ws, const int2 *tab, int ntab, bool mixed,
                                        cudaStream_t s) {
  if (ntab <= 0) return cudaSuccess;
  const int cap = sm_count() * 8;
  const int grid = ntab < cap ? ntab : cap;
  if (mixed) gmat_padding_batched<true><<<grid, 256, 0, s>>>(ws, tab, ntab);
  else gmat_padding_batched<false><<<grid, 256, 0, s>>>(ws, tab, ntab);
  return cudaGetLastError();
}

}  // namespace bpimd
