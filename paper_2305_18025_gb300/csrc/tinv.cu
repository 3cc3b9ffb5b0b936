// Tile inverses of the recursions' lower-triangular solves.
//
// Row tile t (rows r0 = 32t .. r0+31, outputs z_j = Y_{r0+j+1}) of either
// recursion (Eq. our-forward-potential-recurrence / Eq.
// backward-potential-recursion, linear-space form with K(w, r) = c_r H(w, r))
// solves
//     z_j = b_j + sum_{k<j} M[j][k] z_k,   M[j][k] = K(r0+k+1, r0+j),
//     b_j = c_j (sum over sources w < r0) + K(r0, r0+j) Y_{r0},
// i.e. z = T b with T = (I - M)^{-1}, unit lower triangular and nonnegative
// (every entry a sum of products of pair factors and coefficients: no
// cancellation).  T depends on the pair factors and the coefficients only, so
// all tiles' inverses are formed here, in parallel, before the recursions run;
// the recursion kernel then applies T to b instead of stepping through the 32
// dependent rows.  One warp per (recursion, tile): lane c owns column c and
// forms row j as sum_{k=c}^{j-1} M[j][k] T[k][c] in the integer-pipe chain
// format (xi_fma), as four interleaved partial sums.  Output: T[j][i] (row j, source i) at
// Tm/Te[((recursion * NT + t) * 32 + i) * 32 + j] as 64-bit mantissas.
#include "chain_common.cuh"

namespace bpimd {
namespace {

using namespace chain_detail;

struct TinvSmem {
  unsigned long long Mm[TILE][TILE + 1];  // M[j][k] (xk)
  unsigned long long Xm[TILE][TILE + 1];  // T[k][c] (xi)
  int Me[TILE][TILE + 1];
  int Xe[TILE][TILE + 1];
};

template <bool MIXED, bool BWD>
__device__ __forceinline__ void tile_inverse(const Workspace &w, int t, TinvSmem &S) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const int lane = threadIdx.x & 31;
  const int r0 = t * TILE, row = r0 + lane;
  const bool valid = row < w.N;
  const M_t *gm = (const M_t *)chain_gm<BWD>(w);
  const int *ge = chain_ge<BWD>(w);
  // M[j][k] = c_j H(r0+k+1, r0+j) for k+1 <= j (lane = j).  Branch-free: every
  // lane loads 8 entries at a time from in-bounds addresses (the diagonal
  // entry where k+1 > j) and keeps an extended zero outside the triangle.
  const xd c = valid ? xnorm_int(chain_coef<BWD>(w, row)) : xd{1.0, 0};
  const int rowc = valid ? row : r0;  // a row of this tile inside [0, N)
  for (int k0 = 0; k0 < TILE; k0 += 8) {
    M_t m[8];
    int e[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int src = r0 + min(k0 + u + 1, rowc - r0);
      const size_t gi = hidx(src, rowc);
      m[u] = __ldg(gm + gi);
      e[u] = __ldg(ge + gi);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool on = valid && k0 + u + 1 <= lane;
      const xk v = mul_mant<M_t>(c, m[u], on ? e[u] : XZERO_E);
      S.Mm[lane][k0 + u] = v.m;
      S.Me[lane][k0 + u] = on ? max(v.e, XZERO_E) : XZERO_E;
    }
  }
  __syncwarp();
  // column c = lane: T[c][c] = 1, T[j][c] = sum_{k=c}^{j-1} M[j][k] T[k][c],
  // as four interleaved partial sums over a warp-uniform loop; terms outside
  // c <= k < j enter as exact no-ops (an extended-zero factor times 1)
  const int cc = lane;
  S.Xm[cc][cc] = 1ull << 62;
  S.Xe[cc][cc] = 0;
  for (int j = 1; j < TILE; ++j) {
    xi acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = xi{1ull << 62, XZERO_E};
    for (int k0 = 0; k0 < j; k0 += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + u;
        const bool on = k < j && k >= cc;
        const int kc = min(k, TILE - 1);
        const unsigned long long mm = S.Mm[j][kc];
        const int me = S.Me[j][kc];
        const unsigned long long xm = S.Xm[kc][cc];
        const int xe = S.Xe[kc][cc];
        acc[u] = xi_fma<MIXED>(acc[u], mm, on ? me : XZERO_E, on ? xi{xm, xe} : xi{1ull << 62, 0});
      }
    }
    const xi sum = xi_add(xi_add(acc[0], acc[1]), xi_add(acc[2], acc[3]));
    if (j > cc) {
      S.Xm[j][cc] = sum.m;
      S.Xe[j][cc] = sum.e;
    }
  }
  __syncwarp();
  // T[j][i] as xk, written in (source i, row j) order, coalesced along j = lane
  const size_t base = ((size_t)(BWD ? w.NT : 0) + t) * TILE;
  for (int i = 0; i < TILE; ++i) {
    unsigned long long m = 1ull << 63;
    int e = XZERO_E;
    if (lane > i) {
      m = S.Xm[lane][i] << 1;
      e = max(S.Xe[lane][i], XZERO_E);
    } else if (lane == i) {
      e = 0;
    }
    w.Tm[(base + i) * TILE + lane] = m;
    w.Te[(base + i) * TILE + lane] = e;
  }
}

// block b < NT: forward tile b; NT <= b < 2 NT: backward tile b - NT
template <bool MIXED>
__global__ void __launch_bounds__(32) tinv_kernel(Workspace w) {
  __shared__ TinvSmem S;
  pdl_wait();
  const int b = blockIdx.x;
  if (b < w.NT) tile_inverse<MIXED, false>(w, b, S);
  else tile_inverse<MIXED, true>(w, b - w.NT, S);
  pdl_trigger();
}

}  // namespace

cudaError_t launch_tile_inverses(const Workspace &w, cudaStream_t s) {
  if (!w.tile_inv) return cudaSuccess;
  return w.mixed ? launch_pdl(tinv_kernel<true>, 2 * w.NT, 32, 0, s, w)
                 : launch_pdl(tinv_kernel<false>, 2 * w.NT, 32, 0, s, w);
}

}  // namespace bpimd
