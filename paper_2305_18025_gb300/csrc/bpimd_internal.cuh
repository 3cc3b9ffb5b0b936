// Internal definitions of the bpimd CUDA library (not part of the C ABI).
//
// Numerical formulation used on the device
// ----------------------------------------
// The paper evaluates the forward and backward potentials as log-sum-exp
// recursions (Eq. our-forward-potential-recurrence, Eq.
// backward-potential-recursion, shifted as in the Numerical Stability
// section).  On GB300 one FP64 exp costs ~1100 cycles of latency and one FP64
// log ~2000, so a log-sum-exp per sequential step would dominate.  The device
// therefore runs the SAME recursions in linear space, with every quantity
// carried as an extended-range number  x = m * 2^e  (m a float/double
// mantissa, e a 32-bit integer exponent) -- a power-of-two shift per value in
// place of the paper's energy shift E~ (any shift is valid, Numerical
// Stability section).  With the prefix sums
//     C[l]  = sum_{i<=l} (E_int^{(i)} + link_i),  link_i = (1/2)k (r_i^P - r_{i+1}^1)^2,
// the cycle energy factorises (telescoping Eq. e-recurrence-step):
//     E^{[u,v]} = C[v-1] - C[u-1] + E_int^{(v)} + (1/2)k (r_v^P - r_u^1)^2,
// so that, with g(u,v) = exp(-beta (1/2)k (r_v^P - r_u^1)^2) and
// c_v = exp(beta link_v)/v,
//     forward : y_0 = 1,  y_{r+1} = c_{r+1} sum_{w<=r} y_w g(w+1, r+1)
//               (0-based rows r; y_v = exp(-beta (V^{[1,v]} - C[v])))
//     backward: mu_{N} = 1, B_u = sum_{l>=u} g(u,l) mu_l, mu_{u-1} = c_{u-1} B_u
//               (exp(-beta V^{[u,N]}) = exp(beta (C[u-1]-C[N])) B_u / N)
//     Pr[l -> u<=l] = y_{u-1} g(u,l) mu_l / (N y_N)          (Eq. close-cycle)
//     Pr[l -> l+1]  = 1 - y_l B_{l+1} / (N y_N)              (Eq. direct-link)
// Each sequential step is then one multiply-add; no transcendental function
// sits on the dependency chain.  g is computed once per evaluation and shared
// by both recursions and the probability pass.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bpimd.h"

namespace bpimd {

constexpr int TILE = 32;              // row / source tile of the recursions and of g
constexpr int TILE2 = TILE * TILE;
constexpr int XZERO_E = -(1 << 29);   // exponent carried by an extended zero
constexpr int CHAIN_THREADS = 640;     // 20 warps: up to 96 registers per thread
constexpr int CHAIN_CLUSTER = 8;      // CTAs per recursion (small N): one lead + seven bulk CTAs
constexpr int CHAIN_MAX_N = BPIMD_MAX_N;  // largest N the library accepts
constexpr int BATCH_MAX_N = 4096;     // largest replica of a batch (one CTA per recursion)
constexpr int BEAD_BLOCK_PARTICLES = 8;  // particles per block of the bead pass
constexpr double LOG2E = 1.4426950408889634074;
constexpr double LOG2E_LO = 2.0355273740931033e-17;  // log2(e) - LOG2E (double-double tail)
constexpr double LN2 = 0.6931471805599453094;
constexpr double LN2_LO = 2.3190468138462996e-17;    // ln(2) - LN2

// status bits recorded on the device
constexpr int ST_NONFINITE = 1;
constexpr int ST_TIMEOUT = 2;

// ------------------------------------------------------------ extended numbers
struct xd {  // value = m * 2^e
  double m;
  int e;
};

__device__ __forceinline__ double pow2_nonpos(int k) {
  // 2^k for k <= 0; 0 below the normal range (the scaled operand is then
  // below 2^-1022 of the larger one and cannot change a double sum).
  return (k < -1022) ? 0.0 : __longlong_as_double((long long)(k + 1023) << 52);
}
__device__ __forceinline__ float pow2f_nonpos(int k) {
  return (k < -126) ? 0.0f : __int_as_float((k + 127) << 23);
}

// Bring m into [1,2), folding its binary exponent into e.  m >= 0, finite.
__device__ __forceinline__ xd xnorm(double m, int e) {
  if (!(m > 0.0)) return xd{0.0, XZERO_E};
  long long b = __double_as_longlong(m);
  int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) {  // subnormal mantissa: rescale exactly
    m *= 18446744073709551616.0;  // 2^64
    e -= 64;
    b = __double_as_longlong(m);
    ex = (int)((b >> 52) & 0x7ff);
  }
  b = (b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL;
  return xd{__longlong_as_double(b), e + ex - 1023};
}

__device__ __forceinline__ xd xmul(xd a, xd b) { return xnorm(a.m * b.m, a.e + b.e); }

// Convert an extended number to a double (0 below the normal range).
__device__ __forceinline__ double xtod(xd a) {
  if (a.m == 0.0 || a.e < -1100) return 0.0;
  if (a.e > 1023) return __longlong_as_double(0x7ff0000000000000LL);
  // split to stay within the range of pow2 for exponents near the limits
  int e1 = a.e / 2, e2 = a.e - e1;
  double s1 = __longlong_as_double((long long)(e1 + 1023) << 52);
  double s2 = __longlong_as_double((long long)(e2 + 1023) << 52);
  return a.m * s1 * s2;
}
// natural log of an extended number (m > 0)
__device__ __forceinline__ double xlog(xd a) { return log(a.m) + (double)a.e * LN2; }

// ------------------------------------------- programmatic dependent launches
// The three kernels of an evaluation are launched with programmatic stream
// serialisation: a kernel may be scheduled while its predecessor in the
// stream drains (hiding the launch gap), waits (griddepcontrol.wait: the
// predecessor has completed and its writes are visible) before its first
// global-memory access, and lets its own successor launch once its work is
// issued (griddepcontrol.launch_dependents).  A successor launches only after
// every CTA of its predecessor has started, so an early launch never takes
// resources the predecessor still needs.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------------ workspace
struct Workspace {
  int N, P, NT, NB;     // NT = ceil(N/TILE), NB = NT(NT+1)/2 blocks of g
  int mode;             // precision form: BPIMD_FP64, BPIMD_MIXED or BPIMD_MIXED32
  int mixed;            // MIXED32: float32 pair-factor and alpha mantissas, 32-bit recursion chain
  int bead32;           // MIXED and MIXED32: float32 bead differences and spring energies
  double m, omega_P, beta, k, half_k;
  double inv_P;         // 1/P (kernels take it from here: a float64 division costs a GB300 SM ~20 warp-cycles per lane)
  double cx;            // beta (1/2) k log2(e): g = 2^(-cx d^2)
  int recomp;           // recompute mode: no O(N^2) table; g is formed where it is used
  int test_timeout;     // BPIMD_FLAG_TEST_TIMEOUT: the forward lead waits for a hand-off never made
  // periodic cubic box of side L (0: open boundaries); every spring joins the
  // minimum image of its beads.  MIXED keeps the bead-1/bead-P copies in a box
  // as 32-bit fixed-point fractions of L (R1s/RPs reinterpreted as uint32
  // x, y, z, 0), whose wrap-around integer difference is the minimum image.
  double L, invL, invL32;  // invL32 = 2^32 / L
  float Lscale;  // L / 2^32
  int pbc;       // L > 0 (an integer test: a float64 compare would use the slow float64 pipe)
  // O(N) per-particle state
  double *R1, *RP;      // [N][4] bead 1 / bead P positions (x, y, z, 0)
  float *R1s, *RPs;     // MIXED: [N][8] the same positions split into float
                        // high and low parts (hx, hy, hz, 0, lx, ly, lz, 0), so that
                        // a bead difference is formed in float32 to float32 accuracy
  double *Eint, *link;  // [N]
  double *ccm; int *cce;          // c_{i+1} = exp(beta link_i)/(i+1), extended
  int *nexp;            // [N] n_i = integer part of beta link_i log2(e) (in c_{i+1}'s exponent)
  double *Ap;           // [N] E_int_i + (beta link_i log2(e) - n_i) ln2 / beta
  double *C;            // [N+1] reduced prefix sums C'[v] = sum_{i<v} Ap[i] (0-based i)
  // g matrix, tile-packed triangle: block (t, s), s <= t, at (t(t+1)/2 + s) * TILE2,
  // entry [i][j] = g for a = s*TILE + i (bead 1 particle), b = t*TILE + j (bead P particle)
  void *gm;             // double (FP64) or float (MIXED) mantissas
  int *ge;              // exponents
  // the same factors in the backward recursion's coordinates (rows r = N-1-a,
  // sources w = N-1-b), same tile-packed layout, so that both recursions read
  // their blocks with coalesced loads
  void *gbm;
  int *gbe;
  // recursion outputs (extended): forward y[0..N]; backward Yb[0..N]
  // (Yb[w] = mu_{N-1-w} 0-based; the backward row sums are B_{a+1} = Yb[N-a] / c_{a}, 1-based c)
  double *yfm; int *yfe;
  double *ybm; int *ybe;
  // alpha_a = y_a / (N y_N), a = 0..N-1, extended (float mantissa for MIXED),
  // written by the forward recursion once y_N is known
  void *alm; int *ale;
  // scalars: [0] V_B, [1] invZ mantissa, [2] reserved ; int [0] invZ exponent
  double *scal; int *scal_i;
  // force partial sums: rowpart/colpart [NB][TILE][4]
  double *rowpart, *colpart;
  // per row / column tile: number of finished blocks of the probability pass
  // (the last block of a tile forms its forces and resets the count to 0)
  int *rowcnt, *colcnt;
  int *status;          // device status word
  // blocked recursions (cluster kernel): per recursion and row tile, the
  // c-scaled coupling block Dc to the previous tile's unknowns and the tile
  // inverse M = (I - L)^{-1}, as 64-bit integer mantissas in [2^63, 2^64) and
  // exponents, [recursion][tile][Dc, M][row][source]
  int blocks;           // 1: bk/be present (single systems; batch replicas above BATCH_MAX_N)
  unsigned long long *bk;
  int *be;
};

// Precision form of a workspace (the three BPIMD_* precision values).
inline bool valid_precision(int p) { return p == BPIMD_FP64 || p == BPIMD_MIXED || p == BPIMD_MIXED32; }
inline void set_precision(Workspace &w, int p) {
  w.mode = p;
  w.mixed = p == BPIMD_MIXED32;
  w.bead32 = p != BPIMD_FP64;
}

// number of SMs of the current device (cached per device)
inline int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 152;
  }
  return cached[dev];
}

// Minimum image of one coordinate difference (identity for open boundaries).
__device__ __forceinline__ double mimage(const Workspace &w, double d) {
  return w.pbc ? d - w.L * rint(d * w.invL) : d;
}
// Difference a - b of two fixed-point coordinates (fractions of L in units of
// 2^-32): the signed 32-bit wrap-around difference is the minimum image.
__device__ __forceinline__ float fixdiff(unsigned a, unsigned b, float Lscale) {
  return (float)(int)(a - b) * Lscale;
}

// Endpoint copies of the MIXED path, formed the same way wherever a kernel
// needs them, with integer and float32 instructions only (the float64 pipe is
// the scarce one):
//  * a coordinate split into float32 high and low parts, x = hi + lo to
//    2^-46 relative: hi is x with its significand cut to 24 bits, lo the next
//    23 bits of the significand (both exact);
//  * in a box, its fraction of L as a 32-bit fixed-point number,
//    floor(x 2^32 / L) mod 2^32 (invL32 = 2^32 / L).
__device__ __forceinline__ void split_hi_lo(double x, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  if (E >= 943 && E <= 1150) {  // |x| in [2^-80, 2^128): both parts normal floats
    hi = __uint_as_float(sgn | ((unsigned)(E - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    // bits 28..6 of the significand as an integer t < 2^23, times 2^(E - 1069)
    const float t = __uint_as_float(0x4b000000u | (unsigned)((b >> 6) & 0x7fffffu)) - 8388608.0f;
    lo = __uint_as_float(__float_as_uint(t * __uint_as_float((unsigned)(E - 942) << 23)) | sgn);
  } else if (E == 0) {  // zero (and float64 subnormals, far below float32)
    hi = __uint_as_float(sgn);
    lo = hi;
  } else {  // tiny, huge or non-finite: rounded parts
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
}
__device__ __forceinline__ unsigned to_fixed(double x, double invL32) {
  return (unsigned)(unsigned long long)__double2ll_rd(x * invL32);
}

// Periodic box of side L (L <= 0: open boundaries).
inline void set_box(Workspace &w, double L) {
  w.L = L > 0.0 ? L : 0.0;
  w.invL = L > 0.0 ? 1.0 / L : 0.0;
  w.invL32 = w.invL * 4294967296.0;
  w.Lscale = (float)(w.L / 4294967296.0);
  w.pbc = L > 0.0 ? 1 : 0;
}

// Lay the workspace out from `base` (nullptr: only measure); returns the bytes
// used.  Every array starts on a 256-byte boundary.
size_t layout_workspace(Workspace &w, char *base);

// kernel launchers (stream-ordered)
// bead pass and pair factors in one launch (the pair-factor blocks read the
// endpoint beads from the positions themselves, so the two run side by side)
cudaError_t launch_prep(const Workspace &w, const double *pos, double *F, cudaStream_t s);
// fill the pair-factor entries outside a <= b < N (fixed for a given N) with
// extended zeros; needed once per workspace before the first launch_prep
cudaError_t launch_gmat_padding(const Workspace &w, cudaStream_t s);
// both recursions, prefix sums, V_B (device scalar, may be null), normaliser, alpha
cudaError_t launch_chains(const Workspace &w, double *V_B, cudaStream_t s);
// once per process and device, before any stream capture: kernel attributes
// and the cluster-size choice of the recursions
cudaError_t prepare_chains();
// connection probabilities and all exterior-bead forces
cudaError_t launch_prob_forces(const Workspace &w, const double *pos, double *F, cudaStream_t s);
cudaError_t launch_dense_probabilities(const Workspace &w, double *M, cudaStream_t s);
// per block of g: (1/2) m w_P^2 sum Pr[b -> a] |r_b^P - r_a^1|^2 over a <= b (part[NB])
cudaError_t launch_spring_expectation(const Workspace &w, double *part, cudaStream_t s);
// the same per (replica, block) entry of a batch's block table
cudaError_t launch_spring_expectation_batched(const Workspace *ws, const int2 *tab, int ntab, double *part,
                                             cudaStream_t s);
cudaError_t launch_diag_potentials(const Workspace &w, double *Vf, double *Vb, cudaStream_t s);

// Replica batches: ws[r] is replica r's workspace (device array); block tables
// hold (replica, particle block) for the bead pass and (replica, g block) for
// the pair factors and the probability pass; off[r] is the element offset of
// replica r in the packed position/force arrays; order lists replicas by
// decreasing N.
// bead pass (bead_tab: (replica, first particle)) and pair factors (blk_tab:
// (replica, block of g), at most blocks_per_sm * SMs blocks) in one launch
cudaError_t launch_prep_batched(const Workspace *ws, const int2 *bead_tab, int nbead, const int2 *blk_tab,
                                int nblk, const long long *off, int mode, const double *pos, double *F,
                                int blocks_per_sm, cudaStream_t s);
cudaError_t launch_gmat_padding_batched(const Workspace *ws, const int2 *tab, int ntab, bool mixed,
                                        cudaStream_t s);
cudaError_t launch_chains_batched(const Workspace *ws, const int *order, int R, int maxN, bool mixed, double *V_B,
                                  cudaStream_t s);
cudaError_t launch_prob_forces_batched(const Workspace *ws, const int2 *tab, int ntab, const long long *off,
                                      int mode, const double *pos, double *F, int blocks_per_sm, cudaStream_t s);

// B_{a+1} (1-based backward row sum for 0-based particle a) from the stored state
__device__ __forceinline__ xd backward_row_sum(const Workspace &w, int a) {
  const xd Y{w.ybm[w.N - a], w.ybe[w.N - a]};
  if (a == 0) return Y;  // B_1 = Y_N
  // mu_a = c_a B_{a+1}: divide the mantissas, subtract the exponents
  return xnorm(Y.m / w.ccm[a - 1], Y.e - w.cce[a - 1]);
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

}  // namespace bpimd
