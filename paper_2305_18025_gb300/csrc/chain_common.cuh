// Device helpers of the recursion kernels (chain.cu: one cluster per
// recursion; chain_batched.cu: one CTA per recursion of a replica batch).
// Internal; included by those two files only.
#pragma once
#include <type_traits>

#include "bpimd_internal.cuh"
#include "pairg.cuh"

namespace bpimd {
namespace chain_detail {

constexpr int BLK = 32 * 33;  // padded 32 x 32 block in shared memory

// index of H(src, row) in the tile-packed pair-factor layout
__device__ __forceinline__ size_t hidx(int src, int row) {
  const int t = row >> 5, s = src >> 5;
  return ((size_t)(t * (t + 1) / 2 + s) << 10) + ((src & 31) << 5) + (row & 31);
}

// x * 2^k for k <= 0 by integer arithmetic on the exponent field (x >= 0 normal
// or zero); 0 when the result would leave the normal range.
__device__ __forceinline__ double scale_nonpos(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)(b >> 52);  // sign bit is 0
  return (ex + k <= 0) ? 0.0 : __longlong_as_double(b + ((long long)k << 52));
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
__device__ __forceinline__ unsigned long long lds_u64(unsigned a) {
  unsigned long long v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_f32(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
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

// Round the significand of a positive normal double to a float in [1,2] with
// integer ops (no float64 conversion unit); the binary exponent is dropped.
__device__ __forceinline__ float mant_to_float(double m) {
  const long long b = __double_as_longlong(m);
  const long long frac = b & 0x000fffffffffffffLL;
  return __int_as_float((int)((frac + (1LL << 28)) >> 29) + 0x3f800000);
}

// Mantissa in [1,2) as a 53-bit integer (implicit bit set), from a double or a float.
__device__ __forceinline__ unsigned long long mant53(double m) {
  return ((unsigned long long)__double_as_longlong(m) & 0xFFFFFFFFFFFFFull) | (1ull << 52);
}
__device__ __forceinline__ unsigned long long mant53(float m) {
  return ((unsigned long long)((unsigned)__float_as_int(m) & 0x7FFFFFu) | 0x800000ull) << 29;
}

// c * h for extended numbers with mantissas in [1,2): the 53 x 53-bit mantissa
// product on the integer pipe, kept as a 64-bit integer mantissa kk in
// [2^63, 2^64) (value kk 2^(e-63); the 106-bit product truncated to 64 bits),
// so that staging issues no float64 instruction.
struct xk {
  unsigned long long m;
  int e;
};
template <typename M_t>
__device__ __forceinline__ xk mul_mant(xd c, M_t hm, int he) {
  const unsigned long long hi = __umul64hi(mant53(c.m) << 11, mant53(hm) << 11);  // in [2^62, 2^64)
  const int sh = (int)(hi >> 63);
  return xk{hi << (1 - sh), c.e + he + sh};
}

// ------------------------------------------------- the integer-pipe chain format
// The dependency chain of the recursions runs on the integer pipe: a float64
// FMA has a 64-cycle latency on GB300 (plus ~40 cycles before a shuffle can
// read its result), while a 64 x 64-bit integer product, shifts and a 64-bit
// add take a few cycles each.  An extended number is  m * 2^(e - 62)  with an
// integer mantissa m in [2^62, 2^63) (one bit of headroom for an addition);
// the extended zero is 2^62 * 2^(XZERO_E - 62).  Products and alignment shifts
// truncate, at 2^-61 relative: finer than a float64 rounding.
struct xi {
  unsigned long long m;
  int e;
};

// From an extended number with a positive normal double mantissa (any binary
// exponent); zero or negative mantissas give the extended zero.
__device__ __forceinline__ xi xi_from(xd a) {
  const long long b = __double_as_longlong(a.m);
  if (b <= 0) return xi{1ull << 62, XZERO_E};
  return xi{(((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10, a.e + (int)(b >> 52) - 1023};
}
// To an extended number with a double mantissa in [1,2) (truncated to 53 bits).
__device__ __forceinline__ xd xi_to_xd(xi a) {
  return xd{__longlong_as_double((long long)(((a.m >> 10) & 0xFFFFFFFFFFFFFull) | 0x3FF0000000000000ull)), a.e};
}
// s * 2^(E - 62) with s in [2^61, 2^64), brought back to [2^62, 2^63) by
// selecting among s/2, s and 2s on its top three bits (no bit scan).
__device__ __forceinline__ xi xi_norm(unsigned long long s, int E) {
  const unsigned top = (unsigned)(s >> 61);  // 1: [2^61, 2^62), 2-3: in range, 4-7: [2^63, 2^64)
  return xi{top >= 4 ? (s >> 1) : (top >= 2 ? s : (s << 1)), top >= 4 ? E + 1 : (top >= 2 ? E : E - 1)};
}
// a + b
__device__ __forceinline__ xi xi_add(xi a, xi b) {
  const int E = max(a.e, b.e);
  return xi_norm((a.m >> min(E - a.e, 63)) + (b.m >> min(E - b.e, 63)), E);
}
// a * c (c: positive normal double mantissa, any binary exponent)
__device__ __forceinline__ xi xi_mul(xi a, xd c) {
  const long long b = __double_as_longlong(c.m);
  const unsigned long long p = __umul64hi(mant53(c.m) << 11, a.m);  // in [2^61, 2^63)
  return xi_norm(p, a.e + c.e + (int)(b >> 52) - 1023 + 1);
}
// acc + K * y with K = kk 2^(ke - 63), kk in [2^63, 2^64): the step of the
// dependency chain.  The product kk * y.m / 2^64 lies in [2^61, 2^63), the
// aligned sum in [2^61, 2^64); a K carrying an extended-zero exponent leaves
// acc unchanged.  MIXED uses the top 32 bits of kk only (two 32 x 32-bit
// products, relative error below 2^-30: K = c g carries a float32 g there).
template <bool MIXED>
__device__ __forceinline__ xi xi_fma(xi acc, unsigned long long kk, int ke, xi y) {
  unsigned long long p;
  if (MIXED) {
    const unsigned k1 = (unsigned)(kk >> 32);
    p = (unsigned long long)k1 * (unsigned)(y.m >> 32) + (((unsigned long long)k1 * (unsigned)y.m) >> 32);
  } else {
    p = __umul64hi(kk, y.m);
  }
  const int pe = ke + y.e + 1;
  const int E = max(acc.e, pe);
  return xi_norm((acc.m >> min(E - acc.e, 63)) + (p >> min(E - pe, 63)), E);
}

// ----------------------------------------- the 32-bit chain format (MIXED)
// MIXED runs the dependency chain on 32-bit words: m * 2^(e - 30) with m in
// [2^30, 2^31) (one bit of headroom), the factor K by the top 32 bits of its
// mantissa.  A step is one 32 x 32-bit high product, two shifts, one add and a
// select (truncation at 2^-30 per operation, far below the float32 rounding
// of the pair factors the mixed form starts from), and its shuffle moves two
// words instead of three.
struct xs {
  unsigned m;
  int e;
};
__device__ __forceinline__ xs xs_from(xd a) {
  const long long b = __double_as_longlong(a.m);
  if (b <= 0) return xs{1u << 30, XZERO_E};
  return xs{(unsigned)((((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> 22), a.e + (int)(b >> 52) - 1023};
}
__device__ __forceinline__ xd xs_to_xd(xs a) {
  return xd{__longlong_as_double((long long)((((unsigned long long)a.m << 22) & 0xFFFFFFFFFFFFFull) |
                                             0x3FF0000000000000ull)),
            a.e};
}
// s * 2^(E - 30) with s in [2^29, 2^32), brought back to [2^30, 2^31)
__device__ __forceinline__ xs xs_norm(unsigned s, int E) {
  const unsigned top = s >> 29;  // 1: [2^29, 2^30), 2-3: in range, 4-7: [2^31, 2^32)
  return xs{top >= 4 ? (s >> 1) : (top >= 2 ? s : (s << 1)), top >= 4 ? E + 1 : (top >= 2 ? E : E - 1)};
}
__device__ __forceinline__ xs xs_add(xs a, xs b) {
  const int E = max(a.e, b.e);
  return xs_norm((a.m >> min(E - a.e, 31)) + (b.m >> min(E - b.e, 31)), E);
}
// a * c (c: positive normal double mantissa, any binary exponent)
__device__ __forceinline__ xs xs_mul(xs a, xd c) {
  const long long b = __double_as_longlong(c.m);
  const unsigned c32 = (unsigned)((((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> 21);  // [2^31, 2^32)
  return xs_norm(__umulhi(c32, a.m), a.e + c.e + (int)(b >> 52) - 1023 + 1);
}
// acc + K * y with K = kk 2^(ke - 63) (top 32 bits used): the chain step
__device__ __forceinline__ xs xs_fma(xs acc, unsigned long long kk, int ke, xs y) {
  const unsigned p = __umulhi((unsigned)(kk >> 32), y.m);  // in [2^29, 2^31)
  const int pe = ke + y.e + 1;
  const int E = max(acc.e, pe);
  return xs_norm((acc.m >> min(E - acc.e, 31)) + (p >> min(E - pe, 31)), E);
}

// alpha = y * inv for extended numbers with double mantissas in [1,2), with
// integer operations; the mantissa is written as float (MIXED) or double.
template <bool MIXED>
__device__ __forceinline__ void store_alpha(const Workspace &w, int a, xd y, xd inv) {
  const unsigned long long hi = __umul64hi(mant53(y.m) << 11, mant53(inv.m) << 11);  // in [2^62, 2^64)
  const int sh = (int)(hi >> 63);
  if (MIXED)
    ((float *)w.alm)[a] = __int_as_float((int)((hi >> (39 + sh)) & 0x7FFFFFu) | 0x3F800000);
  else
    ((double *)w.alm)[a] =
        __longlong_as_double((long long)(((hi >> (10 + sh)) & 0xFFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
  w.ale[a] = y.e + inv.e + sh;
}

// A positive normal float (or 0) as a double, with integer operations.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned b = (unsigned)__float_as_int(f);
  if (b < 0x00800000u) return 0.0;
  return __longlong_as_double(((long long)((b >> 23) + 896) << 52) | ((long long)(b & 0x7FFFFFu) << 29));
}

// a + b for extended numbers with positive normal (or zero) mantissas: the
// smaller operand is aligned by integer arithmetic, then one float64 add.
__device__ __forceinline__ xd xadd_int(xd a, xd b) {
  const int E = max(a.e, b.e);
  return xd{scale_nonpos(a.m, max(a.e - E, -1100)) + scale_nonpos(b.m, max(b.e - E, -1100)), E};
}

// Online-max merge of a float partial sum (s * 2^E) with a term x * 2^e.
__device__ __forceinline__ void fmerge(float &s, int &E, float x, int e) {
  const int En = max(E, e);
  s = fmaf(x, pow2f_nonpos(e - En), s * pow2f_nonpos(E - En));
  E = En;
}

}  // namespace chain_detail
}  // namespace bpimd

namespace bpimd {
namespace chain_detail {

// Row coefficient of a recursion in its own row coordinates: forward c_{r+1},
// backward c_{N-1-r} (1 for the last row, whose sum is B_1 itself).
template <bool BWD>
__device__ __forceinline__ xd chain_coef(const Workspace &w, int row) {
  if (!BWD) return xd{__ldg(w.ccm + row), __ldg(w.cce + row)};
  if (row >= w.N - 1) return xd{1.0, 0};
  return xd{__ldg(w.ccm + w.N - 2 - row), __ldg(w.cce + w.N - 2 - row)};
}

// The pair factors H(src, row) of a recursion, in its own coordinates.
template <bool BWD>
__device__ __forceinline__ const void *chain_gm(const Workspace &w) { return BWD ? w.gbm : w.gm; }
template <bool BWD>
__device__ __forceinline__ const int *chain_ge(const Workspace &w) { return BWD ? w.gbe : w.ge; }

// Staging issues no float64 instruction (the SM's float64 pipe belongs to the
// dependency chain).  Pairs outside src <= row < N hold the extended zero
// 1 * 2^XZERO_E; loads are coalesced along rows and issued before use.
// Off-diagonal block: H(tt*32+i, (tt+1)*32+lane), rows i in [i0, i0+NR), as
// stored (float for MIXED), into dm/de[i*33 + lane].
template <bool MIXED, bool BWD, int NR>
__device__ __forceinline__ void stage_offdiag(const Workspace &w, int tt, int i0, void *dmv, int *de) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const int lane = threadIdx.x & 31;
  const int srcbase = tt * TILE, row = tt * TILE + TILE + lane;
  const M_t *gm = (const M_t *)chain_gm<BWD>(w);
  const int *ge = chain_ge<BWD>(w);
  M_t *dm = (M_t *)dmv;
#pragma unroll
  for (int i = i0; i < i0 + NR; ++i) {
    M_t m = (M_t)1.0;
    int e = XZERO_E;
    if (row < w.N) {
      const size_t gi = hidx(srcbase + i, row);
      m = __ldg(gm + gi);
      e = __ldg(ge + gi);
    }
    dm[i * 33 + lane] = m;
    de[i * 33 + lane] = e;
  }
}

// Diagonal block of tile tt, K = c_row * H as 64-bit integer mantissas (the
// chain format of xi_fma), rows i in [i0, i0+NR): the mantissa product is
// formed on the integer pipe (mul_mant).
template <bool MIXED, bool BWD, int NR>
__device__ __forceinline__ void stage_diag(const Workspace &w, int tt, int i0, unsigned long long *dm, int *de) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const int lane = threadIdx.x & 31;
  const int r0 = tt * TILE, row = r0 + lane;
  const M_t *gm = (const M_t *)chain_gm<BWD>(w);
  const int *ge = chain_ge<BWD>(w);
  const xd c = (row < w.N) ? xnorm_int(chain_coef<BWD>(w, row)) : xd{1.0, 0};
#pragma unroll
  for (int i = i0; i < i0 + NR; ++i) {
    const int src = r0 + i;
    M_t m = (M_t)1.0;
    int e = XZERO_E;
    if (row < w.N && src <= row) {
      const size_t gi = hidx(src, row);
      m = __ldg(gm + gi);
      e = __ldg(ge + gi);
    }
    const xk k = mul_mant<M_t>(c, m, e);
    dm[i * 33 + lane] = k.m;
    de[i * 33 + lane] = k.e;
  }
}

// ------------------------------------------ recompute mode (no stored g)
// H(src, row) of a recursion from the bead pass's endpoint copies: forward
// H(w, r) = g(a = w, b = r); backward H(w, r) = g(a = N-1-r, b = N-1-w), b the
// bead-P end and a the bead-1 end of the closing spring (the same bits as the
// tabulated factors, pairg.cuh).  The row's endpoint is loaded once per lane.
template <int MODE, bool BWD, bool PBC>
struct RowEnds {
  pairg::EndPt<MODE != BPIMD_FP64, PBC> row;
  __device__ __forceinline__ void load(const Workspace &w, int r) {
    row = pairg::load_end<MODE != BPIMD_FP64, PBC>(w, BWD ? w.N - 1 - r : r, !BWD);
  }
  __device__ __forceinline__ typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type
  h(const Workspace &w, int src, const unsigned long long *T63, int &e) const {
    const auto s = pairg::load_end<MODE != BPIMD_FP64, PBC>(w, BWD ? w.N - 1 - src : src, BWD);
    return BWD ? pairg::g_of<MODE, PBC>(w, s, row, w.cx, T63, e) : pairg::g_of<MODE, PBC>(w, row, s, w.cx, T63, e);
  }
};

// stage_offdiag / stage_diag with H recomputed (same layouts and zeros).
template <int MODE, bool BWD, bool PBC, int NR>
__device__ __forceinline__ void stage_offdiag_rc(const Workspace &w, int tt, int i0, void *dmv, int *de,
                                                 const unsigned long long *T63) {
  using M_t = typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type;
  const int lane = threadIdx.x & 31;
  const int srcbase = tt * TILE, row = tt * TILE + TILE + lane;
  M_t *dm = (M_t *)dmv;
  RowEnds<MODE, BWD, PBC> re;
  if (row < w.N) re.load(w, row);
#pragma unroll 2
  for (int i = i0; i < i0 + NR; ++i) {
    M_t m = (M_t)1.0;
    int e = XZERO_E;
    if (row < w.N) m = re.h(w, srcbase + i, T63, e);
    dm[i * 33 + lane] = m;
    de[i * 33 + lane] = e;
  }
}
template <int MODE, bool BWD, bool PBC, int NR>
__device__ __forceinline__ void stage_diag_rc(const Workspace &w, int tt, int i0, unsigned long long *dm, int *de,
                                              const unsigned long long *T63) {
  using M_t = typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type;
  const int lane = threadIdx.x & 31;
  const int r0 = tt * TILE, row = r0 + lane;
  const xd c = (row < w.N) ? xnorm_int(chain_coef<BWD>(w, row)) : xd{1.0, 0};
  RowEnds<MODE, BWD, PBC> re;
  if (row < w.N) re.load(w, row);
#pragma unroll 2
  for (int i = i0; i < i0 + NR; ++i) {
    const int src = r0 + i;
    M_t m = (M_t)1.0;
    int e = XZERO_E;
    if (row < w.N && src <= row) m = re.h(w, src, T63, e);
    const xk k = mul_mant<M_t>(c, m, e);
    dm[i * 33 + lane] = k.m;
    de[i * 33 + lane] = k.e;
  }
}

// The 32 dependent steps of row tile t, run by one warp.  A is this lane's
// row sum over sources < 32t except tile t-1 (which is in nxt), crow the row's
// coefficient.  K (diagonal, c-scaled, integer mantissas) and H (to tile t+1)
// are the staged blocks.  Y_v lives at Ym/Ye[v & ymask] in shared memory and,
// unless gYm is null, at gYm/gYe[v] in global memory.  On return nxt holds
// the partial sums of tile t+1's rows over source tile t.
// 32 steps, no branches and no stores: rows past N and finished rows see
// extended zeros in the staged blocks, and row j's accumulator is final after
// step j.  The chain (acc, y) is in an integer format (xs for MIXED, xi for
// FP64); block entries of step i+1 are loaded (explicit ld.shared) before
// step i's shuffle.
template <bool MIXED>
__device__ __forceinline__ void chain_tile(int N, int t, xd A, xd crow, xd &nxt, const unsigned long long *Kdm,
                                           const int *Kde, const double *Hom, const int *Hoe, double *Ym, int *Ye,
                                           int ymask, double *gYm, int *gYe) {
  // the chain format: 32-bit words (MIXED, xs) or 64-bit mantissas (FP64, xi)
  using X = typename std::conditional<MIXED, xs, xi>::type;
  const int lane = threadIdx.x & 31;
  const int r0 = t * TILE, row = r0 + lane;
  const xd y0{Ym[r0 & ymask], Ye[r0 & ymask]};
  X acc, y;
  if constexpr (MIXED) {
    acc = xs{1u << 30, XZERO_E};
    if (row < N) acc = xs_mul(xs_add(xs_from(A), xs_from(nxt)), crow);  // c_row * (sum over sources < r0)
    y = xs_from(y0);
  } else {
    acc = xi{1ull << 62, XZERO_E};
    if (row < N) acc = xi_mul(xi_add(xi_from(A), xi_from(nxt)), crow);
    y = xi_from(y0);
  }
  nxt = xd{1.0, XZERO_E};
  float nsum = 0.0f;  // MIXED: the next tile's partial sum in float32
  int nexp = XZERO_E;
  const unsigned aKm = smem_addr(Kdm + lane), aKe = smem_addr(Kde + lane), aHe = smem_addr(Hoe + lane);
  const unsigned aHm = MIXED ? smem_addr((const float *)Hom + lane) : smem_addr(Hom + lane);
  unsigned long long km = lds_u64(aKm);
  double hm = MIXED ? 0.0 : lds_f64(aHm);
  float hf = MIXED ? lds_f32(aHm) : 0.0f;
  int ke = lds_s32(aKe), he = lds_s32(aHe);
#pragma unroll
  for (int i = 0; i < TILE; ++i) {
    unsigned long long km1 = 0;
    double hm1 = 0.0;
    float hf1 = 0.0f;
    int ke1 = 0, he1 = 0;
    if (i + 1 < TILE) {
      km1 = lds_u64(aKm + (i + 1) * 33 * 8);
      if (MIXED) hf1 = lds_f32(aHm + (i + 1) * 33 * 4);
      else hm1 = lds_f64(aHm + (i + 1) * 33 * 8);
      ke1 = lds_s32(aKe + (i + 1) * 33 * 4);
      he1 = lds_s32(aHe + (i + 1) * 33 * 4);
    }
    if constexpr (MIXED) {
      acc = xs_fma(acc, km, ke, y);  // the dependency chain
      // next tile's rows, off the chain: float32 on the top 24 bits of y
      fmerge(nsum, nexp, __int_as_float((int)((y.m >> 7) & 0x7FFFFFu) | 0x3F800000) * hf, he + y.e);
    } else {
      acc = xi_fma<false>(acc, km, ke, y);  // the dependency chain
      nxt = fma_chain(nxt, hm, he, xi_to_xd(y));
    }
    y.m = __shfl_sync(0xffffffffu, acc.m, i);
    y.e = __shfl_sync(0xffffffffu, acc.e, i);
    km = km1; hm = hm1; hf = hf1; ke = ke1; he = he1;
  }
  if (MIXED) nxt = xd{f2d_int(nsum), nexp};

  if (row < N) {  // Y_{row+1} = final accumulator of row `row`
    xd yn;
    if constexpr (MIXED) yn = xs_to_xd(acc);
    else yn = xi_to_xd(acc);
    Ym[(row + 1) & ymask] = yn.m;
    Ye[(row + 1) & ymask] = yn.e;
    if (gYm) {
      gYm[row + 1] = yn.m;
      gYe[row + 1] = yn.e;
    }
  }
  nxt = xnorm_int(nxt);
}

// ------------------------------------------------ asynchronous copies
// Bulk copies (TMA) into this CTA's shared memory signal an mbarrier with
// their byte count; per-thread cp.async copies complete by commit groups.
// Neither is waited for by the CTA or cluster barriers in between, so a copy
// issued in one period of a recursion lands during the next.
__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}
// generic-proxy accesses of a buffer before the bulk copy that overwrites it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// bytes (a multiple of 16) from global src to shared dst (both 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
// Wait for the mbarrier phase of the given parity, bounded (about a second):
// on expiry the status word records ST_TIMEOUT and the caller goes on (the
// evaluation's results are then invalid; the host reports BPIMD_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity, int *status) {
  for (unsigned i = 0; i < (1u << 25); ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (i >= 64) __nanosleep(32);
  }
  atomicOr(status, ST_TIMEOUT);
  return false;
}
// ------------------------------------------ hand-offs between CTAs of a cluster
// A producer stores into another CTA's shared memory with st.async, each store
// completing its byte count on an mbarrier of the receiving CTA; one producer
// thread adds the single expected arrival with the total byte count.  The
// consumer waits for the phase (its transaction count covers the stores).  No cluster barrier
// is involved, so producer and consumer run decoupled.
constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;  // bound of every hand-off wait (1 s)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ unsigned cluster_addr(unsigned local, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async_u64(unsigned raddr, unsigned long long v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr), "l"(v),
               "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void st_async_u32(unsigned raddr, unsigned v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(raddr), "r"(v),
               "r"(rbar)
               : "memory");
}
// the one expected arrival of a hand-off, with its byte count, on a remote mbarrier
__device__ __forceinline__ void mbar_arrive_expect_remote(unsigned rbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.relaxed.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(rbar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test_cluster(unsigned addr, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(addr), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for a hand-off, bounded by WAIT_LIMIT_NS of the global timer.  Once a
// wait of this CTA has expired (*aborted set), later waits return at once and
// the caller stops handing off: the status word records ST_TIMEOUT and the
// evaluation's results are invalid, but every thread still reaches the end.
__device__ __forceinline__ bool handoff_wait(unsigned addr, unsigned parity, int *status, volatile int *aborted) {
  if (*aborted) return false;
  if (mbar_test_cluster(addr, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test_cluster(addr, parity)) {
    if (*aborted || global_ns() - t0 > WAIT_LIMIT_NS) {
      *aborted = 1;
      atomicOr(status, ST_TIMEOUT);
      return false;
    }
  }
  return true;
}
// split cluster barrier: arrive (release) once this thread's part is done, wait later
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cp_async16(unsigned dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// one arrival on a CTA-local mbarrier once this thread's cp.async copies so far
// have landed (the barrier counts one arrival per copying thread)
__device__ __forceinline__ void cp_async_arrive(unsigned mbar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async8(unsigned dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ------------------------------------------------ the blocked recursion
// Sums of products in the chain's integer format.  A term K y (K = kk
// 2^(ke - 63) with kk in [2^63, 2^64), y an xi) is the high product
// p = kk y.m / 2^64 in [2^61, 2^63), of value p 2^(pe - 62), pe = ke + y.e + 1;
// an xi itself is the term (y.m, y.e).  A sum of at most 2^S terms is aligned
// to the largest exponent E with S bits of headroom: s = sum_i p_i >>
// (E - pe_i + S) < 2^63, of value s 2^(E + S - 62); each shift truncates below
// 2^-(61 - S) of the largest term.  Partial sums of one S combine by xsum_add.
struct xsum {
  unsigned long long s;
  int E;
};
__device__ __forceinline__ xsum xsum_add(xsum a, xsum b) {
  const int E = max(a.E, b.E);
  return xsum{(a.s >> min(E - a.E, 63)) + (b.s >> min(E - b.E, 63)), E};
}
// sum over K products kk[i] y[i] plus the term (p0, pe0) (p0 = 0: none)
template <int S, int K>
__device__ __forceinline__ xsum xsum_dot(const unsigned long long *kk, const int *ke, const xi *y,
                                         unsigned long long p0, int pe0) {
  unsigned long long p[K];
  int pe[K];
  int E = pe0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    p[i] = __umul64hi(kk[i], y[i].m);
    pe[i] = ke[i] + y[i].e + 1;
    E = max(E, pe[i]);
  }
  unsigned long long s = p0 >> min(E - pe0 + S, 63);
#pragma unroll
  for (int i = 0; i < K; ++i) s += p[i] >> min(E - pe[i] + S, 63);
  return xsum{s, E};
}
// The sum as an xi (s > 0: every term has a normalised mantissa).  Results
// below the extended zero's exponent become the extended zero, so exponents
// stay far from int32 overflow however many zeros a value has met.
template <int S>
__device__ __forceinline__ xi xsum_fin(xsum a) {
  const int lz = __clzll((long long)a.s);  // 1 <= lz <= S + 2
  const int e = a.E + S - (lz - 1);
  if (e < XZERO_E) return xi{1ull << 62, XZERO_E};
  return xi{a.s << (lz - 1), e};
}
// A float partial sum x 2^E (x >= 0) as an xi.
__device__ __forceinline__ xi xi_from_float(float x, int E) {
  const unsigned b = (unsigned)__float_as_int(x);
  if (b < 0x00800000u) return xi{1ull << 62, XZERO_E};
  return xi{(unsigned long long)((b & 0x7FFFFFu) | 0x800000u) << 39, E + (int)(b >> 23) - 127};
}
// The top 24 bits of an xi mantissa as a float in [1, 2) (exponent y.e).
__device__ __forceinline__ float xi_mant_float(xi y) {
  return __int_as_float((int)((unsigned)(y.m >> 39) & 0x7FFFFFu) | 0x3F800000);
}

// Reduced prefix sums C'[i+1] = sum_{q<=i} Ap[q] of tile t (one warp), and the
// running total of the integer exponent parts n_q that the recursion carries
// in its exponents (ncarry, exact in 64 bits).
__device__ __forceinline__ void prefix_tile(const Workspace &w, int t, double &carry, long long &ncarry) {
  const int lane = threadIdx.x & 31;
  const int i = t * TILE + lane;
  double v = (i < w.N) ? __ldg(w.Ap + i) : 0.0;
  int n = (i < w.N) ? __ldg(w.nexp + i) : 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (i < w.N) w.C[i + 1] = carry + v;
  carry += __shfl_sync(0xffffffffu, v, 31);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  ncarry += n;
}

// V = C' - (ln y - n ln 2)/beta for an extended y = m 2^e whose exponent
// carries n from the coefficients c: (e - n) ln 2 is formed with ln 2 to 106
// bits, so the result is accurate to a few float64 roundings of V's own size.
__device__ __forceinline__ double reduced_potential(double Cp, xd y, long long n, double beta) {
  const double k = (double)((long long)y.e - n);
  const double t = fma(k, LN2, fma(k, LN2_LO, log(y.m)));
  return Cp - t / beta;
}

}  // namespace chain_detail
}  // namespace bpimd
