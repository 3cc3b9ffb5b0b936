// Device helpers of the recursion kernels (chain.cu: one cluster per
// recursion; chain_batched.cu: one CTA per recursion of a replica batch).
// Internal; included by those two files only.
#pragma once
#include <type_traits>

#include "bpimd_internal.cuh"

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

// a * b with integer normalisation (one float64 multiply).
__device__ __forceinline__ xd xmul_int(xd a, xd b) { return xnorm_int(xd{a.m * b.m, a.e + b.e}); }

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

// a * b and a + b for xk numbers (mantissas in [2^63, 2^64)); both truncate.
__device__ __forceinline__ xk xk_mul(xk a, xk b) {
  const unsigned long long hi = __umul64hi(a.m, b.m);  // in [2^62, 2^64)
  const int sh = (int)(hi >> 63);
  return xk{hi << (1 - sh), a.e + b.e + sh};
}
__device__ __forceinline__ xk xk_add(xk a, xk b) {
  const int E = max(a.e, b.e);
  const unsigned long long s = (a.m >> min(E - a.e + 1, 63)) + (b.m >> min(E - b.e + 1, 63));  // [2^62, 2^64)
  const int sh = (int)(s >> 63);
  return xk{s << (1 - sh), E + sh};
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
// kk * ym / 2^64 for kk in [2^63, 2^64), ym in [2^62, 2^63): in [2^61, 2^63).
// MIXED uses the top 32 bits of kk only (two 32 x 32-bit products, relative
// error below 2^-30: K = c g carries a float32 g there).
template <bool MIXED>
__device__ __forceinline__ unsigned long long kprod(unsigned long long kk, unsigned long long ym) {
  if (MIXED) {
    const unsigned k1 = (unsigned)(kk >> 32);
    return (unsigned long long)k1 * (unsigned)(ym >> 32) + (((unsigned long long)k1 * (unsigned)ym) >> 32);
  }
  return __umul64hi(kk, ym);
}

// acc + K * y with K = kk 2^(ke - 63), kk in [2^63, 2^64).  The aligned sum
// lies in [2^61, 2^64); a K carrying an extended-zero exponent leaves acc
// unchanged.
template <bool MIXED>
__device__ __forceinline__ xi xi_fma(xi acc, unsigned long long kk, int ke, xi y) {
  const unsigned long long p = kprod<MIXED>(kk, y.m);
  const int pe = ke + y.e + 1;
  const int E = max(acc.e, pe);
  return xi_norm((acc.m >> min(E - acc.e, 63)) + (p >> min(E - pe, 63)), E);
}

// acc + K1 y1 + K2 y2, the step of the dependency chain: the three terms are
// aligned to the largest exponent with one more bit of headroom (each below
// 2^62, the sum s in [2^60, 3 * 2^62), value s 2^(E - 61)), added, and brought
// back to [2^62, 2^63) by a select on the top bits.
template <bool MIXED>
__device__ __forceinline__ xi xi_fma2(xi acc, unsigned long long k1, int e1, xi y1, unsigned long long k2, int e2,
                                      xi y2) {
  const unsigned long long p1 = kprod<MIXED>(k1, y1.m), p2 = kprod<MIXED>(k2, y2.m);
  const int pe1 = e1 + y1.e + 1, pe2 = e2 + y2.e + 1;
  const int E = max(acc.e, max(pe1, pe2));
  const unsigned long long s =
      (acc.m >> min(E - acc.e + 1, 63)) + (p1 >> min(E - pe1 + 1, 63)) + (p2 >> min(E - pe2 + 1, 63));
  const unsigned t = (unsigned)(s >> 60);  // 1: [2^60,2^61)  2-3: [2^61,2^62)  4-7: [2^62,2^63)  8-11: [2^63,2^64)
  return xi{t >= 8 ? (s >> 1) : (t >= 4 ? s : (t >= 2 ? (s << 1) : (s << 2))),
            E + (t >= 8 ? 2 : (t >= 4 ? 1 : (t >= 2 ? 0 : -1)))};
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

// Diagonal block of tile tt in the chain's look-ahead form.  With K(i, j) =
// c_j H(r0+i, r0+j) (source i, row j of the tile), row j's equation
//   Y_{r0+j+1} = a_j + sum_{i<=j} K(i, j) Y_{r0+i}
// takes in row j-1's equation for Y_{r0+j} (j >= 1):
//   Y_{r0+j+1} = a_j + D_j a_{j-1} + sum_{i<=j-1} Kh(i, j) Y_{r0+i},
//   Kh(i, j) = K(i, j) + D_j K(i, j-1),  D_j = K(j, j),
// so that Y_{r0+j+1} waits for Y_{r0+j-1} at the latest (all terms are
// nonnegative: no cancellation).  Row 0 keeps Kh(0, 0) = K(0, 0).  Staged as
// xk numbers (64-bit integer mantissas) for rows i in [i0, i0+NR) of the
// block, entries outside the look-ahead triangle as extended zeros; the
// warp with i0 = 0 also stores D_j.  Integer pipe only (mul_mant, xk_*).
template <bool MIXED, bool BWD, int NR>
__device__ __forceinline__ void stage_diag(const Workspace &w, int tt, int i0, unsigned long long *dm, int *de,
                                           unsigned long long *dgm, int *dge) {
  using M_t = typename std::conditional<MIXED, float, double>::type;
  const int j = threadIdx.x & 31;
  const int r0 = tt * TILE, row = r0 + j;
  const bool valid = row < w.N;
  const M_t *gm = (const M_t *)chain_gm<BWD>(w);
  const int *ge = chain_ge<BWD>(w);
  const xd c = valid ? xnorm_int(chain_coef<BWD>(w, row)) : xd{1.0, 0};
  const xd cp = (valid && j >= 1) ? xnorm_int(chain_coef<BWD>(w, row - 1)) : xd{1.0, 0};
  M_t hd = (M_t)1.0, hm[NR], hp[NR];
  int hde = XZERO_E, he[NR], hpe[NR];
  if (valid) {
    const size_t gi = hidx(row, row);
    hd = __ldg(gm + gi);
    hde = __ldg(ge + gi);
  }
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const int i = i0 + k;
    hm[k] = (M_t)1.0; hp[k] = (M_t)1.0; he[k] = XZERO_E; hpe[k] = XZERO_E;
    if (valid && (j == 0 ? i == 0 : i <= j - 1)) {
      const size_t gi = hidx(r0 + i, row);
      hm[k] = __ldg(gm + gi);
      he[k] = __ldg(ge + gi);
      if (j >= 1) {
        const size_t gp = hidx(r0 + i, row - 1);
        hp[k] = __ldg(gm + gp);
        hpe[k] = __ldg(ge + gp);
      }
    }
  }
  const xk D = mul_mant<M_t>(c, hd, hde);
  if (i0 == 0) { dgm[j] = D.m; dge[j] = max(D.e, XZERO_E); }
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    xk kh = mul_mant<M_t>(c, hm[k], he[k]);
    if (j >= 1) kh = xk_add(kh, xk_mul(D, mul_mant<M_t>(cp, hp[k], hpe[k])));
    dm[(i0 + k) * 33 + j] = kh.m;
    de[(i0 + k) * 33 + j] = max(kh.e, XZERO_E);  // keeps every exponent sum in int32
  }
}

// The dependent steps of row tile t, run by one warp.  A is this lane's row
// sum over sources < 32t except tile t-1 (which is in nxt), crow the row's
// coefficient; Kh/D (look-ahead form, stage_diag) and H (to tile t+1) are the
// staged blocks.  Y_v lives at Ym/Ye[v & ymask] in shared memory and, unless
// gYm is null, at gYm/gYe[v] in global memory.  On return nxt holds the
// partial sums of tile t+1's rows over source tile t.
// Step 0 adds source 0 (Y_{r0}); step s = 1..15 adds sources 2s-1 and 2s,
// after which rows 2s and 2s+1 are final and their Y are shuffled out: 16
// dependent steps of one three-term aligned sum each.  No branches and no
// stores inside: rows past N and finished rows see extended zeros.  The chain
// is in the integer format xi; the block entries of step s+1 are loaded
// (explicit ld.shared) before step s's shuffles.
template <bool MIXED>
__device__ __forceinline__ void chain_tile(int N, int t, xd A, xd crow, xd &nxt, const unsigned long long *Kdm,
                                           const int *Kde, const unsigned long long *Dm, const int *De,
                                           const double *Hom, const int *Hoe, double *Ym, int *Ye, int ymask,
                                           double *gYm, int *gYe) {
  const int lane = threadIdx.x & 31;
  const int r0 = t * TILE, row = r0 + lane;
  // a_j = c_j (A_j + nxt_j); the look-ahead row starts from a_j + D_j a_{j-1}
  xi a{1ull << 62, XZERO_E};
  if (row < N) a = xi_mul(xi_add(xi_from(A), xi_from(nxt)), crow);
  xi ap;
  ap.m = __shfl_up_sync(0xffffffffu, a.m, 1);
  ap.e = __shfl_up_sync(0xffffffffu, a.e, 1);
  xi acc = (lane >= 1) ? xi_fma<MIXED>(a, Dm[lane], De[lane], ap) : a;
  xi y1 = xi_from(xd{Ym[r0 & ymask], Ye[r0 & ymask]}), y2;
  float nsum = 0.0f;  // MIXED: the next tile's partial sum in float32
  int nexp = XZERO_E;
  xi nx{1ull << 62, XZERO_E};  // FP64: the next tile's partial sum in the integer format
  const unsigned aKm = smem_addr(Kdm + lane), aKe = smem_addr(Kde + lane), aHe = smem_addr(Hoe + lane);
  const unsigned aHm = MIXED ? smem_addr((const float *)Hom + lane) : smem_addr(Hom + lane);
  const int hsz = MIXED ? 4 : 8;
  // H(source i, row of tile t+1) as a chain-format factor (FP64) or float (MIXED)
  auto hk = [&](int i) -> unsigned long long {
    return MIXED ? 0ull : mant53(lds_f64(aHm + i * 33 * 8)) << 11;
  };
  auto hf = [&](int i) -> float { return MIXED ? lds_f32(aHm + i * 33 * 4) : 0.0f; };
  auto nadd = [&](xi y, float h, int e) {  // MIXED: one term of the next tile's sum
    fmerge(nsum, nexp, __int_as_float((int)((y.m >> 39) & 0x7FFFFFu) | 0x3F800000) * h, e + y.e);
  };
  // step 0: source 0
  {
    const unsigned long long k0 = lds_u64(aKm);
    const int ke0 = lds_s32(aKe), he0 = lds_s32(aHe);
    acc = xi_fma<MIXED>(acc, k0, ke0, y1);
    if (MIXED) nadd(y1, hf(0), he0);
    else nx = xi_fma<false>(nx, hk(0), he0, y1);
  }
  unsigned long long ka = lds_u64(aKm + 1 * 33 * 8), kb = lds_u64(aKm + 2 * 33 * 8);
  int kea = lds_s32(aKe + 1 * 33 * 4), keb = lds_s32(aKe + 2 * 33 * 4);
  int hea = lds_s32(aHe + 1 * 33 * 4), heb = lds_s32(aHe + 2 * 33 * 4);
  float hfa = hf(1), hfb = hf(2);
  unsigned long long hka = hk(1), hkb = hk(2);
  y2.m = __shfl_sync(0xffffffffu, acc.m, 1);
  y2.e = __shfl_sync(0xffffffffu, acc.e, 1);
  y1.m = __shfl_sync(0xffffffffu, acc.m, 0);
  y1.e = __shfl_sync(0xffffffffu, acc.e, 0);
#pragma unroll
  for (int s = 1; s < TILE / 2; ++s) {
    unsigned long long ka1 = 0, kb1 = 0, hka1 = 0, hkb1 = 0;
    int kea1 = 0, keb1 = 0, hea1 = 0, heb1 = 0;
    float hfa1 = 0.0f, hfb1 = 0.0f;
    if (s + 1 < TILE / 2) {  // entries of step s+1: sources 2s+1, 2s+2
      ka1 = lds_u64(aKm + (2 * s + 1) * 33 * 8);
      kb1 = lds_u64(aKm + (2 * s + 2) * 33 * 8);
      kea1 = lds_s32(aKe + (2 * s + 1) * 33 * 4);
      keb1 = lds_s32(aKe + (2 * s + 2) * 33 * 4);
      hea1 = lds_s32(aHe + (2 * s + 1) * 33 * 4);
      heb1 = lds_s32(aHe + (2 * s + 2) * 33 * 4);
      hfa1 = hf(2 * s + 1); hfb1 = hf(2 * s + 2);
      hka1 = hk(2 * s + 1); hkb1 = hk(2 * s + 2);
    }
    acc = xi_fma2<MIXED>(acc, ka, kea, y1, kb, keb, y2);  // the dependency chain
    if (MIXED) { nadd(y1, hfa, hea); nadd(y2, hfb, heb); }
    else nx = xi_fma2<false>(nx, hka, hea, y1, hkb, heb, y2);
    y1.m = __shfl_sync(0xffffffffu, acc.m, 2 * s);
    y1.e = __shfl_sync(0xffffffffu, acc.e, 2 * s);
    y2.m = __shfl_sync(0xffffffffu, acc.m, 2 * s + 1);
    y2.e = __shfl_sync(0xffffffffu, acc.e, 2 * s + 1);
    ka = ka1; kb = kb1; kea = kea1; keb = keb1; hea = hea1; heb = heb1;
    hfa = hfa1; hfb = hfb1; hka = hka1; hkb = hkb1;
  }
  // source 31 (Y_{r0+31} = y1) enters only the next tile's sums
  {
    const int he31 = lds_s32(aHe + 31 * 33 * 4);
    if (MIXED) nadd(y1, hf(31), he31);
    else nx = xi_fma<false>(nx, hk(31), he31, y1);
  }
  nxt = MIXED ? xnorm_int(xd{f2d_int(nsum), nexp}) : xi_to_xd(nx);
  if (row < N) {  // Y_{row+1} = final accumulator of row `row`
    const xd yn = xi_to_xd(acc);
    Ym[(row + 1) & ymask] = yn.m;
    Ye[(row + 1) & ymask] = yn.e;
    if (gYm) {
      gYm[row + 1] = yn.m;
      gYe[row + 1] = yn.e;
    }
  }
}

// Prefix sums C[i+1] = sum_{q<=i} (E_int_q + link_q) of tile t, one warp.
__device__ __forceinline__ void prefix_tile(const Workspace &w, int t, double &carry) {
  const int lane = threadIdx.x & 31;
  const int i = t * TILE + lane;
  double v = (i < w.N) ? (__ldg(w.Eint + i) + __ldg(w.link + i)) : 0.0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (i < w.N) w.C[i + 1] = carry + v;
  carry += __shfl_sync(0xffffffffu, v, 31);
}

}  // namespace chain_detail
}  // namespace bpimd
