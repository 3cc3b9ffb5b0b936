// Powers 2^(-x), x >= 0, to float64 accuracy on the integer pipe.
//
// The float64 pipe of a GB300 SM issues one warp instruction about every 64
// cycles, so the O(N^2) pair Boltzmann factors g = exp(-beta (1/2) k d^2)
// avoid it.  Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2), 1989)
// in 64-bit fixed point:
//   x = n + f, n integer, f in [0, 1) as a 64-bit fraction F = f 2^64 (x is
//   the exact product of the argument's factors, up to 128 bits);
//   f = j/256 + r, j = the top 8 bits of F, 0 <= r < 2^-8;
//   2^(-f) = T[j] e^(-u), u = r ln 2 < 0.0028, T[j] = 2^(-j/256) (table of
//   pow2_table.h, 63 fraction bits);
//   e^(-u) = 1 - u (1 - u (1/2 - u (1/6 - u (1/24 - u/120)))), truncation below
//   u^6/720 < 2^-60 relative, evaluated with 64 x 64 -> high-64 products.
// The result is (mantissa in [1, 2) as a double, exponent): value
// m 2^e = 2^(-x) to a few 2^-60 relative -- finer than one float64 rounding.
// x >= 2^28 gives 2^(-2^28): the recursions read exponents below -2^28 as zero.
// Host-compilable (the CPU tests emulate it bit for bit with __int128).
#pragma once
#include <cstdint>

#include "pow2_table.h"

#ifdef __CUDACC__
#define BPIMD_HD __host__ __device__ __forceinline__
#else
#define BPIMD_HD inline
#endif

namespace bpimd {
namespace pow2fx {

#ifdef __CUDA_ARCH__
__device__ const unsigned long long T63[256] = {BPIMD_POW2_T63_INIT};
BPIMD_HD unsigned long long mulhi(unsigned long long a, unsigned long long b) { return __umul64hi(a, b); }
#else
static const unsigned long long T63[256] = {BPIMD_POW2_T63_INIT};
BPIMD_HD unsigned long long mulhi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
#endif

constexpr unsigned long long Q64_HALF = 0x8000000000000000ull;
constexpr unsigned long long Q64_SIXTH = 0xFFFFFFFFFFFFFFFFull / 6;
constexpr unsigned long long Q64_24TH = 0xFFFFFFFFFFFFFFFFull / 24;
constexpr unsigned long long Q64_120TH = 0xFFFFFFFFFFFFFFFFull / 120;
constexpr int ZERO_EXP = -(1 << 28);  // 2^(-2^28): an extended zero for the recursions

struct mexp {
  double m;  // in [1, 2)
  int e;
};

BPIMD_HD double bits_to_double(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, 8);
  return d;
#endif
}
BPIMD_HD unsigned long long double_to_bits(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &d, 8);
  return b;
#endif
}

// 2^(-x) for x = (H 2^64 + L) 2^S, H in [2^63, 2^64) (a normalised 128-bit
// mantissa: exact products of two float64 or float32 mantissas fit in it).
// table: T63 or a shared-memory copy of it.
BPIMD_HD mexp pow2neg_q(unsigned long long H, unsigned long long L, int S, const unsigned long long *table) {
  if (S >= -99) return mexp{1.0, ZERO_EXP};  // x >= 2^28
  const int k = -S - 64;                      // x = (H:L) >> (k + 64); k >= 36
  const unsigned long long n = k < 64 ? (H >> k) : 0ull;
  unsigned long long F;                       // the 64 fraction bits below the binary point
  if (k < 64) F = (L >> k) | (H << (64 - k));
  else F = k < 128 ? (H >> (k - 64)) : 0ull;
  const unsigned j = (unsigned)(F >> 56);
  const unsigned long long r = F & 0x00FFFFFFFFFFFFFFull;  // f - j/256, times 2^64
  const unsigned long long u = mulhi(r, BPIMD_LN2_Q64);      // u 2^64, u = r ln 2
  unsigned long long t = Q64_24TH - mulhi(u, Q64_120TH);     // 1/24 - u/120
  t = Q64_SIXTH - mulhi(u, t);                               // 1/6 - u t
  t = Q64_HALF - mulhi(u, t);                                // 1/2 - u t
  t = 0ull - mulhi(u, t);                                    // 1 - u t, mod 2^64
  const unsigned long long q = mulhi(u, t);                  // 1 - e^(-u)
  const unsigned long long T = table[j];
  unsigned long long res = T - mulhi(T, q);  // 2^(-f) 2^63, in (2^62, 2^63]
  if (res >> 63) return mexp{1.0, -(int)n};
  if (res < (1ull << 62)) res = 1ull << 62;  // truncation cannot take it lower than 2^-1
  // leading bit at 62: mantissa (res << 1) / 2^63 in (1, 2), exponent -n - 1,
  // rounded to 53 bits (to nearest, ties up)
  const unsigned long long v = res << 1;
  unsigned long long m53 = (v >> 11) + ((v >> 10) & 1ull);
  int e = -(int)n - 1;
  if (m53 >> 53) {  // rounded up to the next power of two
    m53 >>= 1;
    e += 1;
  }
  return mexp{bits_to_double((m53 & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull), e};
}

// Full 128-bit product of two 64-bit mantissas, normalised so that the top
// bit of the high word is set (both inputs have their top bit set).
BPIMD_HD void mul128_norm(unsigned long long a, unsigned long long b, unsigned long long &H,
                          unsigned long long &L, int &shift) {
  H = mulhi(a, b);
  L = a * b;
  shift = 0;
  if (!(H >> 63)) {
    H = (H << 1) | (L >> 63);
    L <<= 1;
    shift = 1;
  }
}

// 2^(-x) for a double x >= 0 (its bits read by integer instructions).
BPIMD_HD mexp pow2neg(double x, const unsigned long long *table) {
  const unsigned long long b = double_to_bits(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return mexp{1.0, 0};  // 0 or subnormal: 2^(-x) = 1 to 2^-1000
  const unsigned long long M = ((b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  return pow2neg_q(M, 0ull, E - 1023 - 63 - 64, table);
}

// 2^(-x) for x = a * c with a float32 a >= 0 and a double c > 0: the product
// is formed exactly (24 x 53 bits), so the float32 argument is not rounded
// again.
BPIMD_HD mexp pow2neg_fd(float a, double c, const unsigned long long *table) {
#ifdef __CUDA_ARCH__
  const unsigned ab = (unsigned)__float_as_int(a);
#else
  unsigned ab;
  __builtin_memcpy(&ab, &a, 4);
#endif
  const int Ea = (int)((ab >> 23) & 0xFF);
  if (Ea == 0) return mexp{1.0, 0};
  const unsigned long long cb = double_to_bits(c);
  const int Ec = (int)((cb >> 52) & 0x7FF);
  const unsigned long long ma = (unsigned long long)((ab & 0x7FFFFFu) | 0x800000u) << 40;  // top bit set
  const unsigned long long mc = ((cb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  unsigned long long H, L;
  int sh;
  mul128_norm(ma, mc, H, L, sh);
  // a = ma 2^(Ea-127-63), c = mc 2^(Ec-1023-63): x = (H:L) 2^(Ea-190 + Ec-1086 - sh)
  return pow2neg_q(H, L, (Ea - 190) + (Ec - 1086) - sh, table);
}

// 2^(-x) for x = a * c with doubles a >= 0, c > 0: the 53 x 53-bit mantissa
// product is formed exactly on the integer pipe, so the float64 argument is
// not rounded again either.
BPIMD_HD mexp pow2neg_dd(double a, double c, const unsigned long long *table) {
  const unsigned long long ab = double_to_bits(a), cb = double_to_bits(c);
  const int Ea = (int)((ab >> 52) & 0x7FF), Ec = (int)((cb >> 52) & 0x7FF);
  if (Ea == 0) return mexp{1.0, 0};
  const unsigned long long ma = ((ab & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  const unsigned long long mc = ((cb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  unsigned long long H, L;
  int sh;
  mul128_norm(ma, mc, H, L, sh);
  return pow2neg_q(H, L, (Ea - 1086) + (Ec - 1086) - sh, table);
}

}  // namespace pow2fx
}  // namespace bpimd
