// The pair Boltzmann factor of the closing spring of cycle [a, b] (Eq.
// e-recurrence-step, last term):
//   g(a, b) = exp(-beta (1/2) m w_P^2 |r_b^P - r_a^1|^2) = 2^(-cx d^2),
//   cx = beta (1/2) k log2(e),
// from the endpoint copies of the bead pass, as an extended number (mantissa,
// exponent).  Shared by the kernels that tabulate g (prep.cu) and by those
// that recompute it where it is used (recompute mode: recursions,
// probabilities, diagnostics), so that both give the same bits.
//   FP64   : float64 difference and square (minimum image in a box); 2^(-x)
//            of the exact float64 x float64 product on the integer pipe.
//   MIXED  : float32 difference of the high/low parts (or of the 32-bit
//            fixed-point copies in a box) and float32 square; 2^(-x) of the
//            exact float32 x float64 product on the integer pipe.
//   MIXED32: the same float32 square; hardware ex2.approx of the float32 x.
// Exponents below -2^28 stand for zero (every exponent sum stays in int32).
#pragma once
#include <type_traits>

#include "bpimd_internal.cuh"
#include "pow2_fixed.cuh"

namespace bpimd {
namespace pairg {

// An endpoint bead as the kernels hold it: float64 coordinates (FP64),
// float32 high/low parts (mixed forms, open box) or fixed-point fractions of
// the box (mixed forms, periodic box).
template <bool B32, bool PBC>
struct EndPt;
template <bool PBC>
struct EndPt<false, PBC> {
  double x, y, z;
};
template <>
struct EndPt<true, false> {
  float4 h, l;
};
template <>
struct EndPt<true, true> {
  uint4 u;
};

// Endpoint i from the bead pass's copies: bead 1 (R1/R1s) or bead P (RP/RPs).
template <bool B32, bool PBC>
__device__ __forceinline__ EndPt<B32, PBC> load_end(const Workspace &w, int i, bool beadP) {
  EndPt<B32, PBC> e;
  if constexpr (!B32) {
    const double *r = (beadP ? w.RP : w.R1) + 4 * (size_t)i;
    const double2 xy = *(const double2 *)r;
    e.x = xy.x;
    e.y = xy.y;
    e.z = r[2];
  } else if constexpr (PBC) {
    e.u = *(const uint4 *)((beadP ? w.RPs : w.R1s) + 8 * (size_t)i);
  } else {
    const float4 *r = (const float4 *)((beadP ? w.RPs : w.R1s) + 8 * (size_t)i);
    e.h = r[0];
    e.l = r[1];
  }
  return e;
}

// Squared distance |b - a|^2: float64 (FP64) or float32 (mixed forms).
template <bool PBC>
__device__ __forceinline__ double dist2(const Workspace &w, const EndPt<false, PBC> &b, const EndPt<false, PBC> &a) {
  double dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
  if (PBC) { dx = mimage(w, dx); dy = mimage(w, dy); dz = mimage(w, dz); }
  return fma(dx, dx, fma(dy, dy, dz * dz));
}
__device__ __forceinline__ float dist2(const Workspace &, const EndPt<true, false> &b, const EndPt<true, false> &a) {
  const float fx = (b.h.x - a.h.x) + (b.l.x - a.l.x);
  const float fy = (b.h.y - a.h.y) + (b.l.y - a.l.y);
  const float fz = (b.h.z - a.h.z) + (b.l.z - a.l.z);
  return fmaf(fx, fx, fmaf(fy, fy, fz * fz));
}
__device__ __forceinline__ float dist2(const Workspace &w, const EndPt<true, true> &b, const EndPt<true, true> &a) {
  const float fx = fixdiff(b.u.x, a.u.x, w.Lscale);
  const float fy = fixdiff(b.u.y, a.u.y, w.Lscale);
  const float fz = fixdiff(b.u.z, a.u.z, w.Lscale);
  return fmaf(fx, fx, fmaf(fy, fy, fz * fz));
}

// The difference r_b - r_a: float64 components (FP64, minimum image in a
// box) or float32 components (mixed forms: high/low parts, or fixed point).
template <bool PBC>
__device__ __forceinline__ double3 diff3(const Workspace &w, const EndPt<false, PBC> &b, const EndPt<false, PBC> &a) {
  double dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
  if (PBC) { dx = mimage(w, dx); dy = mimage(w, dy); dz = mimage(w, dz); }
  return make_double3(dx, dy, dz);
}
__device__ __forceinline__ float3 diff3(const Workspace &, const EndPt<true, false> &b, const EndPt<true, false> &a) {
  return make_float3((b.h.x - a.h.x) + (b.l.x - a.l.x), (b.h.y - a.h.y) + (b.l.y - a.l.y),
                     (b.h.z - a.h.z) + (b.l.z - a.l.z));
}
__device__ __forceinline__ float3 diff3(const Workspace &w, const EndPt<true, true> &b, const EndPt<true, true> &a) {
  return make_float3(fixdiff(b.u.x, a.u.x, w.Lscale), fixdiff(b.u.y, a.u.y, w.Lscale), fixdiff(b.u.z, a.u.z, w.Lscale));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// g from a squared distance; cx = beta (1/2) k log2(e) > 0.  Returns the
// mantissa (float for MIXED32, else double in [1, 2)) and sets the exponent.
template <int MODE>
__device__ __forceinline__ typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type
g_of_d2(typename std::conditional<MODE == BPIMD_FP64, double, float>::type d2, double cx,
        const unsigned long long *T63, int &e) {
  if constexpr (MODE == BPIMD_FP64) {
    const pow2fx::mexp g = pow2fx::pow2neg_dd(d2, cx, T63);
    e = g.e;
    return g.m;
  } else if constexpr (MODE == BPIMD_MIXED) {
    const pow2fx::mexp g = pow2fx::pow2neg_fd(d2, cx, T63);
    e = g.e;
    return g.m;
  } else {
    const float x = fmaxf(-(float)cx * d2, -268435456.0f);
    const float n = floorf(x);
    float mm = ex2_approx(x - n);  // in [1, 2]
    e = (int)n;
    if (mm >= 2.0f) { mm *= 0.5f; e += 1; }
    return mm;
  }
}

// g(a, b) from the endpoint b (bead P) and a (bead 1).
template <int MODE, bool PBC>
__device__ __forceinline__ typename std::conditional<MODE == BPIMD_MIXED32, float, double>::type
g_of(const Workspace &w, const EndPt<MODE != BPIMD_FP64, PBC> &b, const EndPt<MODE != BPIMD_FP64, PBC> &a,
     double cx, const unsigned long long *T63, int &e) {
  return g_of_d2<MODE>(dist2(w, b, a), cx, T63, e);
}

// g(a, b) for any precision form and box, dispatched at run time (diagnostic
// kernels of the recompute mode); the table is read from global memory.
__device__ __forceinline__ xd g_runtime(const Workspace &w, int a, int b) {
  int e = 0;
  double m;
  const unsigned long long *T = pow2fx::T63;
  if (w.mode == BPIMD_FP64) {
    if (w.pbc) m = g_of<BPIMD_FP64, true>(w, load_end<false, true>(w, b, true), load_end<false, true>(w, a, false), w.cx, T, e);
    else m = g_of<BPIMD_FP64, false>(w, load_end<false, false>(w, b, true), load_end<false, false>(w, a, false), w.cx, T, e);
  } else if (w.mode == BPIMD_MIXED) {
    if (w.pbc) m = g_of<BPIMD_MIXED, true>(w, load_end<true, true>(w, b, true), load_end<true, true>(w, a, false), w.cx, T, e);
    else m = g_of<BPIMD_MIXED, false>(w, load_end<true, false>(w, b, true), load_end<true, false>(w, a, false), w.cx, T, e);
  } else {
    if (w.pbc) m = g_of<BPIMD_MIXED32, true>(w, load_end<true, true>(w, b, true), load_end<true, true>(w, a, false), w.cx, T, e);
    else m = g_of<BPIMD_MIXED32, false>(w, load_end<true, false>(w, b, true), load_end<true, false>(w, a, false), w.cx, T, e);
  }
  return xd{m, e};
}

// Shared-memory copy of the table of 2^(-j/256) used by the integer power
// (all threads of the block call it; the caller's next barrier publishes it).
__device__ __forceinline__ void table_init(unsigned long long *T) {
  for (int j = threadIdx.x; j < 256; j += blockDim.x) T[j] = pow2fx::T63[j];
}

}  // namespace pairg
}  // namespace bpimd
