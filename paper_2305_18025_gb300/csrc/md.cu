// Molecular dynamics of the bosonic ring polymers.
//
// The paper samples exp(-beta (V^{[1,N]} + U-bar)) (Eq.
// int-of-sum-all-permutations; spring frequency w_P = sqrt(P)/(beta hbar),
// Eq. eperm; U-bar = (1/P) sum_j U(r_1^j..r_N^j)) with molecular dynamics and
// a thermostat, without stating the integrator.  This file runs Cartesian
// BAOAB Langevin steps at temperature kT (default 1/beta) with bead mass m:
//   B  v += (dt/2) F/m            A  x += (dt/2) v
//   O  v  = c1 v + c2 z,  c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT/m)
//   A  x += (dt/2) v              F = -grad(V^{[1,N]} + U-bar)(x)
//   B  v += (dt/2) F/m
// with U = sum_l (1/2) m w0^2 |r_l|^2 (harmonic trap) + sum_{l<l'} g
// exp(-|r_l - r_l'|^2 / (2 s^2)) (Gaussian repulsion) or Lennard-Jones
// 4 eps ((sig/r)^12 - (sig/r)^6) truncated and shifted at rc (liquid helium;
// cell lists in pairs.cu when the box holds >= 3 cutoffs per side) between
// beads of equal index; in a periodic box every spring and pair uses the
// minimum image.  The exchange force is one evaluation of Algorithm 1 (the kernels of
// prep.cu, chain.cu, force.cu).
//
// Thermostat noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
// written here from its published definition.  Element e = 4g + i of the
// velocity array at step s takes word i of the block with counter
// (g, s mod 2^32, s div 2^32, 0) and key (seed mod 2^32, seed div 2^32);
// words become uniforms u = (x + 1/2) 2^-32 and pairs of uniforms become
// normals by the Box-Muller transform (float64; MIXED: float32).
//
// One step (7 kernel launches) is captured once into a CUDA graph bound to the
// caller's position and velocity buffers and replayed; the step counter lives
// in device memory and is advanced by the last kernel of the step.
#include <cmath>
#include <vector>
#include <type_traits>

#include "context.cuh"
#include "pairg.cuh"
#include "pairs.cuh"

namespace bpimd {
namespace {

constexpr int MD_THREADS = 256;
constexpr int EXT_THREADS = 256;
constexpr int EXT_SPLIT = 4;  // lanes per particle in the all-pairs force
constexpr int EXT_PARTICLES = EXT_THREADS / EXT_SPLIT;
constexpr int EXT_CHUNK = 1024;  // positions of one bead index staged per pass

struct alignas(16) Dbl4 {
  double x, y, z, w;
};

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

template <bool MIXED>
__device__ __forceinline__ void box_muller(const uint32_t x[4], double z[4]) {
  if (MIXED) {
    float u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = ((float)x[i] + 0.5f) * 2.3283064365386963e-10f;
    const float ra = sqrtf(-2.0f * logf(u[0])), rb = sqrtf(-2.0f * logf(u[2]));
    float sa, ca, sb, cb;
    sincosf(6.28318530717958648f * u[1], &sa, &ca);
    sincosf(6.28318530717958648f * u[3], &sb, &cb);
    z[0] = ra * ca; z[1] = ra * sa; z[2] = rb * cb; z[3] = rb * sb;
  } else {
    double u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = ((double)x[i] + 0.5) * 2.3283064365386962890625e-10;
    const double two_pi = 6.283185307179586476925286766559;
    const double ra = sqrt(-2.0 * log(u[0])), rb = sqrt(-2.0 * log(u[2]));
    double sa, ca, sb, cb;
    sincos(two_pi * u[1], &sa, &ca);
    sincos(two_pi * u[3], &sb, &cb);
    z[0] = ra * ca; z[1] = ra * sa; z[2] = rb * cb; z[3] = rb * sb;
  }
}

// B A O A of one step (four velocity components per thread: one Philox block).
template <bool MIXED>
__global__ void __launch_bounds__(MD_THREADS) md_baoa_kernel(double *__restrict__ x, double *__restrict__ v,
                                                             const double *__restrict__ F, long long n,
                                                             double half_dt_over_m, double half_dt, double c1,
                                                             double c2, uint32_t k0, uint32_t k1,
                                                             const unsigned long long *__restrict__ step) {
  const unsigned long long s = *step;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; 4 * g < n;
       g += (long long)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)g, (uint32_t)s, (uint32_t)(s >> 32), 0u};
    philox4x32_10(c, k0, k1);
    double z[4];
    box_muller<MIXED>(c, z);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long e = 4 * g + i;
      if (e < n) {
        double vi = v[e] + half_dt_over_m * F[e];  // B
        double xi = x[e] + half_dt * vi;           // A
        vi = c1 * vi + c2 * z[i];                  // O
        x[e] = xi + half_dt * vi;                  // A
        v[e] = vi;
      }
    }
  }
}

// Closing B of a step; advances the step counter.
__global__ void __launch_bounds__(MD_THREADS) md_kick_kernel(double *__restrict__ v, const double *__restrict__ F,
                                                             long long n, double half_dt_over_m,
                                                             unsigned long long *step) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    v[e] += half_dt_over_m * F[e];
  if (blockIdx.x == 0 && threadIdx.x == 0) *step += 1ull;
}

// Deterministic block sum (fixed shuffle tree, then warps in order); thread 0 gets it.
// m 2^e of the integer-pipe power of two as a double (e <= 0; the exponent is
// added with integer instructions; results below the normal range give 0)
__device__ __forceinline__ double pow2_value(pow2fx::mexp r) {
  const long long b = __double_as_longlong(r.m);
  return ((int)(b >> 52) + r.e <= 0) ? 0.0 : __longlong_as_double(b + ((long long)r.e << 52));
}

// float64 -> float32, round to nearest even, on the integer pipe (a
// conversion instruction runs on GB300's narrow float64 pipe); results below
// the float32 normal range flush to a signed zero, so the value must be
// finite and below 2^128 in magnitude.  Bit-identical to __double2float_rn
// for every normal float32 result.
__device__ __forceinline__ float f32_of_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  unsigned r = (unsigned)(m >> 29);
  const unsigned long long rem = m & ((1ull << 29) - 1);
  r += (rem > (1ull << 28)) || (rem == (1ull << 28) && (r & 1u));
  return ex <= 0 ? __uint_as_float(sign) : __uint_as_float(sign | (((unsigned)ex << 23) + r));
}

// float32 -> float64 on the integer pipe (exact; zero and subnormal inputs give
// a signed zero; the value must be finite)
__device__ __forceinline__ double f64_of_f32(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned ex = (b >> 23) & 0xffu;
  const unsigned long long s = (unsigned long long)(b & 0x80000000u) << 32;
  if (ex == 0) return __longlong_as_double((long long)s);
  return __longlong_as_double(
      (long long)(s | ((unsigned long long)(ex - 127 + 1023) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// block-wide sum of a float32 per thread: float32 warp sums, float64 across warps
__device__ __forceinline__ double block_sum_f(float v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f64_of_f32(v);
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  __syncthreads();
  return s;
}

// -grad U-bar added to F, per bead index j = blockIdx.y and particle
// l = blockIdx.x * (256 / SPLIT) + thread / SPLIT (all pairs).  The SPLIT
// lanes of one particle take the partners q = sub, sub + SPLIT, ...
// of each staged chunk and combine their sums by a fixed shuffle butterfly;
// U-bar partial sum per block.  The positions of bead j of all particles pass
// through shared memory in chunks.  Pairs: Gaussian g exp(-r^2/(2 s^2)), or
// Lennard-Jones 4 eps ((sig/r)^12 - (sig/r)^6) truncated and shifted at rc; in a
// periodic box (PBC) pair distances by minimum image.  MIXED: pair terms in
// float32, accumulated per lane in float32 and added to the float64 force.
template <bool MIXED, bool PBC, int SPLIT>
__device__ __forceinline__ double ext_force_body(const double *__restrict__ pos, double *__restrict__ F, int N,
                                                 int P, const PairParams &pp, int lb, int j,
                                                 typename std::conditional<MIXED, float4, Dbl4>::type *sr,
                                                 double *red, unsigned long long *T63s) {
  using R = typename std::conditional<MIXED, float, double>::type;
  using R4 = typename std::conditional<MIXED, float4, Dbl4>::type;
  constexpr int PARTICLES = EXT_THREADS / SPLIT;
  const int sub = threadIdx.x % SPLIT;
  const int l = lb * PARTICLES + threadIdx.x / SPLIT;
  const bool valid = l < N;
  double rx = 0, ry = 0, rz = 0;
  if (valid) {
    const double *r = pos + ((size_t)l * P + j) * 3;
    rx = r[0]; ry = r[1]; rz = r[2];
  }
  // mixed: float32 positions and constants from integer-pipe conversions
  // and host-formed copies, so that no per-thread float64 work remains but the
  // three force accumulations
  R px, py, pz, a, L, invL, sig2, rc2;
  if constexpr (MIXED) {
    px = f32_of_f64(rx); py = f32_of_f64(ry); pz = f32_of_f64(rz);
    a = pp.fa; L = pp.fL; invL = pp.finvL; sig2 = pp.fsig2; rc2 = pp.frc2;
  } else {
    px = rx; py = ry; pz = rz;
    a = -0.5 * pp.inv_s2; L = pp.L; invL = pp.invL; sig2 = pp.sig2; rc2 = pp.rc2;
  }
  if (!MIXED) pairg::table_init(T63s);  // float64: the integer-pipe power of two (read after the first barrier)
  auto img = [&](R d) -> R {
    if constexpr (PBC) return d - L * (MIXED ? (R)rintf((float)(d * invL)) : (R)rint((double)(d * invL)));
    else return d;
  };
  R fx = 0, fy = 0, fz = 0, u = 0;
  int nin = 0;  // Lennard-Jones pairs inside the cutoff (each carries the shift)
  if (pp.pair != BPIMD_PAIR_NONE) {
    for (int base = 0; base < N; base += EXT_CHUNK) {
      const int cnt = min(EXT_CHUNK, N - base);
      __syncthreads();
      for (int q = threadIdx.x; q < cnt; q += EXT_THREADS) {
        const double *r = pos + ((size_t)(base + q) * P + j) * 3;
        R4 t;
        if constexpr (MIXED) { t.x = f32_of_f64(r[0]); t.y = f32_of_f64(r[1]); t.z = f32_of_f64(r[2]); }
        else { t.x = r[0]; t.y = r[1]; t.z = r[2]; }
        t.w = (R)0;
        sr[q] = t;
      }
      __syncthreads();
      if (valid && pp.pair == BPIMD_PAIR_GAUSSIAN) {
#pragma unroll 4
        for (int q = sub; q < cnt; q += SPLIT) {
          const R4 t = sr[q];
          const R dx = img(px - t.x), dy = img(py - t.y), dz = img(pz - t.z);
          const R d2 = dx * dx + dy * dy + dz * dz;
          R e;
          if constexpr (MIXED) e = __expf(a * d2);
          else e = pow2_value(pow2fx::pow2neg_dd((double)d2, pp.g2c, T63s));  // exactly 1 at d = 0
          fx += e * dx; fy += e * dy; fz += e * dz;
          u += e;
        }
      } else if (valid) {  // Lennard-Jones: force over 24 eps, energy over 4 eps
#pragma unroll 4
        for (int q = sub; q < cnt; q += SPLIT) {
          const R4 t = sr[q];
          const R dx = img(px - t.x), dy = img(py - t.y), dz = img(pz - t.z);
          const R r2 = dx * dx + dy * dy + dz * dz;
          if (r2 > (R)0 && r2 < rc2) {
            const R s2 = sig2 / r2, s6 = s2 * s2 * s2;
            const R c = (2 * s6 * s6 - s6) / r2;
            fx += c * dx; fy += c * dy; fz += c * dz;
            u += s6 * s6 - s6;
            ++nin;
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 1; o < SPLIT; o <<= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
    u += __shfl_xor_sync(0xffffffffu, u, o);
    nin += __shfl_xor_sync(0xffffffffu, nin, o);
  }
  if constexpr (MIXED) {
    float ulf = 0.0f;
    if (valid && sub == 0) {
      if (pp.pair == BPIMD_PAIR_GAUSSIAN) u -= 1.0f;  // the self term (d = 0, e = 1) carries no force
      double *f = F + ((size_t)l * P + j) * 3;
      f[0] += f64_of_f32(pp.finv_P * (pp.ffs * fx - pp.fkt * px));
      f[1] += f64_of_f32(pp.finv_P * (pp.ffs * fy - pp.fkt * py));
      f[2] += f64_of_f32(pp.finv_P * (pp.ffs * fz - pp.fkt * pz));
      const float up = pp.pair == BPIMD_PAIR_GAUSSIAN ? pp.fup * u : pp.fup * u - pp.fush * (float)nin;
      ulf = pp.finv_P * (up + 0.5f * pp.fkt * (px * px + py * py + pz * pz));
    }
    return block_sum_f(ulf, red);
  }
  double ul = 0.0;
  if (valid && sub == 0) {
    if (pp.pair == BPIMD_PAIR_GAUSSIAN) u -= (R)1;  // the self term (d = 0, e = 1) carries no force
    double *f = F + ((size_t)l * P + j) * 3;
    const double fs = pp.pair == BPIMD_PAIR_GAUSSIAN ? pp.ga * pp.inv_s2 : 24.0 * pp.eps;
    f[0] += pp.inv_P * (fs * (double)fx - pp.kt * rx);
    f[1] += pp.inv_P * (fs * (double)fy - pp.kt * ry);
    f[2] += pp.inv_P * (fs * (double)fz - pp.kt * rz);
    const double up = pp.pair == BPIMD_PAIR_GAUSSIAN ? 0.5 * pp.ga * (double)u
                                                    : 0.5 * (4.0 * pp.eps * (double)u - pp.ushift * nin);
    ul = pp.inv_P * (up + 0.5 * pp.kt * (rx * rx + ry * ry + rz * rz));
  }
  return block_sum(ul, red);
}

template <bool MIXED, bool PBC>
__global__ void __launch_bounds__(EXT_THREADS) ext_force_kernel(const double *__restrict__ pos, double *__restrict__ F,
                                                                int N, int P, PairParams pp, double *ubar_part) {
  using R4 = typename std::conditional<MIXED, float4, Dbl4>::type;
  __shared__ R4 sr[EXT_CHUNK];
  __shared__ double red[EXT_THREADS / 32];
  __shared__ unsigned long long T63s[256];  // float64: the table of the integer-pipe power of two
  const double s = ext_force_body<MIXED, PBC, EXT_SPLIT>(pos, F, N, P, pp, blockIdx.x, blockIdx.y, sr, red, T63s);
  if (threadIdx.x == 0) ubar_part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// ----------------------------------------------------------- replica batches
// Replica r of a batch occupies elements [off[r], off[r] + 3 N_r P_r) of the
// packed arrays; the replica of element e by binary search over off.
__device__ __forceinline__ int replica_of(const long long *__restrict__ off, int R, long long e) {
  int lo = 0, hi = R - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// B A O A over every replica of a batch: as md_baoa_kernel, with the
// thermostat amplitude c2 of each element's replica (its own temperature).
template <bool MIXED>
__global__ void __launch_bounds__(MD_THREADS) md_baoa_batched(double *__restrict__ x, double *__restrict__ v,
                                                              const double *__restrict__ F, long long n,
                                                              double half_dt_over_m, double half_dt, double c1,
                                                              const double *__restrict__ c2r,
                                                              const long long *__restrict__ off, int R, uint32_t k0,
                                                              uint32_t k1, const unsigned long long *__restrict__ step) {
  const unsigned long long s = *step;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; 4 * g < n;
       g += (long long)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)g, (uint32_t)s, (uint32_t)(s >> 32), 0u};
    philox4x32_10(c, k0, k1);
    double z[4];
    box_muller<MIXED>(c, z);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long e = 4 * g + i;
      if (e < n) {
        const double c2 = __ldg(c2r + replica_of(off, R, e));
        double vi = v[e] + half_dt_over_m * F[e];  // B
        double xi = x[e] + half_dt * vi;           // A
        vi = c1 * vi + c2 * z[i];                  // O
        x[e] = xi + half_dt * vi;                  // A
        v[e] = vi;
      }
    }
  }
}

// Trap and pair forces of every replica: entry k of tab is (replica,
// particle block, bead index); the trap frequency and pair parameters are
// shared, 1/P_r is the replica's.  SPLIT lanes per particle, 256 / SPLIT
// particles per block (the batch's pair tile, bpimd_batch_set_pair_tile).
template <bool MIXED, int SPLIT>
__global__ void __launch_bounds__(EXT_THREADS) ext_force_batched(const double *__restrict__ pos,
                                                                 double *__restrict__ F,
                                                                 const Workspace *__restrict__ ws,
                                                                 const long long *__restrict__ off,
                                                                 const int4 *__restrict__ tab, int ntab, PairParams pp,
                                                                 double *ubar_part) {
  using R4 = typename std::conditional<MIXED, float4, Dbl4>::type;
  __shared__ R4 sr[EXT_CHUNK];
  __shared__ double red[EXT_THREADS / 32];
  __shared__ unsigned long long T63s[256];
  for (int k = blockIdx.x; k < ntab; k += gridDim.x) {
    const int4 e = tab[k];
    const int N = ws[e.x].N, P = ws[e.x].P;
    PairParams q = pp;
    q.inv_P = ws[e.x].inv_P;
    q.finv_P = f32_of_f64(q.inv_P);
    const double s = ext_force_body<MIXED, false, SPLIT>(pos + off[e.x], F + off[e.x], N, P, q, e.y, e.z, sr, red, T63s);
    if (threadIdx.x == 0) ubar_part[k] = s;
    __syncthreads();  // sr is reused by the next entry
  }
}

// energies[4 r + 0..3] of replica r (one block each): V_B, U-bar, kinetic,
// primitive estimator, from the partial sums of the last force pass.
__global__ void __launch_bounds__(MD_THREADS) energies_batched(const Workspace *__restrict__ ws,
                                                               const long long *__restrict__ off,
                                                               const double *__restrict__ VBr,
                                                               const double *__restrict__ ubar_part,
                                                               const int *__restrict__ ext_first,
                                                               const double *__restrict__ spring_part,
                                                               const int *__restrict__ blk_first,
                                                               const double *__restrict__ v, double half_m,
                                                               double *energies) {
  __shared__ double red[MD_THREADS / 32];
  const int r = blockIdx.x;
  const Workspace &w = ws[r];
  double sp = 0.0, ub = 0.0, ke = 0.0;
  for (int q = blk_first[r] + threadIdx.x; q < blk_first[r + 1]; q += blockDim.x) sp += spring_part[q];
  for (int l = threadIdx.x; l < w.N; l += blockDim.x) {
    sp += w.Eint[l];
    if (l + 1 < w.N) sp += direct_link_prob(w, l) * w.link[l];
  }
  for (int q = ext_first[r] + threadIdx.x; q < ext_first[r + 1]; q += blockDim.x) ub += ubar_part[q];
  const long long n = 3LL * w.N * w.P;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) ke += v[off[r] + e] * v[off[r] + e];
  sp = block_sum(sp, red);
  ub = block_sum(ub, red);
  ke = block_sum(ke, red);
  if (threadIdx.x == 0) {
    double *en = energies + 4 * (size_t)r;
    en[0] = VBr[r];
    en[1] = ub;
    en[2] = half_m * ke;
    en[3] = 1.5 * (double)w.N * (double)w.P / w.beta - sp + ub;
    for (int i = 0; i < 4; ++i)
      if (!isfinite(en[i])) atomicOr(w.status, ST_NONFINITE);
  }
}

__global__ void __launch_bounds__(MD_THREADS) ke_kernel(const double *__restrict__ v, long long n, double half_m,
                                                        double *ke_part) {
  __shared__ double red[MD_THREADS / 32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    acc += v[e] * v[e];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) ke_part[blockIdx.x] = half_m * s;
}

// energies[0..3] = V_B, U-bar, kinetic, primitive estimator 3NP/(2 beta) - <springs> + U-bar,
// with <springs> = sum_l E_int + sum Pr[l -> u<=l] (1/2)k d^2 + sum Pr[l -> l+1] link_l.
__global__ void __launch_bounds__(MD_THREADS) energies_kernel(Workspace w, const double *VB, const double *ubar_part,
                                                              int n_ubar, const double *ke_part, int n_ke,
                                                              const double *spring_part, double *energies) {
  __shared__ double red[MD_THREADS / 32];
  double sp = 0.0, ub = 0.0, ke = 0.0;
  for (int q = threadIdx.x; q < w.NB; q += blockDim.x) sp += spring_part[q];
  for (int l = threadIdx.x; l < w.N; l += blockDim.x) {
    sp += w.Eint[l];
    if (l + 1 < w.N) sp += direct_link_prob(w, l) * w.link[l];
  }
  for (int q = threadIdx.x; q < n_ubar; q += blockDim.x) ub += ubar_part[q];
  for (int q = threadIdx.x; q < n_ke; q += blockDim.x) ke += ke_part[q];
  sp = block_sum(sp, red);
  ub = block_sum(ub, red);
  ke = block_sum(ke, red);
  if (threadIdx.x == 0) {
    energies[0] = *VB;
    energies[1] = ub;
    energies[2] = ke;
    energies[3] = 1.5 * (double)w.N * (double)w.P / w.beta - sp + ub;
    for (int i = 0; i < 4; ++i)
      if (!isfinite(energies[i])) atomicOr(w.status, ST_NONFINITE);
  }
}

struct MDParams {
  long long n;
  double half_dt_over_m, half_dt, c1, c2;
  PairParams pp;
  int cell_nc;  // > 0: Lennard-Jones by cell lists with cell_nc^3 cells per bead index
  uint32_t k0, k1;
};

int md_params(const bpimd_config &c, MDParams &p) {
  if (!(c.dt > 0.0) || !std::isfinite(c.dt) || !(c.gamma >= 0.0) || !std::isfinite(c.gamma)) return BPIMD_ERR_ARG;
  if (!(c.kT_bead >= 0.0) || !std::isfinite(c.kT_bead) || !(c.omega0 >= 0.0) || !std::isfinite(c.omega0))
    return BPIMD_ERR_ARG;
  if (c.pair_type != BPIMD_PAIR_NONE && c.pair_type != BPIMD_PAIR_GAUSSIAN && c.pair_type != BPIMD_PAIR_LJ)
    return BPIMD_ERR_ARG;
  if (c.pair_type != BPIMD_PAIR_NONE &&
      (!std::isfinite(c.pair_a) || !(c.pair_b > 0.0) || !std::isfinite(c.pair_b)))
    return BPIMD_ERR_ARG;
  const double L = c.box_L;
  if (c.pair_type == BPIMD_PAIR_LJ) {
    // a cutoff is required; in a box it may not exceed half the side (minimum image)
    if (!(c.pair_rc > 0.0) || !std::isfinite(c.pair_rc)) return BPIMD_ERR_ARG;
    if (L > 0.0 && c.pair_rc > 0.5 * L) return BPIMD_ERR_ARG;
  }
  const double kT = c.kT_bead > 0.0 ? c.kT_bead : 1.0 / c.beta;
  p.n = (long long)c.N * c.P * 3;
  p.half_dt_over_m = 0.5 * c.dt / c.m;
  p.half_dt = 0.5 * c.dt;
  p.c1 = std::exp(-c.gamma * c.dt);
  p.c2 = std::sqrt((1.0 - p.c1 * p.c1) * kT / c.m);
  PairParams &q = p.pp;
  q = PairParams{};
  q.pair = c.pair_type;
  q.inv_P = 1.0 / c.P;
  q.kt = c.m * c.omega0 * c.omega0;
  if (c.pair_type == BPIMD_PAIR_GAUSSIAN) {
    q.ga = c.pair_a;
    q.inv_s2 = 1.0 / (c.pair_b * c.pair_b);
    q.g2c = 0.5 * q.inv_s2 * 1.4426950408889634;  // log2(e) / (2 s^2)
  }
  if (c.pair_type == BPIMD_PAIR_LJ) {
    q.eps = c.pair_a;
    q.sig2 = c.pair_b * c.pair_b;
    q.rc2 = c.pair_rc * c.pair_rc;
    const double sr2 = q.sig2 / q.rc2, sr6 = sr2 * sr2 * sr2;
    q.ushift = 4.0 * c.pair_a * (sr6 * sr6 - sr6);
  }
  q.L = L > 0.0 ? L : 0.0;
  q.invL = L > 0.0 ? 1.0 / L : 0.0;
  q.Lscale = (float)(q.L / 4294967296.0);
  q.pbc = L > 0.0 ? 1 : 0;
  q.fa = (float)(-0.5 * q.inv_s2);
  q.ffs = (float)(c.pair_type == BPIMD_PAIR_GAUSSIAN ? q.ga * q.inv_s2 : 24.0 * q.eps);
  q.fup = (float)(c.pair_type == BPIMD_PAIR_GAUSSIAN ? 0.5 * q.ga : 2.0 * q.eps);
  q.fkt = (float)q.kt;
  q.fL = (float)q.L;
  q.finvL = (float)q.invL;
  q.fsig2 = (float)q.sig2;
  q.frc2 = (float)q.rc2;
  q.fush = (float)(0.5 * q.ushift);
  q.finv_P = (float)q.inv_P;
  p.cell_nc = 0;
  if (c.pair_type == BPIMD_PAIR_LJ && L > 0.0) {
    const int nc = (int)std::floor(L / c.pair_rc);
    if (nc >= 3 && (long long)nc * nc * nc * c.P <= (1LL << 26)) p.cell_nc = nc;
  }
  p.k0 = (uint32_t)c.seed;
  p.k1 = (uint32_t)(c.seed >> 32);
  return BPIMD_OK;
}

int grid_for(long long work, int threads) {
  const long long b = (work + threads - 1) / threads;
  const long long cap = (long long)sm_count() * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// F(pos) = exchange force (Algorithm 1) + physical force, U-bar partials.
int total_force(bpimd_ctx *ctx, const MDParams &p, const double *pos) {
  MDState &md = ctx->md;
  int rc = evaluate(ctx, pos, md.VB, md.F);
  if (rc != BPIMD_OK) return rc;
  if (p.cell_nc > 0)
    return cell_list_forces(pos, md.F, ctx->cfg.N, ctx->cfg.P, p.pp, ctx->w.bead32, md.cells, md.ubar_part,
                            ctx->stream) == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
  const dim3 grid((ctx->cfg.N + EXT_PARTICLES - 1) / EXT_PARTICLES, ctx->cfg.P);
  const int N = ctx->cfg.N, P = ctx->cfg.P;
  if (ctx->w.bead32) {
    if (p.pp.pbc) ext_force_kernel<true, true><<<grid, EXT_THREADS, 0, ctx->stream>>>(pos, md.F, N, P, p.pp, md.ubar_part);
    else ext_force_kernel<true, false><<<grid, EXT_THREADS, 0, ctx->stream>>>(pos, md.F, N, P, p.pp, md.ubar_part);
  } else {
    if (p.pp.pbc) ext_force_kernel<false, true><<<grid, EXT_THREADS, 0, ctx->stream>>>(pos, md.F, N, P, p.pp, md.ubar_part);
    else ext_force_kernel<false, false><<<grid, EXT_THREADS, 0, ctx->stream>>>(pos, md.F, N, P, p.pp, md.ubar_part);
  }
  return cudaGetLastError() == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
}

// Enqueue one step (B A O A, force, B) on the context stream.
int enqueue_step(bpimd_ctx *ctx, const MDParams &p, double *pos, double *vel) {
  MDState &md = ctx->md;
  cudaStream_t s = ctx->stream;
  const int g4 = grid_for((p.n + 3) / 4, MD_THREADS), g1 = grid_for(p.n, MD_THREADS);
  if (ctx->w.bead32)
    md_baoa_kernel<true><<<g4, MD_THREADS, 0, s>>>(pos, vel, md.F, p.n, p.half_dt_over_m, p.half_dt, p.c1, p.c2,
                                                   p.k0, p.k1, md.step);
  else
    md_baoa_kernel<false><<<g4, MD_THREADS, 0, s>>>(pos, vel, md.F, p.n, p.half_dt_over_m, p.half_dt, p.c1, p.c2,
                                                    p.k0, p.k1, md.step);
  if (cudaGetLastError() != cudaSuccess) return BPIMD_ERR_CUDA;
  int rc = total_force(ctx, p, pos);
  if (rc != BPIMD_OK) return rc;
  md_kick_kernel<<<g1, MD_THREADS, 0, s>>>(vel, md.F, p.n, p.half_dt_over_m, md.step);
  return cudaGetLastError() == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
}

int md_alloc(bpimd_ctx *ctx, const MDParams &p) {
  MDState &md = ctx->md;
  if (p.cell_nc > 0) {
    const size_t bytes = cell_list_bytes(ctx->cfg.N, ctx->cfg.P, p.cell_nc, ctx->w.bead32);
    if (cudaMalloc(&md.cell_block, bytes) != cudaSuccess) {
      cudaGetLastError();
      return BPIMD_ERR_NOMEM;
    }
    cell_list_layout(md.cells, (char *)md.cell_block, ctx->cfg.N, ctx->cfg.P, p.cell_nc, ctx->w.bead32);
  }
  const size_t n = (size_t)ctx->cfg.N * ctx->cfg.P * 3;
  md.ext_blocks = p.cell_nc > 0 ? cell_list_partials(ctx->cfg.N, ctx->cfg.P)
                                 : ((ctx->cfg.N + EXT_PARTICLES - 1) / EXT_PARTICLES) * ctx->cfg.P;
  md.ke_blocks = grid_for((long long)n, MD_THREADS);
  md.spring_blocks = ctx->w.NB;
  if (cudaMalloc(&md.F, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&md.VB, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&md.ubar_part, sizeof(double) * md.ext_blocks) != cudaSuccess ||
      cudaMalloc(&md.ke_part, sizeof(double) * md.ke_blocks) != cudaSuccess ||
      cudaMalloc(&md.spring_part, sizeof(double) * md.spring_blocks) != cudaSuccess ||
      cudaMalloc(&md.step, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    md_free(&md);
    return BPIMD_ERR_NOMEM;
  }
  if (cudaMemsetAsync(md.step, 0, sizeof(unsigned long long), ctx->stream) != cudaSuccess) return BPIMD_ERR_CUDA;
  md.ready = true;
  return BPIMD_OK;
}

}  // namespace

void md_init(MDState *md) { *md = MDState{}; }

void md_free(MDState *md) {
  cudaFree(md->VBr);
  cudaFree(md->c2r);
  cudaFree(md->ext_tab);
  cudaFree(md->ext_first);
  cudaFree(md->blk_first);
  if (md->exec) cudaGraphExecDestroy(md->exec);
  if (md->graph) cudaGraphDestroy(md->graph);
  cudaFree(md->F);
  cudaFree(md->VB);
  cudaFree(md->ubar_part);
  cudaFree(md->ke_part);
  cudaFree(md->spring_part);
  cudaFree(md->step);
  cudaFree(md->cell_block);
  *md = MDState{};
}

int md_run(bpimd_ctx *ctx, double *pos, double *vel, int32_t nsteps, double *energies) {
  MDParams p;
  int rc = md_params(ctx->cfg, p);
  if (rc != BPIMD_OK) return rc;
  MDState &md = ctx->md;
  if (!md.ready && (rc = md_alloc(ctx, p)) != BPIMD_OK) return rc;
  // stage profiling is not recorded inside MD steps
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;
  // the caller may have moved the positions since the last call
  rc = total_force(ctx, p, pos);
  // capture one step into a graph (not possible on the legacy default stream)
  const bool use_graph = ctx->stream != nullptr && nsteps > 1;
  if (rc == BPIMD_OK && use_graph && (!md.exec || md.g_pos != pos || md.g_vel != vel)) {
    if (md.exec) { cudaGraphExecDestroy(md.exec); md.exec = nullptr; }
    if (md.graph) { cudaGraphDestroy(md.graph); md.graph = nullptr; }
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = BPIMD_ERR_CUDA;
    } else {
      const int rc_step = enqueue_step(ctx, p, pos, vel);
      const cudaError_t e = cudaStreamEndCapture(ctx->stream, &md.graph);
      if (rc_step != BPIMD_OK || e != cudaSuccess ||
          cudaGraphInstantiate(&md.exec, md.graph, 0) != cudaSuccess) {
        cudaGetLastError();
        rc = BPIMD_ERR_CUDA;
      } else {
        md.g_pos = pos;
        md.g_vel = vel;
      }
    }
  }
  for (int32_t s = 0; s < nsteps && rc == BPIMD_OK; ++s) {
    if (use_graph) rc = cudaGraphLaunch(md.exec, ctx->stream) == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
    else rc = enqueue_step(ctx, p, pos, vel);
  }
  if (rc == BPIMD_OK) md.steps_taken += (uint64_t)nsteps;
  if (rc == BPIMD_OK && energies) {
    cudaStream_t s = ctx->stream;
    const int g1 = md.ke_blocks;
    ke_kernel<<<g1, MD_THREADS, 0, s>>>(vel, p.n, 0.5 * ctx->cfg.m, md.ke_part);
    if (cudaGetLastError() != cudaSuccess || launch_spring_expectation(ctx->w, md.spring_part, s) != cudaSuccess)
      rc = BPIMD_ERR_CUDA;
    if (rc == BPIMD_OK) {
      energies_kernel<<<1, MD_THREADS, 0, s>>>(ctx->w, md.VB, md.ubar_part, md.ext_blocks, md.ke_part, g1,
                                              md.spring_part, energies);
      if (cudaGetLastError() != cudaSuccess) rc = BPIMD_ERR_CUDA;
    }
  }
  ctx->prof_on = prof;
  return rc;
}

// ----------------------------------------------------------- replica batches
// bpimd_step on a batch context: every replica advances by the same BAOAB
// steps (shared dt, gamma, trap, Gaussian pair potential and seed; each
// replica thermostatted at its own kT = 1/beta_r unless cfg.kT_bead > 0).
// One step is: the batched B A O A kernel, the three evaluation launches of
// the batch (plus one per replica above 4096 particles), the batched trap and
// pair forces, and the closing B -- captured once into a CUDA graph bound to
// the caller's buffers and replayed.  Thermostat noise: Philox4x32-10 with the
// element index of the packed arrays as the counter.
namespace {

// (replica, particle block, bead index) table of the batched pair forces for
// `lanes` lanes per particle (256 / lanes particles per block)
void pair_table(const bpimd_ctx *ctx, int lanes, std::vector<int4> &tab, std::vector<int> &ext_first) {
  const int R = ctx->R, pb = EXT_THREADS / lanes;
  tab.clear();
  ext_first.assign(R + 1, 0);
  for (int r = 0; r < R; ++r) {
    const Workspace &w = ctx->h_ws[r];
    ext_first[r] = (int)tab.size();
    for (int j = 0; j < w.P; ++j)
      for (int lb = 0; lb * pb < w.N; ++lb) tab.push_back(make_int4(r, lb, j, 0));
  }
  ext_first[R] = (int)tab.size();
}

int md_alloc_batched(bpimd_ctx *ctx, const MDParams &p) {
  MDState &md = ctx->md;
  const int R = ctx->R;
  const size_t n = (size_t)ctx->total_elems;
  std::vector<int4> tab;
  std::vector<int> ext_first, blk_first(R + 1);
  pair_table(ctx, 8, tab, ext_first);  // the largest table: its size is the capacity
  md.ext_cap = (int)tab.size();
  pair_table(ctx, ctx->pair_lanes, tab, ext_first);
  int blk = 0;
  for (int r = 0; r < R; ++r) {
    blk_first[r] = blk;
    blk += ctx->h_ws[r].NB;
  }
  blk_first[R] = blk;
  md.n_ext = (int)tab.size();
  md.spring_blocks = ctx->n_blk_tab;
  md.ke_blocks = 0;
  md.ext_blocks = md.n_ext;
  std::vector<double> c2(R);
  for (int r = 0; r < R; ++r) {
    const double kT = ctx->cfg.kT_bead > 0.0 ? ctx->cfg.kT_bead : 1.0 / ctx->h_ws[r].beta;
    c2[r] = std::sqrt((1.0 - p.c1 * p.c1) * kT / ctx->cfg.m);
  }
  if (cudaMalloc(&md.F, sizeof(double) * n) != cudaSuccess || cudaMalloc(&md.VBr, sizeof(double) * R) != cudaSuccess ||
      cudaMalloc(&md.c2r, sizeof(double) * R) != cudaSuccess ||
      cudaMalloc(&md.ext_tab, sizeof(int4) * md.ext_cap) != cudaSuccess ||
      cudaMalloc(&md.ext_first, sizeof(int) * (R + 1)) != cudaSuccess ||
      cudaMalloc(&md.blk_first, sizeof(int) * (R + 1)) != cudaSuccess ||
      cudaMalloc(&md.ubar_part, sizeof(double) * md.ext_cap) != cudaSuccess ||
      cudaMalloc(&md.spring_part, sizeof(double) * md.spring_blocks) != cudaSuccess ||
      cudaMalloc(&md.step, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    md_free(&md);
    return BPIMD_ERR_NOMEM;
  }
  cudaStream_t s = ctx->stream;
  if (cudaMemcpyAsync(md.c2r, c2.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(md.ext_tab, tab.data(), sizeof(int4) * md.n_ext, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(md.ext_first, ext_first.data(), sizeof(int) * (R + 1), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(md.blk_first, blk_first.data(), sizeof(int) * (R + 1), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(md.step, 0, sizeof(unsigned long long), s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)  // the host tables go out of scope
    return BPIMD_ERR_CUDA;
  md.ready = true;
  return BPIMD_OK;
}

int total_force_batched(bpimd_ctx *ctx, const MDParams &p, const double *pos) {
  MDState &md = ctx->md;
  int rc = evaluate_batched(ctx, pos, md.VBr, md.F);
  if (rc != BPIMD_OK) return rc;
  const int grid = md.n_ext < sm_count() * 8 ? md.n_ext : sm_count() * 8;
  auto go = [&](auto kernel) {
    kernel<<<grid, EXT_THREADS, 0, ctx->stream>>>(pos, md.F, ctx->d_ws, ctx->d_off, md.ext_tab, md.n_ext, p.pp,
                                                  md.ubar_part);
  };
  const bool m = ctx->w.bead32;
  switch (ctx->pair_lanes) {
    case 2: m ? go(ext_force_batched<true, 2>) : go(ext_force_batched<false, 2>); break;
    case 8: m ? go(ext_force_batched<true, 8>) : go(ext_force_batched<false, 8>); break;
    default: m ? go(ext_force_batched<true, 4>) : go(ext_force_batched<false, 4>); break;
  }
  return cudaGetLastError() == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
}

int enqueue_step_batched(bpimd_ctx *ctx, const MDParams &p, double *pos, double *vel) {
  MDState &md = ctx->md;
  cudaStream_t s = ctx->stream;
  const long long n = ctx->total_elems;
  const int g4 = grid_for((n + 3) / 4, MD_THREADS), g1 = grid_for(n, MD_THREADS);
  if (ctx->w.bead32)
    md_baoa_batched<true><<<g4, MD_THREADS, 0, s>>>(pos, vel, md.F, n, p.half_dt_over_m, p.half_dt, p.c1, md.c2r,
                                                    ctx->d_off, ctx->R, p.k0, p.k1, md.step);
  else
    md_baoa_batched<false><<<g4, MD_THREADS, 0, s>>>(pos, vel, md.F, n, p.half_dt_over_m, p.half_dt, p.c1, md.c2r,
                                                     ctx->d_off, ctx->R, p.k0, p.k1, md.step);
  if (cudaGetLastError() != cudaSuccess) return BPIMD_ERR_CUDA;
  int rc = total_force_batched(ctx, p, pos);
  if (rc != BPIMD_OK) return rc;
  md_kick_kernel<<<g1, MD_THREADS, 0, s>>>(vel, md.F, n, p.half_dt_over_m, md.step);
  return cudaGetLastError() == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
}

}  // namespace

// A new pair tile for a batch: with MD state allocated, rebuild the pair-force
// table (within the capacity of the 8-lane table) and drop the captured step,
// which is recaptured by the next bpimd_step; forces, velocities and the
// thermostat counter are kept, so a trajectory goes on unchanged.
int md_set_pair_tile(bpimd_ctx *ctx, int lanes) {
  MDState &md = ctx->md;
  if (md.ready && lanes != ctx->pair_lanes) {
    std::vector<int4> tab;
    std::vector<int> ext_first;
    pair_table(ctx, lanes, tab, ext_first);
    if ((int)tab.size() > md.ext_cap) return BPIMD_ERR_STATE;
    cudaStream_t s = ctx->stream;
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpyAsync(md.ext_tab, tab.data(), sizeof(int4) * tab.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(md.ext_first, ext_first.data(), sizeof(int) * ext_first.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)  // the host tables go out of scope
      return BPIMD_ERR_CUDA;
    md.n_ext = (int)tab.size();
    md.ext_blocks = md.n_ext;
    if (md.exec) { cudaGraphExecDestroy(md.exec); md.exec = nullptr; }
    if (md.graph) { cudaGraphDestroy(md.graph); md.graph = nullptr; }
    md.g_pos = md.g_vel = nullptr;
  }
  ctx->pair_lanes = lanes;
  return BPIMD_OK;
}

int md_run_batched(bpimd_ctx *ctx, double *pos, double *vel, int32_t nsteps, double *energies) {
  bpimd_config c = ctx->cfg;
  if (c.pair_type == BPIMD_PAIR_LJ) return BPIMD_ERR_ARG;  // batches have no periodic box
  c.N = 1;
  c.P = 2;
  c.beta = 1.0;  // md_params' kT only fills p.c2, which batches replace per replica
  MDParams p;
  int rc = md_params(c, p);
  if (rc != BPIMD_OK) return rc;
  p.n = ctx->total_elems;
  MDState &md = ctx->md;
  if (!md.ready && (rc = md_alloc_batched(ctx, p)) != BPIMD_OK) return rc;
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;
  rc = total_force_batched(ctx, p, pos);
  const bool use_graph = ctx->stream != nullptr && nsteps > 1;
  if (rc == BPIMD_OK && use_graph && (!md.exec || md.g_pos != pos || md.g_vel != vel)) {
    if (md.exec) { cudaGraphExecDestroy(md.exec); md.exec = nullptr; }
    if (md.graph) { cudaGraphDestroy(md.graph); md.graph = nullptr; }
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = BPIMD_ERR_CUDA;
    } else {
      const int rc_step = enqueue_step_batched(ctx, p, pos, vel);
      const cudaError_t e = cudaStreamEndCapture(ctx->stream, &md.graph);
      if (rc_step != BPIMD_OK || e != cudaSuccess || cudaGraphInstantiate(&md.exec, md.graph, 0) != cudaSuccess) {
        cudaGetLastError();
        rc = BPIMD_ERR_CUDA;
      } else {
        md.g_pos = pos;
        md.g_vel = vel;
      }
    }
  }
  for (int32_t k = 0; k < nsteps && rc == BPIMD_OK; ++k) {
    if (use_graph) rc = cudaGraphLaunch(md.exec, ctx->stream) == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
    else rc = enqueue_step_batched(ctx, p, pos, vel);
  }
  if (rc == BPIMD_OK) md.steps_taken += (uint64_t)nsteps;
  if (rc == BPIMD_OK && energies) {
    cudaStream_t s = ctx->stream;
    if (launch_spring_expectation_batched(ctx->d_ws, ctx->d_blk_tab, ctx->n_blk_tab, md.spring_part, s) !=
        cudaSuccess)
      rc = BPIMD_ERR_CUDA;
    if (rc == BPIMD_OK) {
      energies_batched<<<ctx->R, MD_THREADS, 0, s>>>(ctx->d_ws, ctx->d_off, md.VBr, md.ubar_part, md.ext_first,
                                                     md.spring_part, md.blk_first, vel, 0.5 * ctx->cfg.m, energies);
      if (cudaGetLastError() != cudaSuccess) rc = BPIMD_ERR_CUDA;
    }
  }
  ctx->prof_on = prof;
  return rc;
}

}  // namespace bpimd
