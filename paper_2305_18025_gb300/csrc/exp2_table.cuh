// Float64 powers of two by Tang's table-driven method (P. T. P. Tang, ACM
// TOMS 15(2), 1989), for kernels whose float64 pipe is the scarce unit: about
// 10 float64 instructions per power.
//   y = k/64 + r with k = round(64 y), |r| <= 1/128;
//   2^y = 2^(k >> 6) * T[k & 63] * 2^r with T[j] = 2^(j/64) (a 64-entry
//   shared-memory table, one CUDA exp2 per entry, exp2_table_init);
//   2^r = 1 + sum_{i=1..5} (r ln 2)^i / i!, truncation below 3.6e-17 relative;
//   2^(k >> 6) is applied to the exponent bits (an integer add).
// The rounding of 64 y uses the 1.5 * 2^52 constant: t = 64 y + 1.5 * 2^52
// holds round(64 y) in its low word while |64 y| < 2^31.
#pragma once

namespace bpimd {

// Fill T[0..63] = 2^(j/64) (threads 0..63 of the block; the caller's next
// __syncthreads publishes it).
__device__ __forceinline__ void exp2_table_init(double *T) {
  if (threadIdx.x < 64) T[threadIdx.x] = exp2((double)threadIdx.x * 0.015625);
}

// T[k & 63] * 2^r for y = k/64 + r: the power without its factor 2^(k >> 6),
// which is returned in k.  Exact (1, k = 0) at y = 0.
__device__ __forceinline__ double exp2_table_part(double y, const double *T, int &k) {
  constexpr double C1 = 0.6931471805599453, C2 = 0.24022650695910072, C3 = 0.05550410866482158,
                   C4 = 0.009618129107628477, C5 = 0.0013333558146428443;  // (ln 2)^i / i!
  constexpr double MAGIC = 6755399441055744.0;                            // 1.5 * 2^52
  const double t = fma(y, 64.0, MAGIC);
  k = __double2loint(t);
  const double r = fma(t - MAGIC, -0.015625, y);
  const double p = fma(r, fma(r, fma(r, fma(r, fma(r, C5, C4), C3), C2), C1), 1.0);
  return T[k & 63] * p;
}

// 2^y for y <= 0, clamped to 2^-1000 below (a normal number; nothing the
// callers sum can see the difference).
__device__ __forceinline__ double exp2_table(double y, const double *T) {
  int k;
  const double v = exp2_table_part(fmax(y, -1000.0), T, k);
  return __longlong_as_double(__double_as_longlong(v) + ((long long)(k >> 6) << 52));
}

}  // namespace bpimd
