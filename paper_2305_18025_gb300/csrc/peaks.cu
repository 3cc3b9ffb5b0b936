// Throughput probes for the roofline figures of the benchmark: the float64
// FMA rate of the whole GPU (the unit that bounds the float64 stages) and the
// integer 32 x 32 -> 64-bit multiply-add rate (the unit of the integer-pipe
// recursions and pair factors).  Each thread runs eight independent chains,
// so the measured rate is the pipe's throughput, not one chain's latency.
#include "bpimd_internal.cuh"

namespace bpimd {
namespace {

constexpr int PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS) fp64_fma_probe(long long iters, double *sink) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  const double b = 0.999999, c = 1e-7;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.0) sink[blockIdx.x] = s;  // keeps the chains alive; never true for these inputs
}

__global__ void __launch_bounds__(PEAK_THREADS) int_mad_probe(long long iters, unsigned long long *sink) {
  unsigned long long a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 7919ull + k;
  const unsigned b = 2654435761u;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (unsigned long long)(unsigned)a[k] * b + (a[k] >> 32);
  }
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= a[k];
  if (s == 0x1234567ull) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace bpimd

extern "C" int bpimd_peak_probe(int32_t kind, int64_t iters, void *sink, void *cuda_stream, int64_t *ops) {
  using namespace bpimd;
  if ((kind != 0 && kind != 1) || iters < 1 || !sink || ((uintptr_t)sink & 7)) return BPIMD_ERR_ARG;
  const int blocks = sm_count() * 8;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (kind == 0) fp64_fma_probe<<<blocks, PEAK_THREADS, 0, s>>>(iters, (double *)sink);
  else int_mad_probe<<<blocks, PEAK_THREADS, 0, s>>>(iters, (unsigned long long *)sink);
  if (ops) *ops = (int64_t)blocks * PEAK_THREADS * 8 * iters;
  return cudaGetLastError() == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
}

// ------------------------------------------------ powers-of-two self-test
// The device's own powers of two on caller-given arguments, for tests that
// compare them with a reference exp2, both by the integer-pipe fixed-point
// method (pow2_fixed.cuh), x >= 0, the result as a double (0 below the normal
// range): method 0 = 2^(-x c) with the exact double x double product of the
// float64 MD Gaussian (pow2neg_dd, c = 1/2, so that the reference argument is
// exact too); method 1 = 2^(-x) as for the float64 pair factors (pow2neg).
#include "pow2_fixed.cuh"

namespace bpimd {
namespace {
__global__ void pow2_selftest_kernel(int method, const double *__restrict__ x, double *__restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const pow2fx::mexp g =
        method == 0 ? pow2fx::pow2neg_dd(x[i], 0.5, pow2fx::T63) : pow2fx::pow2neg(x[i], pow2fx::T63);
    out[i] = g.e < -1022 ? 0.0 : g.m * __longlong_as_double((long long)(g.e + 1023) << 52);
  }
}
}  // namespace
}  // namespace bpimd

extern "C" int bpimd_pow2_selftest(int32_t method, const double *x, double *out, int32_t n, void *cuda_stream) {
  using namespace bpimd;
  if ((method != 0 && method != 1) || n < 0 || (n > 0 && (!x || !out))) return BPIMD_ERR_ARG;
  if (n == 0) return BPIMD_OK;
  pow2_selftest_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, (cudaStream_t)cuda_stream>>>(
      method, x, out, n);
  return cudaGetLastError() == cudaSuccess ? BPIMD_OK : BPIMD_ERR_CUDA;
}
