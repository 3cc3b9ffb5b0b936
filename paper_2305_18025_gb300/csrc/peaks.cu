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
