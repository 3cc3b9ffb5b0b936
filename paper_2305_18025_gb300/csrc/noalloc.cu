// Allocation-free exchange evaluation.
//
// Some callers cannot allocate device memory when they need this computation:
// a host program whose memory manager owns every device allocation and forbids
// others, a simulation loop that may not call cudaMalloc/cudaFree because those
// calls can synchronise the whole device and stall other streams, or an
// embedding with a fixed memory budget set up front.  For them this entry point
// runs the same kernels as bpimd_exchange_energy_forces, but its scratch memory
// (pair factors, recursion state, force partial sums) lives in one file-scope
// __device__ array of fixed size, so no call allocates anything.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress and caches it for that
// device.  That first call should therefore come before any stream capture.
// Shared state: every call on a device uses the same array, which keeps the
// previous call's contents; each call clears the parts that must start at zero
// (the device status word and the tile counters) and rewrites the padding of
// the pair factors, which depends on N.  Two calls whose work overlaps on the GPU (for
// example on two different streams) race on the array and give wrong results.
#include <mutex>

#include "bpimd_internal.cuh"

namespace bpimd {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)2 << 20;  // 2 MiB per device
static_assert(BPIMD_NOALLOC_MAX_N >= 1, "maximum size must be positive");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES];  // device address of the array, per device

// Device address of the scratch array on the current device (set up once).
int noalloc_scratch(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return BPIMD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return BPIMD_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return BPIMD_OK;
}

bool positive_finite(double x) { return x > 0.0 && x < __builtin_huge_val(); }

}  // namespace
}  // namespace bpimd

extern "C" int bpimd_exchange_energy_forces_noalloc(const bpimd_config *cfg, const double *positions,
                                                    double *V_B, double *forces, void *cuda_stream) {
  using namespace bpimd;
  if (!cfg || !positions || !forces) return BPIMD_ERR_ARG;
  if ((((uintptr_t)positions) & 15) || (((uintptr_t)forces) & 15)) return BPIMD_ERR_ARG;
  if (V_B && (((uintptr_t)V_B) & 7)) return BPIMD_ERR_ARG;
  if (cfg->N < 1 || cfg->P < 2 || cfg->flags != 0) return BPIMD_ERR_ARG;
  if (!valid_precision(cfg->precision)) return BPIMD_ERR_ARG;
  if (!positive_finite(cfg->m) || !positive_finite(cfg->omega_P) || !positive_finite(cfg->beta))
    return BPIMD_ERR_ARG;
  if (cfg->N > BPIMD_NOALLOC_MAX_N || (long long)cfg->N * cfg->P > (1LL << 31) / 3) return BPIMD_ERR_SIZE;

  Workspace w{};
  w.N = cfg->N;
  w.P = cfg->P;
  w.NT = (w.N + TILE - 1) / TILE;
  w.NB = w.NT * (w.NT + 1) / 2;
  set_precision(w, cfg->precision);
  w.m = cfg->m;
  w.omega_P = cfg->omega_P;
  w.beta = cfg->beta;
  w.k = cfg->m * cfg->omega_P * cfg->omega_P;
  w.half_k = 0.5 * w.k;
  w.cx = w.beta * w.half_k * LOG2E;
  w.blocks = 1;
  if (!(cfg->box_L >= 0.0) || !(cfg->box_L < __builtin_huge_val())) return BPIMD_ERR_ARG;
  set_box(w, cfg->box_L);
  if (layout_workspace(w, nullptr) > NOALLOC_SCRATCH_BYTES) return BPIMD_ERR_SIZE;

  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the scratch array used is the current device's: a stream of another
  // device would run these kernels against the wrong device's array
  if (s != nullptr) {
    int cur = -1, sdev = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return BPIMD_ERR_CUDA;
    }
    if (sdev != cur) return BPIMD_ERR_ARG;
  }
  void *base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != BPIMD_OK) return rc;
  layout_workspace(w, (char *)base);

  if (cudaMemsetAsync(w.status, 0, sizeof(int), s) != cudaSuccess) return BPIMD_ERR_CUDA;
  // the tile counters of the probability pass start at zero (a previous call
  // with another N leaves its counters at zero, but at other offsets)
  if (cudaMemsetAsync(w.rowcnt, 0, sizeof(int) * w.NT, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (cudaMemsetAsync(w.colcnt, 0, sizeof(int) * w.NT, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_gmat_padding(w, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_prep(w, positions, forces, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_chains(w, V_B, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_prob_forces(w, positions, forces, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  return BPIMD_OK;
}
