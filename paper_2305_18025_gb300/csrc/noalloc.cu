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
// previous call's contents; this file clears the part that must start at zero
// (the device status word).  Two calls whose work overlaps on the GPU (for
// example on two different streams) race on the array and give wrong results.
#include <mutex>

#include "bpimd_internal.cuh"

namespace bpimd {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)1 << 20;  // 1 MiB per device
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

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// Lay the workspace out from `base` (nullptr: only measure).  Returns the bytes used.
size_t noalloc_layout(Workspace &w, char *base) {
  const size_t N = w.N, NB = w.NB, gelems = NB * TILE2;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    char *p = base ? base + off : nullptr;
    off += round256(bytes);
    return p;
  };
  w.R1 = (double *)take(sizeof(double) * 4 * N);
  w.RP = (double *)take(sizeof(double) * 4 * N);
  w.Eint = (double *)take(sizeof(double) * N);
  w.link = (double *)take(sizeof(double) * N);
  w.ccm = (double *)take(sizeof(double) * N);
  w.cce = (int *)take(sizeof(int) * N);
  w.icm = (double *)take(sizeof(double) * N);
  w.ice = (int *)take(sizeof(int) * N);
  w.C = (double *)take(sizeof(double) * (N + 1));
  w.gm = (void *)take((w.mixed ? sizeof(float) : sizeof(double)) * gelems);
  w.ge = (int *)take(sizeof(int) * gelems);
  w.gbm = (void *)take((w.mixed ? sizeof(float) : sizeof(double)) * gelems);
  w.gbe = (int *)take(sizeof(int) * gelems);
  w.yfm = (double *)take(sizeof(double) * (N + 1));
  w.yfe = (int *)take(sizeof(int) * (N + 1));
  w.ybm = (double *)take(sizeof(double) * (N + 1));
  w.ybe = (int *)take(sizeof(int) * (N + 1));
  w.scal = (double *)take(sizeof(double) * 4);
  w.scal_i = (int *)take(sizeof(int) * 4);
  w.rowpart = (double *)take(sizeof(double) * NB * TILE * 4);
  w.colpart = (double *)take(sizeof(double) * NB * TILE * 4);
  w.status = (int *)take(sizeof(int) * 4);
  return off;
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
  if (cfg->precision != BPIMD_FP64 && cfg->precision != BPIMD_MIXED) return BPIMD_ERR_ARG;
  if (!positive_finite(cfg->m) || !positive_finite(cfg->omega_P) || !positive_finite(cfg->beta))
    return BPIMD_ERR_ARG;
  if (cfg->N > BPIMD_NOALLOC_MAX_N || (long long)cfg->N * cfg->P > (1LL << 31) / 3) return BPIMD_ERR_SIZE;

  Workspace w{};
  w.N = cfg->N;
  w.P = cfg->P;
  w.NT = (w.N + TILE - 1) / TILE;
  w.NB = w.NT * (w.NT + 1) / 2;
  w.mixed = cfg->precision == BPIMD_MIXED;
  w.m = cfg->m;
  w.omega_P = cfg->omega_P;
  w.beta = cfg->beta;
  w.k = cfg->m * cfg->omega_P * cfg->omega_P;
  w.half_k = 0.5 * w.k;
  if (noalloc_layout(w, nullptr) > NOALLOC_SCRATCH_BYTES) return BPIMD_ERR_SIZE;

  void *base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != BPIMD_OK) return rc;
  noalloc_layout(w, (char *)base);

  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(w.status, 0, sizeof(int), s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_bead_pass(w, positions, forces, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_gmat(w, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_chains(w, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_scalars(w, V_B, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_prob_blocks(w, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  if (launch_force_finalize(w, positions, forces, s) != cudaSuccess) return BPIMD_ERR_CUDA;
  return BPIMD_OK;
}
