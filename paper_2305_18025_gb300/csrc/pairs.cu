// Lennard-Jones forces of the MD step in a periodic box by cell lists
// (O(N P) per step instead of O(N^2 P)).
//
// Per bead index j the box is cut into nc^3 cells of side L/nc >= rc, so all
// partners within rc of a bead lie in its own and the 26 neighbouring cells
// (nc >= 3 keeps those 27 cells distinct).  Per step:
//   bin     each bead's cell and its wrapped coordinates (MIXED: 32-bit
//           fixed-point fractions of L, whose wrap-around difference is the
//           minimum image exactly; float64: coordinates in [0, L));
//   scan    cell starts (exclusive prefix sum of the counts, one CTA);
//   scatter bead indices into their cells;
//   sort    each cell's indices ascending, so that every force is summed in
//           a fixed order (results do not depend on the order of atomics);
//   gather  coordinates into cell order (one load per candidate pair later);
//   force   one thread per slot of the cell-ordered list: the 27 cells in a
//           fixed order, pairs inside rc, force and energy (MIXED: float32
//           pair terms).
#include <type_traits>

#include "bpimd_internal.cuh"
#include "pairs.cuh"

namespace bpimd {
namespace {

constexpr int CL_THREADS = 128;  // force kernel: bead slots per block
constexpr int SCAN_THREADS = 1024;

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

template <bool MIXED>
__global__ void __launch_bounds__(256) cl_bin(const double *__restrict__ pos, int N, int P, int nc, double invL,
                                              int *__restrict__ cellof, void *__restrict__ crd,
                                              int *__restrict__ count) {
  const long long nb = (long long)N * P;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(b % P);
    const double *r = pos + 3 * b;
    double f[3];
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double t = r[d] * invL;
      f[d] = t - floor(t);  // fraction of the box in [0, 1)
      c[d] = min((int)(f[d] * nc), nc - 1);
    }
    const int cid = ((j * nc + c[2]) * nc + c[1]) * nc + c[0];
    cellof[b] = cid;
    if (MIXED) {
      uint4 u;
      u.x = (unsigned)fmin(f[0] * 4294967296.0, 4294967295.0);
      u.y = (unsigned)fmin(f[1] * 4294967296.0, 4294967295.0);
      u.z = (unsigned)fmin(f[2] * 4294967296.0, 4294967295.0);
      u.w = 0u;
      ((uint4 *)crd)[b] = u;
    } else {
      const double L = 1.0 / invL;
      ((double4 *)crd)[b] = make_double4(f[0] * L, f[1] * L, f[2] * L, 0.0);
    }
    atomicAdd(count + cid, 1);
  }
}

// exclusive prefix sum of count into start (one CTA)
__global__ void __launch_bounds__(SCAN_THREADS) cl_scan(const int *__restrict__ count, int *__restrict__ start,
                                                        int n) {
  __shared__ int warp_tot[SCAN_THREADS / 32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n; base += SCAN_THREADS) {
    const int i = base + threadIdx.x;
    const int x = i < n ? count[i] : 0;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const int incl = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + v;
    if (i < n) start[i] = incl - x;
    __syncthreads();
    if (threadIdx.x == SCAN_THREADS - 1) carry = incl;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) cl_scatter(const int *__restrict__ cellof, int N, int P,
                                                  const int *__restrict__ start, int *__restrict__ fill,
                                                  int *__restrict__ list) {
  const long long nb = (long long)N * P;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
    const int cid = cellof[b];
    list[start[cid] + atomicAdd(fill + cid, 1)] = (int)b;
  }
}

// each cell's bead indices ascending (insertion sort; cells hold a few beads;
// one cell holds one bead index j, so this orders by particle)
__global__ void __launch_bounds__(256) cl_sort(const int *__restrict__ start, const int *__restrict__ count,
                                               int ncells, int *__restrict__ list) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    int *a = list + start[c];
    const int n = count[c];
    for (int i = 1; i < n; ++i) {
      const int key = a[i];
      int k = i - 1;
      while (k >= 0 && a[k] > key) {
        a[k + 1] = a[k];
        --k;
      }
      a[k + 1] = key;
    }
  }
}

// coordinates in cell order: sorted[slot] = crd[list[slot]]
template <bool MIXED>
__global__ void __launch_bounds__(256) cl_gather(const int *__restrict__ list, long long nb,
                                                 const void *__restrict__ crd, void *__restrict__ sorted) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nb; q += (long long)gridDim.x * blockDim.x) {
    if (MIXED) ((uint4 *)sorted)[q] = ((const uint4 *)crd)[list[q]];
    else ((double4 *)sorted)[q] = ((const double4 *)crd)[list[q]];
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(CL_THREADS) cl_force(long long nb, int P, PairParams pp, int nc,
                                                       const int *__restrict__ cellof, const void *__restrict__ sorted,
                                                       const int *__restrict__ start, const int *__restrict__ count,
                                                       const int *__restrict__ list, const double *__restrict__ pos,
                                                       double *__restrict__ F, double *ubar_part) {
  // one thread per slot of the cell-ordered bead list: neighbouring threads
  // work on the same or adjacent cells, whose coordinates they share in cache
  using R = typename std::conditional<MIXED, float, double>::type;
  __shared__ double red[CL_THREADS / 32];
  const long long slot = blockIdx.x * (long long)CL_THREADS + threadIdx.x;
  const bool valid = slot < nb;
  R fx = 0, fy = 0, fz = 0, u = 0;
  int nin = 0;
  double rx = 0, ry = 0, rz = 0;
  int b = 0;
  if (valid) {
    b = list[slot];
    const int j = b % P;
    const double *r = pos + 3 * (long long)b;
    rx = r[0]; ry = r[1]; rz = r[2];
    const int cell = cellof[b] - j * nc * nc * nc;
    const int cx = cell % nc, cy = (cell / nc) % nc, cz = cell / (nc * nc);
    const R sig2 = (R)pp.sig2, rc2 = (R)pp.rc2;
    uint4 ui = make_uint4(0, 0, 0, 0);
    double4 di = make_double4(0, 0, 0, 0);
    if (MIXED) ui = ((const uint4 *)sorted)[slot];
    else di = ((const double4 *)sorted)[slot];
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int nx = (cx + dx + nc) % nc, ny = (cy + dy + nc) % nc, nz = (cz + dz + nc) % nc;
          const int nid = ((j * nc + nz) * nc + ny) * nc + nx;
          const int s0 = start[nid], n = count[nid];
          for (int q = s0; q < s0 + n; ++q) {
            if (q == slot) continue;
            R ex, ey, ez;
            if (MIXED) {
              const uint4 uj = ((const uint4 *)sorted)[q];
              ex = (R)fixdiff(ui.x, uj.x, pp.Lscale);
              ey = (R)fixdiff(ui.y, uj.y, pp.Lscale);
              ez = (R)fixdiff(ui.z, uj.z, pp.Lscale);
            } else {
              const double4 dj = ((const double4 *)sorted)[q];
              ex = (R)(di.x - dj.x); ey = (R)(di.y - dj.y); ez = (R)(di.z - dj.z);
              ex -= (R)(pp.L * rint((double)ex * pp.invL));
              ey -= (R)(pp.L * rint((double)ey * pp.invL));
              ez -= (R)(pp.L * rint((double)ez * pp.invL));
            }
            const R r2 = ex * ex + ey * ey + ez * ez;
            if (r2 > (R)0 && r2 < rc2) {
              const R s2 = sig2 / r2, s6 = s2 * s2 * s2;
              const R c = (2 * s6 * s6 - s6) / r2;
              fx += c * ex; fy += c * ey; fz += c * ez;
              u += s6 * s6 - s6;
              ++nin;
            }
          }
        }
  }
  double ul = 0.0;
  if (valid) {
    double *f = F + 3 * (long long)b;
    const double fs = 24.0 * pp.eps;
    f[0] += pp.inv_P * (fs * (double)fx - pp.kt * rx);
    f[1] += pp.inv_P * (fs * (double)fy - pp.kt * ry);
    f[2] += pp.inv_P * (fs * (double)fz - pp.kt * rz);
    ul = pp.inv_P * (0.5 * (4.0 * pp.eps * (double)u - pp.ushift * nin) + 0.5 * pp.kt * (rx * rx + ry * ry + rz * rz));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ul += __shfl_xor_sync(0xffffffffu, ul, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ul;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < CL_THREADS / 32; ++q) t += red[q];
    ubar_part[blockIdx.x] = t;
  }
}

}  // namespace

int cell_list_partials(int N, int P) { return ((N + CL_THREADS - 1) / CL_THREADS) * P; }

size_t cell_list_bytes(int N, int P, int nc, bool mixed) {
  const size_t nb = (size_t)N * P, ncells = (size_t)P * nc * nc * nc;
  return a256(sizeof(int) * nb) + 2 * a256((mixed ? 16 : 32) * nb) + 3 * a256(sizeof(int) * ncells) +
         a256(sizeof(int) * nb);
}

void cell_list_layout(CellList &cl, char *base, int N, int P, int nc, bool mixed) {
  const size_t nb = (size_t)N * P, ncells = (size_t)P * nc * nc * nc;
  cl.nc = nc;
  cl.ncells = (int)ncells;
  size_t off = 0;
  cl.cellof = (int *)(base + off); off += a256(sizeof(int) * nb);
  cl.crd = (void *)(base + off); off += a256((mixed ? 16 : 32) * nb);
  cl.sorted = (void *)(base + off); off += a256((mixed ? 16 : 32) * nb);
  cl.count = (int *)(base + off); off += a256(sizeof(int) * ncells);
  cl.fill = (int *)(base + off); off += a256(sizeof(int) * ncells);
  cl.start = (int *)(base + off); off += a256(sizeof(int) * ncells);
  cl.list = (int *)(base + off);
}

cudaError_t cell_list_forces(const double *pos, double *F, int N, int P, const PairParams &pp, bool mixed,
                             const CellList &cl, double *ubar_part, cudaStream_t s) {
  const long long nb = (long long)N * P;
  const long long want = (nb + 255) / 256, cap = (long long)sm_count() * 16;
  const int g = (int)(want < cap ? want : cap);
  cudaError_t e = cudaMemsetAsync(cl.count, 0, sizeof(int) * cl.ncells, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cl.fill, 0, sizeof(int) * cl.ncells, s);
  if (e != cudaSuccess) return e;
  if (mixed) cl_bin<true><<<g, 256, 0, s>>>(pos, N, P, cl.nc, pp.invL, cl.cellof, cl.crd, cl.count);
  else cl_bin<false><<<g, 256, 0, s>>>(pos, N, P, cl.nc, pp.invL, cl.cellof, cl.crd, cl.count);
  cl_scan<<<1, SCAN_THREADS, 0, s>>>(cl.count, cl.start, cl.ncells);
  cl_scatter<<<g, 256, 0, s>>>(cl.cellof, N, P, cl.start, cl.fill, cl.list);
  cl_sort<<<(cl.ncells + 255) / 256, 256, 0, s>>>(cl.start, cl.count, cl.ncells, cl.list);
  if (mixed) cl_gather<true><<<g, 256, 0, s>>>(cl.list, nb, cl.crd, cl.sorted);
  else cl_gather<false><<<g, 256, 0, s>>>(cl.list, nb, cl.crd, cl.sorted);
  const int blocks = cell_list_partials(N, P);  // one U-bar partial per block
  if (mixed)
    cl_force<true><<<blocks, CL_THREADS, 0, s>>>(nb, P, pp, cl.nc, cl.cellof, cl.sorted, cl.start, cl.count, cl.list,
                                                 pos, F, ubar_part);
  else
    cl_force<false><<<blocks, CL_THREADS, 0, s>>>(nb, P, pp, cl.nc, cl.cellof, cl.sorted, cl.start, cl.count, cl.list,
                                                  pos, F, ubar_part);
  return cudaGetLastError();
}

}  // namespace bpimd
