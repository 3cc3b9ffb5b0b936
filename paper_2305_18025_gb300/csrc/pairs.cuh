// Physical pair potential of the MD step: parameters and the cell-list path
// (internal; used by md.cu).
#pragma once
#include <cuda_runtime.h>

namespace bpimd {

// U = sum_l (1/2) kt |r_l|^2 + pairs between beads of equal index, all scaled by 1/P.
struct PairParams {
  int pair;              // BPIMD_PAIR_NONE / GAUSSIAN / LJ
  double inv_P, kt;      // 1/P, m w0^2 (trap)
  double ga, inv_s2;     // Gaussian g, 1/s^2
  double g2c;            // log2(e) / (2 s^2): the Gaussian is 2^(-g2c d^2)
  double eps, sig2, rc2; // Lennard-Jones eps, sigma^2, cutoff^2
  double ushift;         // LJ energy at the cutoff (subtracted per pair inside it)
  double L, invL;        // periodic box (L = 0: open)
  float Lscale;          // L / 2^32 (fixed-point differences)
  int pbc;               // L > 0 (integer test; float64 compares use the slow float64 pipe)
  // float32 copies for the mixed forms, formed on the host (a conversion in a
  // kernel runs on the narrow float64 pipe): -1/(2 s^2), the force factor
  // (g/s^2 or 24 eps), the energy factor (g/2 or 2 eps), kt, L, 1/L, sigma^2, rc^2
  float fa, ffs, fup, fkt, fL, finvL, fsig2, frc2;
  float fush, finv_P;    // ushift / 2, 1/P
};

// Cell lists per bead index: nc^3 cells of side L/nc >= rc in a periodic box.
struct CellList {
  int nc;            // cells per side (>= 3)
  int ncells;        // P nc^3
  int *cellof;       // [N*P] cell of bead (l, j), index l*P + j
  void *crd;         // [N*P] wrapped coordinates: uint4 fixed point (MIXED) or double4 (float64)
  void *sorted;      // [N*P] the same coordinates in cell order (slot q holds bead list[q])
  int *count, *fill, *start;  // [ncells]
  int *list;         // [N*P] bead indices l*P + j grouped by cell, ascending within a cell
};

// Bytes of the cell-list buffers for N particles, P beads, nc cells per side.
size_t cell_list_bytes(int N, int P, int nc, bool mixed);
// Number of U-bar partial sums cell_list_forces writes.
int cell_list_partials(int N, int P);
// Lay the buffers out from base (cudaMalloc'd, 256-byte aligned).
void cell_list_layout(CellList &cl, char *base, int N, int P, int nc, bool mixed);
// Bin, sort and evaluate Lennard-Jones (+ trap) forces added to F; U-bar
// partial sums per (particle block of 128, bead index), as the all-pairs kernel.
cudaError_t cell_list_forces(const double *pos, double *F, int N, int P, const PairParams &pp, bool mixed,
                             const CellList &cl, double *ubar_part, cudaStream_t s);

}  // namespace bpimd
