/*
 * md_oracle.c -- plain CPU oracle for the molecular-dynamics step that drives
 * the bosonic ring polymers (Feldman & Hirshberg, "Quadratic Scaling Bosonic
 * Path Integral Molecular Dynamics").
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference arm of bench.py.  It shares no code with the CUDA
 * library.
 *
 * The paper samples exp(-beta (V^{[1,N]} + U-bar)) (Eq.
 * int-of-sum-all-permutations, spring frequency w_P = sqrt(P)/(beta hbar) of
 * Eq. eperm, U-bar = (1/P) sum_j U(r_1^j..r_N^j)) by molecular dynamics with a
 * thermostat; it does not state its integrator or thermostat (Methods,
 * "Numerical Validation").  This file follows the reading used by the library:
 * Cartesian BAOAB Langevin splitting (half kick B, half drift A, exact
 * Ornstein-Uhlenbeck velocity update O, half drift A, force, half kick B) at
 * temperature kT = 1/beta, with bead mass m, and
 *   U = sum_l (1/2) m w0^2 |r_l|^2                 (isotropic harmonic trap)
 *     + sum_{l<l'} g exp(-|r_l - r_l'|^2 / (2 s^2))  (Gaussian repulsion)
 *     or sum_{l<l'} 4 eps ((sig/r)^12 - (sig/r)^6), truncated and shifted at rc
 *                                                     (Lennard-Jones, liquid helium)
 * acting between beads of equal index j, scaled by 1/P; in a periodic box of
 * side L every pair and every spring uses the minimum image.
 *
 * The thermostat noise comes from the counter-based generator Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11), implemented here from its published definition; the library
 * implements the same generator on its own.  Element e = 4 g + i (i = 0..3) of
 * the velocity array at step s draws its normal from block
 * Philox(counter = (g, s mod 2^32, s div 2^32, 0), key = (seed mod 2^32,
 * seed div 2^32)): the four 32-bit words x_i give uniforms
 * u_i = (x_i + 1/2) 2^-32 and, by the Box-Muller transform,
 *   z_0 = sqrt(-2 ln u_0) cos(2 pi u_1),  z_1 = sqrt(-2 ln u_0) sin(2 pi u_1),
 *   z_2 = sqrt(-2 ln u_2) cos(2 pi u_3),  z_3 = sqrt(-2 ln u_2) sin(2 pi u_3).
 */
#include "bpimd_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORA_LONG_DOUBLE
#define SQRT sqrtl
#define EXPR expl
#else
#define SQRT sqrt
#define EXPR exp
#endif

/* ----------------------------------------------------------- Philox4x32-10 */
/* One round: two 32x32 -> 64-bit multiplications by the published constants,
 * then the word permutation and the key xor; the key is bumped by the
 * published Weyl increments between rounds. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Index of the first element in the counter mapping: 0 for a single system;
 * a replica of a packed batch takes the counters of its elements' positions
 * in the packed array (set by ora_set_noise_offset, reset by ora_md_run). */
static uint64_t ora_noise_e0 = 0;
void ora_set_noise_offset(uint64_t e0) { ora_noise_e0 = e0; }

/* Standard normals for elements 0..n-1 of step `step` (mapping in the header);
 * element i takes word (e0 + i) mod 4 of the block with counter (e0 + i) div 4. */
void ora_thermostat_normals(uint64_t seed, uint64_t step, int64_t n, double *z) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two_pi = 6.283185307179586476925286766559;
  const uint64_t e0 = ora_noise_e0;
  for (uint64_t g = e0 / 4; 4 * g < e0 + (uint64_t)n; ++g) {
    const uint32_t ctr[4] = {(uint32_t)g, (uint32_t)step, (uint32_t)(step >> 32), 0u};
    uint32_t x[4];
    ora_philox4x32_10(ctr, key, x);
    double u[4];
    for (int i = 0; i < 4; ++i) u[i] = ((double)x[i] + 0.5) * 2.3283064365386962890625e-10;
    const double ra = sqrt(-2.0 * log(u[0])), rb = sqrt(-2.0 * log(u[2]));
    const double zz[4] = {ra * cos(two_pi * u[1]), ra * sin(two_pi * u[1]),
                          rb * cos(two_pi * u[3]), rb * sin(two_pi * u[3])};
    for (int i = 0; i < 4; ++i) {
      const uint64_t e = 4 * g + (uint64_t)i;
      if (e >= e0 && e < e0 + (uint64_t)n) z[e - e0] = zz[i];
    }
  }
}

#ifdef ORA_LONG_DOUBLE
#define RINTR rintl
#else
#define RINTR rint
#endif

/* Physical forces -grad U-bar added to F, and U-bar in *ubar.
 * pair_type: 0 none, 1 Gaussian (a = g, b = s), 2 Lennard-Jones
 * 4 a ((b/r)^12 - (b/r)^6) truncated at rc and shifted to 0 there (rc <= 0:
 * no cutoff).  L > 0: periodic cubic box, pair distances by minimum image. */
int ora_external_forces(int N, int P, ora_real m, ora_real omega0, int pair_type, ora_real pa,
                        ora_real pb, ora_real rc, ora_real L, const ora_real *pos, ora_real *F,
                        ora_real *ubar) {
  if (N < 1 || P < 2 || !pos || !F) return -1;
  if (pair_type != 0 && pair_type != 1 && pair_type != 2) return -1;
  ora_real ushift = 0.0;
  if (pair_type == 2 && rc > 0.0) {
    const ora_real sr6 = (pb / rc) * (pb / rc) * (pb / rc) * (pb / rc) * (pb / rc) * (pb / rc);
    ushift = 4.0 * pa * (sr6 * sr6 - sr6);
  }
  ora_real U = 0.0;
  const ora_real invP = (ora_real)1.0 / (ora_real)P;
  for (int l = 1; l <= N; ++l)
    for (int j = 1; j <= P; ++j) {
      const ora_real *r = &pos[((size_t)(l - 1) * P + (j - 1)) * 3];
      ora_real *f = &F[((size_t)(l - 1) * P + (j - 1)) * 3];
      if (omega0 > 0.0) {
        const ora_real kt = m * omega0 * omega0;
        U += invP * 0.5 * kt * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        for (int d = 0; d < 3; ++d) f[d] -= invP * kt * r[d];
      }
      if (pair_type == 1) {
        for (int lp = 1; lp <= N; ++lp) {
          if (lp == l) continue;
          const ora_real *q = &pos[((size_t)(lp - 1) * P + (j - 1)) * 3];
          ora_real dx = r[0] - q[0], dy = r[1] - q[1], dz = r[2] - q[2];
          if (L > 0.0) {
            dx -= L * RINTR(dx / L);
            dy -= L * RINTR(dy / L);
            dz -= L * RINTR(dz / L);
          }
          const ora_real e = pa * EXPR(-(dx * dx + dy * dy + dz * dz) / (2.0 * pb * pb));
          if (lp > l) U += invP * e;
          /* -d/dr_l of g exp(-d^2/(2 s^2)) = g exp(..) d / s^2 */
          f[0] += invP * e * dx / (pb * pb);
          f[1] += invP * e * dy / (pb * pb);
          f[2] += invP * e * dz / (pb * pb);
        }
      }
      if (pair_type == 2) {
        for (int lp = 1; lp <= N; ++lp) {
          if (lp == l) continue;
          const ora_real *q = &pos[((size_t)(lp - 1) * P + (j - 1)) * 3];
          ora_real dx = r[0] - q[0], dy = r[1] - q[1], dz = r[2] - q[2];
          if (L > 0.0) {
            dx -= L * RINTR(dx / L);
            dy -= L * RINTR(dy / L);
            dz -= L * RINTR(dz / L);
          }
          const ora_real r2 = dx * dx + dy * dy + dz * dz;
          if (rc > 0.0 && r2 >= rc * rc) continue;
          const ora_real s2 = pb * pb / r2, s6 = s2 * s2 * s2;
          if (lp > l) U += invP * (4.0 * pa * (s6 * s6 - s6) - ushift);
          /* -dU/dr_l = 24 eps (2 (s/r)^12 - (s/r)^6) d / r^2 */
          const ora_real c = invP * 24.0 * pa * (2.0 * s6 * s6 - s6) / r2;
          f[0] += c * dx;
          f[1] += c * dy;
          f[2] += c * dz;
        }
      }
    }
  if (ubar) *ubar = U;
  return 0;
}

/* Total force: -grad (V^{[1,N]} + U-bar) by Algorithm 1 plus the physical part. */
static int total_force(int N, int P, ora_real m, ora_real omega_P, ora_real beta, ora_real omega0,
                       int pair_type, ora_real pa, ora_real pb, ora_real pc, ora_real L, const ora_real *x,
                       ora_real *F, ora_real *VB, ora_real *ubar, ora_real *M) {
  ora_set_box(L);
  int rc = ora_fast_pimdb(N, P, m, omega_P, beta, x, VB, F, NULL, NULL, M);
  if (!rc) rc = ora_external_forces(N, P, m, omega0, pair_type, pa, pb, pc, L, x, F, ubar);
  return rc;
}

/* nsteps BAOAB steps from (pos, vel) in place; step indices step0..step0+nsteps-1
 * select the thermostat noise.  kT <= 0 means 1/beta.  energies (may be NULL)
 * receives, after the last step: [0] V^{[1,N]}, [1] U-bar, [2] sum (1/2) m v^2,
 * [3] the primitive energy estimator 3NP/(2 beta) - <E^{G[sigma]}> + U-bar. */
int ora_md_run(int N, int P, ora_real m, ora_real omega_P, ora_real beta, ora_real dt, ora_real gamma,
               ora_real kT, ora_real omega0, int pair_type, ora_real pa, ora_real pb, ora_real pc,
               ora_real L, uint64_t seed, uint64_t step0, int nsteps, ora_real *pos, ora_real *vel,
               ora_real *energies) {
  if (N < 1 || P < 2 || nsteps < 0 || !pos || !vel || !(dt > 0.0) || gamma < 0.0) return -1;
  if (!(kT > 0.0)) kT = 1.0 / beta;
  const size_t n = (size_t)N * P * 3;
  ora_real *F = (ora_real *)malloc(sizeof(ora_real) * n);
  ora_real *M = (ora_real *)malloc(sizeof(ora_real) * (size_t)N * N);
  double *z = (double *)malloc(sizeof(double) * n);
  int rc = (F && M && z) ? 0 : -1;
  ora_real VB = 0.0, ubar = 0.0;
  /* O step: v <- c1 v + c2 z, the exact Ornstein-Uhlenbeck update over dt */
  const ora_real c1 = EXPR(-gamma * dt);
  const ora_real c2 = SQRT((1.0 - c1 * c1) * kT / m);
  if (!rc) rc = total_force(N, P, m, omega_P, beta, omega0, pair_type, pa, pb, pc, L, pos, F, &VB, &ubar, M);
  for (int s = 0; s < nsteps && !rc; ++s) {
    ora_thermostat_normals(seed, step0 + (uint64_t)s, (int64_t)n, z);
    for (size_t i = 0; i < n; ++i) {
      vel[i] += 0.5 * dt * F[i] / m;     /* B */
      pos[i] += 0.5 * dt * vel[i];       /* A */
      vel[i] = c1 * vel[i] + c2 * z[i];  /* O */
      pos[i] += 0.5 * dt * vel[i];       /* A */
    }
    rc = total_force(N, P, m, omega_P, beta, omega0, pair_type, pa, pb, pc, L, pos, F, &VB, &ubar, M);
    for (size_t i = 0; i < n && !rc; ++i) vel[i] += 0.5 * dt * F[i] / m; /* B */
  }
  if (!rc && energies) {
    ora_real ke = 0.0, spring = 0.0;
    for (size_t i = 0; i < n; ++i) ke += 0.5 * m * vel[i] * vel[i];
    rc = ora_expected_spring_energy(N, P, m, omega_P, pos, M, &spring);
    energies[0] = VB;
    energies[1] = ubar;
    energies[2] = ke;
    energies[3] = 3.0 * N * P / (2.0 * beta) - spring + ubar;
  }
  ora_set_box(0.0);
  ora_noise_e0 = 0;
  free(F);
  free(M);
  free(z);
  return rc;
}
