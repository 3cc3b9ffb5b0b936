/*
 * bpimd_oracle.h -- plain FP64 CPU oracle for the bosonic exchange potential
 * V^{[1,N]} and its bead forces (Feldman & Hirshberg, "Quadratic Scaling
 * Bosonic Path Integral Molecular Dynamics").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and the CPU-baseline /
 * reference arm of bench.py use it.  It shares no code with the CUDA library.
 *
 * Conventions (all functions):
 *   pos  : [N][P][3] row-major ora_real values; bead j (1-based) of particle l (1-based)
 *          is pos[((l-1)*P + (j-1))*3 + d].
 *   m, omega_P, beta : mass, ring-polymer spring frequency, inverse temperature;
 *          the spring prefactor is (1/2) m omega_P^2 (Eq. eperm).
 *   E    : N*N values, E[(u-1)*N + (v-1)] = E^{[u,v]} for u <= v (cycle energy
 *          of the ring through particles u..v); entries with u > v unused.
 *   V    : N+1 values, V[v] = V^{[1,v]}, V[0] = 0.
 *   W    : N+1 values, W[u-1] = V^{[u,N]} for u = 1..N+1, so W[N] = 0.
 *   M    : N*N values, M[(l-1)*N + (l'-1)] = Pr[l -> l'], the probability that
 *          bead P of particle l is joined to bead 1 of particle l'.
 *   F    : [N][P][3] forces -grad V^{[1,N]}.
 * Return value of int functions: 0 on success, -1 on invalid arguments.
 */
#ifndef BPIMD_ORACLE_H
#define BPIMD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Floating-point type of every array and parameter.  The default build is
 * float64.  Compiling with -DORA_LONG_DOUBLE gives the same routines in long
 * double (64-bit mantissa on x86-64, 113-bit on aarch64); that build serves as
 * a higher-precision referee in the tests, where float64 rounding of the
 * oracle itself would otherwise be compared with the tolerances. */
#ifdef ORA_LONG_DOUBLE
typedef long double ora_real;
#else
typedef double ora_real;
#endif

/* Periodic cubic box of side L for every following call (L <= 0: open
 * boundaries, the default).  In a box every spring -- interior, link and
 * closing -- joins the minimum image of its two beads; positions need not be
 * wrapped.  Process-wide setting (the oracle is single threaded). */
void ora_set_box(ora_real L);

/* Shift choice for the log-sum-exp steps (Methods, "Numerical Stability"). */
#define ORA_SHIFT_MIN_ALL 0   /* Eq. full-elong: min over all terms of the step   */
#define ORA_SHIFT_TWO_TERM 1  /* Eq. original-elong: min of two designated terms  */

/* Eq. e-interior: E_int^{(l)} for every particle. */
int ora_interior_energies(int N, int P, ora_real m, ora_real omega_P,
                          const ora_real *pos, ora_real *Eint);

/* Algorithm 1 cycle-energy stage: base case Eq. e-recurrence-base and the
 * O(1) step Eq. e-recurrence-step, v ascending, u descending. */
int ora_cycle_energies(int N, int P, ora_real m, ora_real omega_P,
                       const ora_real *pos, ora_real *E);

/* Eq. Ek: the direct double sum over the ring through u..v (O(P N^3) total). */
int ora_cycle_energies_direct(int N, int P, ora_real m, ora_real omega_P,
                              const ora_real *pos, ora_real *E);

/* Eq. our-forward-potential-recurrence with the shifted form of the
 * Numerical Stability section.  Writes V[0..N]. */
int ora_forward_potentials(int N, ora_real beta, const ora_real *E, int shift_mode,
                           ora_real *V);

/* Eq. backward-potential-recursion (Theorem backward-recurrence), shifted.
 * Writes W[0..N] (W[u-1] = V^{[u,N]}). */
int ora_backward_potentials(int N, ora_real beta, const ora_real *E, int shift_mode,
                            ora_real *W);

/* Definition backward-potential: the O(N^3) route to V^{[u,N]}. */
int ora_backward_potentials_definition(int N, ora_real beta, const ora_real *E,
                                       ora_real *W);

/* Eq. direct-link-probability and Eq. close-cycle-probability; zero for
 * l' > l + 1 (Lemma zero-connection-probability). */
int ora_connection_probabilities(int N, ora_real beta, const ora_real *E,
                                 const ora_real *V, const ora_real *W, ora_real *M);

/* Interior-bead forces (Eq. intermediate-bead-force) and exterior-bead forces
 * (Eq. force-on-1/P-sum-neighbors) with Algorithm 1's trimmed sum limits. */
int ora_forces(int N, int P, ora_real m, ora_real omega_P, const ora_real *pos,
               const ora_real *M, ora_real *F);

/* Algorithm 1 (Fast PIMD-B) end to end.  Returns 0/-1; *V_B = V^{[1,N]}.
 * Optional outputs (may be NULL): V (N+1), W (N+1), M (N*N). */
int ora_fast_pimdb(int N, int P, ora_real m, ora_real omega_P, ora_real beta,
                   const ora_real *pos, ora_real *V_B, ora_real *F,
                   ora_real *V, ora_real *W, ora_real *M);

/* Algorithm 2 (Original PIMD-B): O(P N^3) potential and per-bead force
 * recursion.  Returns 0/-1; *V_B = V^{[1,N]}. */
int ora_original_pimdb(int N, int P, ora_real m, ora_real omega_P, ora_real beta,
                       const ora_real *pos, ora_real *V_B, ora_real *F);

/* Spring part of the primitive energy estimator of the bosonic ring polymer:
 * sum_l E_int^{(l)} + sum_{l,l'} Pr[l->l'] (1/2) m omega_P^2 |r_l^P - r_l'^1|^2,
 * i.e. the expectation over representative permutations of E^{G[sigma]}. */
int ora_expected_spring_energy(int N, int P, ora_real m, ora_real omega_P,
                               const ora_real *pos, const ora_real *M, ora_real *out);

/* ------------------------------------------------ molecular dynamics (md_oracle.c) */
#include <stdint.h>

/* Philox4x32-10 block function (published definition, 10 rounds). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Thermostat normals for elements 0..n-1 of step `step` (float64 Box-Muller of
 * Philox4x32-10 words; mapping in md_oracle.c). */
void ora_thermostat_normals(uint64_t seed, uint64_t step, int64_t n, double *z);

/* Physical forces -grad U-bar added to F (harmonic trap of frequency omega0 if
 * omega0 > 0; pair_type 1: Gaussian g = pa, s = pb; 2: Lennard-Jones eps = pa,
 * sigma = pb, truncated and shifted at pc (pc <= 0: no cutoff); pairs between
 * equal-index beads, minimum image in a periodic box of side L > 0);
 * *ubar = U-bar (may be NULL). */
int ora_external_forces(int N, int P, ora_real m, ora_real omega0, int pair_type, ora_real pa,
                        ora_real pb, ora_real pc, ora_real L, const ora_real *pos, ora_real *F,
                        ora_real *ubar);

/* Element offset of the thermostat counters for the next ora_md_run (a
 * replica at element offset e0 of a packed batch); reset to 0 by it. */
void ora_set_noise_offset(uint64_t e0);

/* nsteps BAOAB Langevin steps in place (kT <= 0: 1/beta; L > 0: periodic box
 * for the springs and the pairs); energies (may be NULL): [0] V^{[1,N]},
 * [1] U-bar, [2] kinetic, [3] primitive estimator. */
int ora_md_run(int N, int P, ora_real m, ora_real omega_P, ora_real beta, ora_real dt, ora_real gamma,
               ora_real kT, ora_real omega0, int pair_type, ora_real pa, ora_real pb, ora_real pc,
               ora_real L, uint64_t seed, uint64_t step0, int nsteps, ora_real *pos, ora_real *vel,
               ora_real *energies);

#ifdef __cplusplus
}
#endif
#endif
