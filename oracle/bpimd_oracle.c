/*
 * bpimd_oracle.c -- plain, slow, FP64 CPU oracle for the bosonic exchange
 * potential and forces (Feldman & Hirshberg, "Quadratic Scaling Bosonic Path
 * Integral Molecular Dynamics").
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference arm of bench.py.  It shares no code with the CUDA
 * library and the CUDA library never calls it.
 *
 * Every loop follows the paper's 1-based notation: particles l, u, v in 1..N,
 * beads j in 1..P.  Nothing is blocked, fused or reordered beyond what the
 * cited equation or algorithm states.  Single threaded, -O2, no vector
 * intrinsics, so results are the same on x86-64 and aarch64 hosts.
 */
#include "bpimd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORA_LONG_DOUBLE
#define EXP expl
#define LOG logl
#define EXPM1 expm1l
#define INF_REAL HUGE_VALL
#else
#define EXP exp
#define LOG log
#define EXPM1 expm1
#define INF_REAL HUGE_VAL
#endif

/* bead j of particle l, coordinate d (1-based l, j; 0-based d) */
#define BEAD(pos, P, l, j) (&(pos)[((size_t)((l) - 1) * (size_t)(P) + (size_t)((j) - 1)) * 3])
#define EIDX(N, u, v) ((size_t)((u) - 1) * (size_t)(N) + (size_t)((v) - 1))

/* Periodic cubic box of side g_box (0: open boundaries), set by ora_set_box.
 * In a periodic box every spring joins the minimum image of its two beads
 * (the paper is silent on boundaries; this is the usual path-integral
 * convention for bulk liquids).  With g_box = 0 every expression below is the
 * plain open-boundary one, operation for operation. */
static ora_real g_box = 0.0;

void ora_set_box(ora_real L) { g_box = L > 0.0 ? L : 0.0; }

#ifdef ORA_LONG_DOUBLE
#define RINT rintl
#else
#define RINT rint
#endif

/* minimum image of one coordinate difference */
static ora_real mi1(ora_real d) { return g_box > 0.0 ? d - g_box * RINT(d / g_box) : d; }

/* 2 r - a - b, i.e. (r - a) + (r - b) with each spring taken as a minimum image */
static ora_real lap1(ora_real r, ora_real a, ora_real b) {
  return g_box > 0.0 ? mi1(r - a) + mi1(r - b) : 2.0 * r - a - b;
}

static ora_real sqdist(const ora_real *a, const ora_real *b) {
  ora_real dx = mi1(a[0] - b[0]), dy = mi1(a[1] - b[1]), dz = mi1(a[2] - b[2]);
  return dx * dx + dy * dy + dz * dz;
}

static int bad_args(int N, int P) { return N < 1 || P < 2; }

/* Eq. e-interior: E_int^{(l)} = (1/2) m w_P^2 sum_{j=1}^{P-1} (r_l^{j+1} - r_l^j)^2.
 * The spring from bead P is not part of it. */
int ora_interior_energies(int N, int P, ora_real m, ora_real omega_P,
                          const ora_real *pos, ora_real *Eint) {
  if (bad_args(N, P) || !pos || !Eint) return -1;
  const ora_real half_k = 0.5 * m * omega_P * omega_P;
  for (int l = 1; l <= N; ++l) {
    ora_real s = 0.0;
    for (int j = 1; j <= P - 1; ++j) s += sqdist(BEAD(pos, P, l, j + 1), BEAD(pos, P, l, j));
    Eint[l - 1] = half_k * s;
  }
  return 0;
}

/* Algorithm 1, cycle-energy stage.
 *   base: E^{[v,v]} = E_int^{(v)} + (1/2)k (r_v^P - r_v^1)^2       (Eq. e-recurrence-base)
 *   step: E^{[u,v]} = E^{[u+1,v]} - (1/2)k (r_v^P - r_{u+1}^1)^2
 *                     + (1/2)k (r_u^P - r_{u+1}^1)^2 + E_int^{(u)}
 *                     + (1/2)k (r_v^P - r_u^1)^2                 (Eq. e-recurrence-step)
 * with (1/2)k = (1/2) m w_P^2. */
int ora_cycle_energies(int N, int P, ora_real m, ora_real omega_P,
                       const ora_real *pos, ora_real *E) {
  if (bad_args(N, P) || !pos || !E) return -1;
  const ora_real half_k = 0.5 * m * omega_P * omega_P;
  ora_real *Eint = (ora_real *)malloc(sizeof(ora_real) * (size_t)N);
  if (!Eint) return -1;
  ora_interior_energies(N, P, m, omega_P, pos, Eint);
  for (int v = 1; v <= N; ++v) {
    E[EIDX(N, v, v)] = Eint[v - 1] + half_k * sqdist(BEAD(pos, P, v, P), BEAD(pos, P, v, 1));
    for (int u = v - 1; u >= 1; --u) {
      E[EIDX(N, u, v)] = E[EIDX(N, u + 1, v)]
                         - half_k * sqdist(BEAD(pos, P, v, P), BEAD(pos, P, u + 1, 1))
                         + half_k * sqdist(BEAD(pos, P, u, P), BEAD(pos, P, u + 1, 1))
                         + Eint[u - 1]
                         + half_k * sqdist(BEAD(pos, P, v, P), BEAD(pos, P, u, 1));
    }
  }
  free(Eint);
  return 0;
}

/* Eq. Ek with the ring through u..v: E^{[u,v]} = (1/2)k sum_{l=u}^{v} sum_{j=1}^{P}
 * (r_l^{j+1} - r_l^j)^2 where r_l^{P+1} = r_{l+1}^1, except r_v^{P+1} = r_u^1. */
int ora_cycle_energies_direct(int N, int P, ora_real m, ora_real omega_P,
                              const ora_real *pos, ora_real *E) {
  if (bad_args(N, P) || !pos || !E) return -1;
  const ora_real half_k = 0.5 * m * omega_P * omega_P;
  for (int v = 1; v <= N; ++v) {
    for (int u = 1; u <= v; ++u) {
      ora_real s = 0.0;
      for (int l = u; l <= v; ++l) {
        for (int j = 1; j <= P; ++j) {
          const ora_real *next;
          if (j < P) next = BEAD(pos, P, l, j + 1);
          else if (l < v) next = BEAD(pos, P, l + 1, 1);
          else next = BEAD(pos, P, u, 1);
          s += sqdist(next, BEAD(pos, P, l, j));
        }
      }
      E[EIDX(N, u, v)] = half_k * s;
    }
  }
  return 0;
}

/* Eq. our-forward-potential-recurrence, shifted as in the Numerical Stability
 * section:  V^{[1,v]} = Et - (1/beta) ln[(1/v) sum_{k=1}^{v}
 *                          EXP(-beta (V^{[1,v-k]} + E^{[v-k+1,v]} - Et))],
 * V^{[1,0]} = 0.  Et is Eq. full-elong (min over the v terms) or Eq.
 * original-elong (min of E^{[1,v]} and V^{[1,v-1]} + E^{[v,v]}). */
int ora_forward_potentials(int N, ora_real beta, const ora_real *E, int shift_mode,
                           ora_real *V) {
  if (N < 1 || !(beta > 0.0) || !E || !V) return -1;
  V[0] = 0.0;
  for (int v = 1; v <= N; ++v) {
    ora_real Et;
    if (shift_mode == ORA_SHIFT_TWO_TERM) {
      ora_real a = E[EIDX(N, 1, v)], b = V[v - 1] + E[EIDX(N, v, v)];
      Et = a < b ? a : b;
    } else {
      Et = INF_REAL;
      for (int k = 1; k <= v; ++k) {
        ora_real t = V[v - k] + E[EIDX(N, v - k + 1, v)];
        if (t < Et) Et = t;
      }
    }
    ora_real s = 0.0;
    for (int k = 1; k <= v; ++k)
      s += EXP(-beta * (V[v - k] + E[EIDX(N, v - k + 1, v)] - Et));
    V[v] = Et - (1.0 / beta) * LOG(s / (ora_real)v);
  }
  return 0;
}

/* Eq. backward-potential-recursion (Theorem backward-recurrence), shifted:
 *   V^{[u,N]} = Et - (1/beta) ln[ sum_{l=u}^{N} (1/l) EXP(-beta (E^{[u,l]}
 *                                   + V^{[l+1,N]} - Et)) ],   V^{[N+1,N]} = 0,
 * Et = min over the terms (Eq. full-elong) or the two-term form of Eq.
 * original-elong (E^{[u,u]} + V^{[u+1,N]} and E^{[u,N]}). */
int ora_backward_potentials(int N, ora_real beta, const ora_real *E, int shift_mode,
                            ora_real *W) {
  if (N < 1 || !(beta > 0.0) || !E || !W) return -1;
  /* W[u-1] holds V^{[u,N]} */
  W[N] = 0.0;
  for (int u = N; u >= 1; --u) {
    ora_real Et;
    if (shift_mode == ORA_SHIFT_TWO_TERM) {
      ora_real a = E[EIDX(N, u, u)] + W[u], b = E[EIDX(N, u, N)];
      Et = a < b ? a : b;
    } else {
      Et = INF_REAL;
      for (int l = u; l <= N; ++l) {
        ora_real t = E[EIDX(N, u, l)] + W[l];
        if (t < Et) Et = t;
      }
    }
    ora_real s = 0.0;
    for (int l = u; l <= N; ++l)
      s += (1.0 / (ora_real)l) * EXP(-beta * (E[EIDX(N, u, l)] + W[l] - Et));
    W[u - 1] = Et - (1.0 / beta) * LOG(s);
  }
  return 0;
}

/* Definition backward-potential, evaluated literally: for each u,
 *   EXP(-beta V^{[u,v]}) = (1/v) sum_{k=1}^{v-u+1} EXP(-beta (V^{[u,v-k]} + E^{[v-k+1,v]}))
 * for v = u..N with EXP(-beta V^{[u,u-1]}) = 1; then V^{[u,N]} is the v = N value.
 * O(N^2) per u, O(N^3) overall.  Same min-shift as the forward recursion. */
int ora_backward_potentials_definition(int N, ora_real beta, const ora_real *E,
                                       ora_real *W) {
  if (N < 1 || !(beta > 0.0) || !E || !W) return -1;
  /* X[v - (u-1)] = V^{[u,v]} for v = u-1..N */
  ora_real *X = (ora_real *)malloc(sizeof(ora_real) * (size_t)(N + 2));
  if (!X) return -1;
  W[N] = 0.0;
  for (int u = 1; u <= N; ++u) {
    X[0] = 0.0; /* V^{[u,u-1]} */
    for (int v = u; v <= N; ++v) {
      ora_real Et = INF_REAL;
      for (int k = 1; k <= v - u + 1; ++k) {
        ora_real t = X[v - k - (u - 1)] + E[EIDX(N, v - k + 1, v)];
        if (t < Et) Et = t;
      }
      ora_real s = 0.0;
      for (int k = 1; k <= v - u + 1; ++k)
        s += EXP(-beta * (X[v - k - (u - 1)] + E[EIDX(N, v - k + 1, v)] - Et));
      X[v - (u - 1)] = Et - (1.0 / beta) * LOG(s / (ora_real)v);
    }
    W[u - 1] = X[N - (u - 1)];
  }
  free(X);
  return 0;
}

/* Connection probabilities (Methods, "Expressions for connection probabilities"):
 *   Pr[l -> l+1] = 1 - EXP(-beta (V^{[1,l]} + V^{[l+1,N]} - V^{[1,N]}))   (Eq. direct-link)
 *   Pr[l -> l']  = (1/l) EXP(-beta (V^{[1,l'-1]} + E^{[l',l]} + V^{[l+1,N]}
 *                                   - V^{[1,N]}))  for l' <= l           (Eq. close-cycle)
 *   Pr[l -> l']  = 0 for l' > l + 1           (Lemma zero-connection-probability)
 * The direct link uses -EXPM1(-x) for 1 - EXP(-x). */
int ora_connection_probabilities(int N, ora_real beta, const ora_real *E,
                                 const ora_real *V, const ora_real *W, ora_real *M) {
  if (N < 1 || !(beta > 0.0) || !E || !V || !W || !M) return -1;
  memset(M, 0, sizeof(ora_real) * (size_t)N * (size_t)N);
  const ora_real VN = V[N];
  for (int l = 1; l <= N - 1; ++l)
    M[EIDX(N, l, l + 1)] = -EXPM1(-beta * (V[l] + W[l] - VN)); /* W[l] = V^{[l+1,N]} */
  for (int lp = 1; lp <= N; ++lp)
    for (int l = lp; l <= N; ++l)
      M[EIDX(N, l, lp)] = (1.0 / (ora_real)l) *
                          EXP(-beta * (V[lp - 1] + E[EIDX(N, lp, l)] + W[l] - VN));
  return 0;
}

/* Forces of Algorithm 1.
 *   interior (j = 2..P-1): -m w_P^2 (2 r_l^j - r_l^{j+1} - r_l^{j-1})     (Eq. intermediate-bead-force)
 *   bead 1: -sum_{l'=l-1}^{N} Pr[l'->l] m w_P^2 (2 r_l^1 - r_l^2 - r_{l'}^P)
 *   bead P: -sum_{l'=1}^{l+1} Pr[l->l'] m w_P^2 (2 r_l^P - r_{l'}^1 - r_l^{P-1})
 * with the edge limits clipped to 1..N (Algorithm 1, exterior-force lines). */
int ora_forces(int N, int P, ora_real m, ora_real omega_P, const ora_real *pos,
               const ora_real *M, ora_real *F) {
  if (bad_args(N, P) || !pos || !M || !F) return -1;
  const ora_real k = m * omega_P * omega_P;
  for (int l = 1; l <= N; ++l)
    for (int j = 2; j <= P - 1; ++j)
      for (int d = 0; d < 3; ++d)
        BEAD(F, P, l, j)[d] = -k * lap1(BEAD(pos, P, l, j)[d], BEAD(pos, P, l, j + 1)[d],
                                        BEAD(pos, P, l, j - 1)[d]);
  for (int l = 1; l <= N; ++l) {
    ora_real f1[3] = {0.0, 0.0, 0.0}, fP[3] = {0.0, 0.0, 0.0};
    int lo = l - 1 < 1 ? 1 : l - 1;
    for (int lp = lo; lp <= N; ++lp) {
      ora_real pr = M[EIDX(N, lp, l)];
      for (int d = 0; d < 3; ++d)
        f1[d] -= pr * k * lap1(BEAD(pos, P, l, 1)[d], BEAD(pos, P, l, 2)[d], BEAD(pos, P, lp, P)[d]);
    }
    int hi = l + 1 > N ? N : l + 1;
    for (int lp = 1; lp <= hi; ++lp) {
      ora_real pr = M[EIDX(N, l, lp)];
      for (int d = 0; d < 3; ++d)
        fP[d] -= pr * k * lap1(BEAD(pos, P, l, P)[d], BEAD(pos, P, lp, 1)[d], BEAD(pos, P, l, P - 1)[d]);
    }
    for (int d = 0; d < 3; ++d) {
      BEAD(F, P, l, 1)[d] = f1[d];
      BEAD(F, P, l, P)[d] = fP[d];
    }
  }
  return 0;
}

/* Algorithm 1 (Fast PIMD-B): cycle energies, forward potentials, backward
 * potentials, connection probabilities, interior and exterior forces. */
int ora_fast_pimdb(int N, int P, ora_real m, ora_real omega_P, ora_real beta,
                   const ora_real *pos, ora_real *V_B, ora_real *F,
                   ora_real *Vout, ora_real *Wout, ora_real *Mout) {
  if (bad_args(N, P) || !(beta > 0.0) || !(m > 0.0) || !(omega_P > 0.0) || !pos || !F)
    return -1;
  size_t NN = (size_t)N * (size_t)N;
  ora_real *E = (ora_real *)malloc(sizeof(ora_real) * NN);
  ora_real *M = Mout ? Mout : (ora_real *)malloc(sizeof(ora_real) * NN);
  ora_real *V = Vout ? Vout : (ora_real *)malloc(sizeof(ora_real) * (size_t)(N + 1));
  ora_real *W = Wout ? Wout : (ora_real *)malloc(sizeof(ora_real) * (size_t)(N + 1));
  int rc = -1;
  if (E && M && V && W) {
    rc = ora_cycle_energies(N, P, m, omega_P, pos, E);
    if (!rc) rc = ora_forward_potentials(N, beta, E, ORA_SHIFT_MIN_ALL, V);
    if (!rc) rc = ora_backward_potentials(N, beta, E, ORA_SHIFT_MIN_ALL, W);
    if (!rc) rc = ora_connection_probabilities(N, beta, E, V, W, M);
    if (!rc) rc = ora_forces(N, P, m, omega_P, pos, M, F);
    if (!rc && V_B) *V_B = V[N];
  }
  free(E);
  if (!Mout) free(M);
  if (!Vout) free(V);
  if (!Wout) free(W);
  return rc;
}

/* Gradient of the cycle energy E^{[u,v]} with respect to bead (l, j), written
 * into g[3] (Algorithm 2, cycle-energy derivative lines): m w_P^2 (2 r_l^j -
 * r_l^{j+1} - r_l^{j-1}) with r_l^0 = r_{l-1}^P, r_l^{P+1} = r_{l+1}^1, except
 * r_u^0 = r_v^P and r_v^{P+1} = r_u^1; zero when l is outside [u, v]. */
static void cycle_energy_gradient(int P, ora_real k, const ora_real *pos, int u, int v,
                                  int l, int j, ora_real *g) {
  if (l < u || l > v) { g[0] = g[1] = g[2] = 0.0; return; }
  const ora_real *next, *prev;
  if (j < P) next = BEAD(pos, P, l, j + 1);
  else next = (l < v) ? BEAD(pos, P, l + 1, 1) : BEAD(pos, P, u, 1);
  if (j > 1) prev = BEAD(pos, P, l, j - 1);
  else prev = (l > u) ? BEAD(pos, P, l - 1, P) : BEAD(pos, P, v, P);
  const ora_real *r = BEAD(pos, P, l, j);
  for (int d = 0; d < 3; ++d) g[d] = k * lap1(r[d], next[d], prev[d]);
}

/* Algorithm 2 (Original PIMD-B).
 * Cycle energies by the direct sum of Algorithm 2 (interior springs of u..v,
 * links l -> l+1 for l = u..v-1, closing spring v -> u); forward potentials as
 * in Algorithm 1; then for every bead the recursion obtained by differentiating
 * Eq. our-forward-potential-recurrence:
 *   grad V^{[1,v]} = sum_{k=1}^{v} (grad E^{[v-k+1,v]} + grad V^{[1,v-k]})
 *                    EXP(-beta (E^{[v-k+1,v]} + V^{[1,v-k]})) / (v EXP(-beta V^{[1,v]})),
 * grad V^{[1,0]} = 0, and F = -grad V^{[1,N]}. */
int ora_original_pimdb(int N, int P, ora_real m, ora_real omega_P, ora_real beta,
                       const ora_real *pos, ora_real *V_B, ora_real *F) {
  if (bad_args(N, P) || !(beta > 0.0) || !(m > 0.0) || !(omega_P > 0.0) || !pos || !F)
    return -1;
  const ora_real half_k = 0.5 * m * omega_P * omega_P, k = m * omega_P * omega_P;
  size_t NN = (size_t)N * (size_t)N;
  ora_real *E = (ora_real *)malloc(sizeof(ora_real) * NN);
  ora_real *V = (ora_real *)malloc(sizeof(ora_real) * (size_t)(N + 1));
  ora_real *dV = (ora_real *)malloc(sizeof(ora_real) * 3 * (size_t)(N + 1));
  if (!E || !V || !dV) { free(E); free(V); free(dV); return -1; }
  for (int v = 1; v <= N; ++v) {
    for (int u = 1; u <= v; ++u) {
      ora_real s = 0.0;
      for (int l = u; l <= v; ++l)
        for (int j = 1; j <= P - 1; ++j) s += sqdist(BEAD(pos, P, l, j + 1), BEAD(pos, P, l, j));
      for (int l = u; l <= v - 1; ++l) s += sqdist(BEAD(pos, P, l + 1, 1), BEAD(pos, P, l, P));
      s += sqdist(BEAD(pos, P, u, 1), BEAD(pos, P, v, P));
      E[EIDX(N, u, v)] = half_k * s;
    }
  }
  ora_forward_potentials(N, beta, E, ORA_SHIFT_MIN_ALL, V);
  for (int l = 1; l <= N; ++l) {
    for (int j = 1; j <= P; ++j) {
      dV[0] = dV[1] = dV[2] = 0.0;
      for (int v = 1; v <= N; ++v) {
        ora_real acc[3] = {0.0, 0.0, 0.0};
        for (int kk = 1; kk <= v; ++kk) {
          int u = v - kk + 1;
          ora_real g[3];
          cycle_energy_gradient(P, k, pos, u, v, l, j, g);
          /* EXP(-beta(E + V^{[1,v-k]})) / (v EXP(-beta V^{[1,v]})) */
          ora_real w = EXP(-beta * (E[EIDX(N, u, v)] + V[v - kk] - V[v])) / (ora_real)v;
          for (int d = 0; d < 3; ++d) acc[d] += (g[d] + dV[3 * (v - kk) + d]) * w;
        }
        for (int d = 0; d < 3; ++d) dV[3 * v + d] = acc[d];
      }
      for (int d = 0; d < 3; ++d) BEAD(F, P, l, j)[d] = -dV[3 * N + d];
    }
  }
  if (V_B) *V_B = V[N];
  free(E); free(V); free(dV);
  return 0;
}

/* Expected spring energy over representative permutations:
 * sum_l E_int^{(l)} + sum_l sum_{l'} Pr[l->l'] (1/2) m w_P^2 (r_l^P - r_{l'}^1)^2.
 * Linear in the exterior springs, so the expectation over the distribution of
 * Eq. representative-distribution reduces to the connection probabilities. */
int ora_expected_spring_energy(int N, int P, ora_real m, ora_real omega_P,
                               const ora_real *pos, const ora_real *M, ora_real *out) {
  if (bad_args(N, P) || !pos || !M || !out) return -1;
  const ora_real half_k = 0.5 * m * omega_P * omega_P;
  ora_real *Eint = (ora_real *)malloc(sizeof(ora_real) * (size_t)N);
  if (!Eint) return -1;
  ora_interior_energies(N, P, m, omega_P, pos, Eint);
  ora_real s = 0.0;
  for (int l = 1; l <= N; ++l) {
    s += Eint[l - 1];
    for (int lp = 1; lp <= N; ++lp) {
      ora_real pr = M[EIDX(N, l, lp)];
      if (pr != 0.0) s += pr * half_k * sqdist(BEAD(pos, P, l, P), BEAD(pos, P, lp, 1));
    }
  }
  free(Eint);
  *out = s;
  return 0;
}
