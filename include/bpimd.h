/*
 * bpimd.h -- C ABI of the GB300 (sm_103a) bosonic PIMD exchange library.
 *
 * The library evaluates the bosonic exchange potential V_B = V^{[1,N]} of N
 * ring polymers with P beads each, and its force on every bead, following
 * Feldman & Hirshberg, "Quadratic Scaling Bosonic Path Integral Molecular
 * Dynamics":
 *   - cycle energies E^{[u,v]}  (Eq. Ek, Eq. e-interior, Eq. e-recurrence-step/base)
 *   - forward potentials V^{[1,v]}  (Eq. our-forward-potential-recurrence)
 *   - backward potentials V^{[u,N]} (Eq. backward-potential-recursion)
 *   - connection probabilities Pr[l -> l'] (Eq. direct-link-probability,
 *     Eq. close-cycle-probability, Lemma zero-connection-probability)
 *   - forces: interior beads (Eq. intermediate-bead-force), beads 1 and P
 *     (Eq. force-on-1-sum-neighbors, Eq. force-on-P-sum-neighbors), i.e.
 *     Algorithm 1 ("Fast PIMD-B") of the appendix.
 * and, for molecular dynamics, a Langevin/velocity-Verlet step that adds the
 * physical potential U-bar = (1/P) sum_j U(r_1^j..r_N^j) of Eq.
 * int-of-sum-all-permutations (harmonic trap plus a same-bead pair potential).
 *
 * Every computation runs in this library's own CUDA kernels on one GPU; there
 * is no CPU fallback.  All entry points return an int status (BPIMD_OK = 0 or a
 * negative BPIMD_ERR_* code) and never abort the process.
 *
 * Memory layout shared by all calls
 *   positions, forces, velocities: [N][P][3] row-major float64, i.e. bead j
 *   (0-based) of particle l (0-based) coordinate d at index (l*P + j)*3 + d.
 *   Device pointers must be 16-byte aligned.  The caller owns these buffers;
 *   the library never frees or retains them beyond the call.
 *
 * Streams and synchronisation
 *   A context is bound to one CUDA stream given at creation (NULL = the legacy
 *   default stream).  Calls that take device pointers enqueue their work on
 *   that stream and return without waiting for it, unless stated otherwise;
 *   the caller orders its own use of outputs with that stream.  Calls whose
 *   name ends in _host take host pointers, copy in, compute, copy out and
 *   synchronise the stream before returning.  A context must not be used from
 *   two host threads at once.
 *
 * Errors
 *   Argument errors are detected on the host before anything is enqueued
 *   (BPIMD_ERR_ARG).  Device-side conditions (non-finite positions or results)
 *   are recorded in a device status word; they surface as BPIMD_ERR_NONFINITE
 *   from the next call that synchronises (the _host calls, bpimd_sync,
 *   bpimd_step).  The CTAs of a recursion cluster hand their results to one
 *   another through shared-memory mbarriers; each such wait is bounded (one
 *   second of the GPU's global timer).  A wait that expires records
 *   BPIMD_ERR_TIMEOUT: the CTAs then stop waiting and handing off, every
 *   kernel runs to its end (the evaluation's outputs are invalid), and the
 *   context and the CUDA context stay usable.  BPIMD_FLAG_TEST_TIMEOUT makes
 *   this happen on purpose, for tests of the error path.
 */
#ifndef BPIMD_H
#define BPIMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define BPIMD_OK 0
#define BPIMD_ERR_ARG (-1)       /* invalid size, parameter or null pointer      */
#define BPIMD_ERR_NONFINITE (-2) /* NaN/Inf in positions or in a result          */
#define BPIMD_ERR_CUDA (-3)      /* a CUDA runtime call failed                  */
#define BPIMD_ERR_TIMEOUT (-4)   /* a bounded device-side wait expired           */
#define BPIMD_ERR_NOMEM (-5)     /* device or host allocation failed            */
#define BPIMD_ERR_STATE (-6)     /* call not valid for this context's state     */
#define BPIMD_ERR_SIZE (-7)      /* problem larger than a fixed-size buffer      */

/* ---------------------------------------------------------------- precision */
/* The precision forms.  Each names what every step computes in; "integer"
 * steps carry extended numbers m 2^e with an integer mantissa m and an int32
 * exponent.
 *
 * BPIMD_FP64: float64 bead differences, spring energies, closing-spring
 *   distances and forces; pair Boltzmann factors g = 2^(-x) of the exact
 *   float64 product x by a 64-bit fixed-point table method (integer pipe,
 *   2^-60 relative before the final float64 rounding); the blocked recursions
 *   (tile inverses, the lead's tile products and the bulk sums) on 64-bit
 *   integer mantissas with int32 exponents (truncation 2^-61 per operation);
 *   float64 probabilities and force sums.
 * BPIMD_MIXED: float32 bead differences, per-particle spring energies (float32
 *   warp sums) and closing-spring distances; everything after them at float64
 *   accuracy or better: the link coefficients and the prefix sums of spring
 *   energies in float64, g = 2^(-x) of the exact product of the float32
 *   closing-spring term and the float64 constant beta k/2 log2(e) by the same
 *   integer table method, the recursions on 64-bit integer mantissas as in
 *   BPIMD_FP64, probabilities Pr = alpha mu g from 64-bit integer
 *   mantissa products, and the probability and force sums as unevaluated
 *   sums of two float32 numbers (compensated: 2^-46 relative) over float32
 *   bead differences.
 * BPIMD_MIXED32: the fastest form: float32 bead differences and spring
 *   energies, g from the float32 hardware exponential (ex2.approx), the
 *   recursions' bulk sums as float32 products over 8 sources, the tile
 *   inverses and the lead's tile products on 64-bit integer mantissas,
 *   float32 probabilities and block-local force sums (combined across blocks
 *   with float32 TwoSum compensation); float64 prefix sums, link coefficients,
 *   and outputs.
 * Replica batches (bpimd_create_batched) run each recursion of a replica of
 * up to 4096 particles on one CTA as 32 dependent steps per tile, in the same
 * formats, except that BPIMD_MIXED32 multiplies there by the top 32 bits of
 * the 64-bit factor mantissa (truncation 2^-30 per step).
 * All three meet the mixed tolerances (1e-6 relative on V_B, 1e-5 RMS on
 * forces); BPIMD_FP64 meets 1e-12 / 1e-10. */
#define BPIMD_FP64 0
#define BPIMD_MIXED 1
#define BPIMD_MIXED32 2

/* ------------------------------------------------------------ storage */
/* Largest N a single system accepts. */
#define BPIMD_MAX_N 16384
/* Up to this N a context tabulates the pair Boltzmann factors g(u, v) of the
 * closing springs once per evaluation (two coalesced copies, O(N^2) device
 * memory: 12 or 16 bytes per pair and copy, ~0.8 GB at N = 8192) and the
 * probability pass keeps O(N^2 / 32) block partial sums.  Above it -- or at
 * any N when cfg.flags has BPIMD_FLAG_RECOMPUTE -- nothing O(N^2) is stored:
 * the recursions and the probability pass recompute each g where they use it
 * (the same bits), and the probability pass forms every pair twice, once for
 * its row and once for its column, so that each force sum is completed by one
 * CTA.  Device memory is then O(N + N P). */
#define BPIMD_STORE_MAX_N 8192
#define BPIMD_FLAG_RECOMPUTE 1
/* Test hook of the error path (bpimd_create only): the forward recursion's
 * first hand-off wait waits for a hand-off that is never made, so every
 * evaluation of the context ends with BPIMD_ERR_TIMEOUT after about one
 * second, with invalid outputs.  No GPU fault is involved: the wait gives up,
 * and the kernels finish. */
#define BPIMD_FLAG_TEST_TIMEOUT 2

/* --------------------------------------------------------- pair potentials */
#define BPIMD_PAIR_NONE 0
#define BPIMD_PAIR_GAUSSIAN 1 /* g exp(-r^2 / (2 s^2)) between same-index beads */
#define BPIMD_PAIR_LJ 2       /* 4 eps ((sigma/r)^12 - (sigma/r)^6), truncated at rc
                                 and shifted to 0 there (liquid helium)          */

typedef struct bpimd_ctx bpimd_ctx; /* opaque; owns the device workspace */

/* Problem description (Eq. eperm and Eq. int-of-sum-all-permutations).
 * N >= 1 particles, P >= 2 beads (the bead-1 / bead-P formulas need two
 * distinct exterior beads).  m, omega_P, beta > 0 and finite; omega_P is passed
 * explicitly (sqrt(P)/(beta hbar) in the paper's convention).  The fields
 * after `precision` are used only by bpimd_step and may be zero otherwise. */
typedef struct {
  int32_t N;
  int32_t P;
  double m;
  double omega_P;
  double beta;
  int32_t precision; /* BPIMD_FP64, BPIMD_MIXED or BPIMD_MIXED32 */
  int32_t flags;     /* 0, BPIMD_FLAG_RECOMPUTE, BPIMD_FLAG_TEST_TIMEOUT; other bits must be 0 */
  /* molecular dynamics (bpimd_step) */
  double dt;         /* time step                                   */
  double gamma;      /* Langevin friction (0 = NVE)                  */
  double kT_bead;    /* thermostat kT of the bead momenta; 0 => 1/beta, the temperature
                        at which exp(-beta (V_B + U-bar)) is sampled with w_P = sqrt(P)/(beta hbar) */
  double omega0;     /* isotropic harmonic trap frequency (0 = none) */
  int32_t pair_type; /* BPIMD_PAIR_*                                 */
  int32_t pad0;
  double pair_a;     /* Gaussian g  | LJ epsilon                      */
  double pair_b;     /* Gaussian s  | LJ sigma                        */
  double pair_rc;    /* LJ cutoff rc > 0 (at most box_L/2 in a box)   */
  double box_L;      /* periodic cubic box side (0 = open boundaries):
                        every spring -- interior, link, closing -- and
                        every pair joins the minimum image of its two
                        beads; positions need not be wrapped.  Used by
                        the exchange evaluation and by bpimd_step; not
                        by replica batches (must be 0 there).          */
  uint64_t seed;     /* counter-based RNG key for the thermostat      */
} bpimd_config;

/* Create a context for one system.  Validates cfg (BPIMD_ERR_ARG; 1 <= N <=
 * BPIMD_MAX_N), allocates the workspace on the current CUDA device
 * (BPIMD_ERR_NOMEM; O(N^2) up to BPIMD_STORE_MAX_N, else O(N P)), binds
 * `cuda_stream` (a cudaStream_t, NULL = default stream).  On error *out is set
 * to NULL.  Destroy with bpimd_destroy. */
int bpimd_create(bpimd_ctx **out, const bpimd_config *cfg, void *cuda_stream);

/* Release all device and host memory of the context.  NULL-safe.
 * Synchronises the context's stream first. */
int bpimd_destroy(bpimd_ctx *ctx);

/* Exchange potential and forces, Algorithm 1 (appendix "Algorithm Pseudocode").
 *   positions : device, [N][P][3] float64, read only.
 *   V_B       : device pointer to one float64; receives V^{[1,N]}.  May be NULL.
 *   forces    : device, [N][P][3] float64; overwritten with -grad V^{[1,N]}
 *               (interior springs included; no physical potential).
 * Enqueued on the context stream; asynchronous. */
int bpimd_exchange_energy_forces(bpimd_ctx *ctx, const double *positions,
                                 double *V_B, double *forces);

/* Same computation with HOST buffers: copies positions in, computes, copies
 * V_B (may be NULL) and forces out, synchronises.  Host buffers may be pageable
 * or pinned; pinned memory is faster.  With pinned buffers on a non-default
 * stream (and stage profiling off) the whole call -- copies, the evaluation
 * kernels and the status read -- is captured once into a CUDA graph for that
 * (positions, forces) pair and replayed on later calls. */
int bpimd_exchange_energy_forces_host(bpimd_ctx *ctx, const double *positions,
                                      double *V_B, double *forces);

/* Wait for the context stream and report any device-side status recorded by
 * earlier calls (BPIMD_ERR_NONFINITE), clearing it. */
int bpimd_sync(bpimd_ctx *ctx);

/* Intermediate results of the last bpimd_exchange_energy_forces* call, copied
 * to HOST arrays (synchronises).  Any pointer may be NULL.
 *   V_fwd : N+1 float64, V_fwd[v] = V^{[1,v]} (V_fwd[0] = 0).
 *   V_bwd : N+1 float64, V_bwd[u-1] = V^{[u,N]} for u = 1..N+1 (V_bwd[N] = 0).
 *   Eint  : N float64, E_int^{(l)} (Eq. e-interior).
 * For testing and diagnostics; O(N) data. */
int bpimd_get_potentials(bpimd_ctx *ctx, double *V_fwd, double *V_bwd, double *Eint);

/* Dense connection-probability matrix of the last evaluation, recomputed on
 * the device from the stored O(N) state: M[(l-1)*N + (l'-1)] = Pr[l -> l']
 * (0 for l' > l+1).  M is a DEVICE buffer of N*N float64 owned by the caller.
 * O(N^2) memory; intended for tests and diagnostics.  Asynchronous. */
int bpimd_connection_probabilities(bpimd_ctx *ctx, double *M);

/* Run `nsteps` molecular-dynamics steps in place, sampling
 * exp(-beta (V_B + U-bar)) (Eq. int-of-sum-all-permutations; the paper does not
 * state its integrator): BAOAB Langevin splitting -- half kick, half drift,
 * exact Ornstein-Uhlenbeck velocity update v = c1 v + c2 z (c1 = exp(-gamma dt),
 * c2 = sqrt((1 - c1^2) kT / m)), half drift, force evaluation, half kick -- with
 * bead mass m and the full force = exchange force (Algorithm 1) + harmonic trap
 * (omega0) + pair potential of cfg, U-bar = (1/P) sum_j U(r_1^j..r_N^j).
 * Thermostat normals: Philox4x32-10 (Salmon et al., SC'11) keyed by cfg.seed,
 * counter (element/4, step index) with Box-Muller; the step index counts the
 * steps this context has taken (0 at creation).
 *   positions, velocities : device [N][P][3] float64, updated in place.
 *   energies : optional device array of 4 float64 receiving, after the last
 *              step: [0] V_B, [1] U-bar, [2] kinetic energy sum (1/2) m v^2,
 *              [3] primitive energy estimator 3NP/(2 beta) - <E^{G[sigma]}> + U-bar,
 *              where <E^{G[sigma]}> is the spring energy averaged over the
 *              connection probabilities.  May be NULL.
 * Each call first evaluates the force at the given positions.  On a stream
 * other than the legacy default stream the step is captured once into a CUDA
 * graph (bound to these position/velocity buffers) and replayed.
 * Lennard-Jones in a box of at least 3 cutoffs per side runs on cell lists
 * (O(N P) per step); otherwise pairs are summed over all partners.
 * On a replica-batch context (bpimd_create_batched) every replica advances by
 * the same steps: positions and velocities are the packed arrays of the batch,
 * dt, gamma, omega0, the Gaussian pair potential and the seed are shared,
 * each replica is thermostatted at kT = 1/beta_r (or cfg.kT_bead), the
 * thermostat counter is the element index in the packed array, and energies
 * (if not NULL) receives 4 float64 per replica in replica order.  Batches
 * take no Lennard-Jones pairs (they have no periodic box).
 * Errors: BPIMD_ERR_ARG for nsteps < 0, misaligned pointers, dt <= 0,
 * gamma < 0, kT_bead < 0, omega0 < 0, an unknown pair_type, a Gaussian width
 * or Lennard-Jones sigma <= 0, a Lennard-Jones cutoff <= 0 or above box_L/2.
 * Synchronises and returns device status. */
int bpimd_step(bpimd_ctx *ctx, double *positions, double *velocities,
               int32_t nsteps, double *energies);

/* --------------------------------------------------------- replica batches */
/* Many independent systems ("replicas") of uneven size and temperature
 * evaluated together: the same Algorithm 1 per replica, three kernel launches
 * per batch whatever the number of replicas, plus one recursion launch per
 * replica with N > 4096 (those take the cluster recursion kernel of single
 * systems; the other replicas run one CTA per recursion).  The paper has no batched form;
 * it serves workloads such as parallel tempering or many small trapped
 * systems that are too small to fill a GPU one at a time.
 *
 * bpimd_create_batched: cfg supplies m, precision, flags (0) and the
 * molecular-dynamics fields (its N, P, omega_P and beta are ignored); host
 * arrays of length R give each
 * replica's N[r] (1..BPIMD_STORE_MAX_N), P[r] (>= 2), omega_P[r] and beta[r] (> 0, finite).
 * Packed layout of positions and forces: replica r occupies
 * [N[r]][P[r]][3] float64 starting at element offset
 * off[r] = 3 * sum_{q<r} N[q] P[q] (bpimd_batch_info returns them).
 * Errors: BPIMD_ERR_ARG (sizes, parameters), BPIMD_ERR_NOMEM.  Single-system
 * calls on a batch context (and batch calls on a single-system context)
 * return BPIMD_ERR_STATE; bpimd_step (molecular dynamics of every replica),
 * bpimd_sync, bpimd_profile_* and bpimd_destroy work on both.  cfg's
 * molecular-dynamics fields (dt, gamma, kT_bead, omega0, the Gaussian pair
 * potential, seed) are used by bpimd_step. */
int bpimd_create_batched(bpimd_ctx **out, const bpimd_config *cfg, int32_t R,
                         const int32_t *N, const int32_t *P, const double *omega_P,
                         const double *beta, void *cuda_stream);

/* One evaluation of every replica (asynchronous on the context stream):
 *   positions : device, packed [sum 3 N_r P_r] float64 (16-byte aligned).
 *   V_B       : device array of R float64 receiving V^{[1,N_r]}; may be NULL.
 *   forces    : device, packed like positions; overwritten with -grad V. */
int bpimd_exchange_energy_forces_batched(bpimd_ctx *ctx, const double *positions,
                                         double *V_B, double *forces);

/* Batch geometry: *R, the total number of float64 elements of the packed
 * arrays, and (if not NULL) offsets[R] in elements.  Any pointer may be NULL. */
int bpimd_batch_info(bpimd_ctx *ctx, int32_t *R, int64_t *elements, int64_t *offsets);

/* Launch shape of the batched pair-factor and probability passes: at most
 * blocks_per_sm x (number of SMs) CTAs each (1..64; default 8); the
 * pair-factor CTAs run in the same launch as the bead pass, after its CTAs.  Set by the
 * autotuner (paper_2305_18025_gb300/autotune.py); results do not depend on it. */
int bpimd_batch_set_tuning(bpimd_ctx *ctx, int32_t pair_blocks_per_sm, int32_t prob_blocks_per_sm);

/* Pair tile of the batch's molecular dynamics (bpimd_step): the trap and pair
 * forces between beads of equal index (the potential U of Eq.
 * int-of-sum-all-permutations) run one 256-thread block per (replica, block
 * of particles, bead index), lanes_per_particle lanes sharing each particle's
 * partners (2, 4 or 8: 128, 64 or 32 particles per block; default 4).  Few
 * lanes suit large replicas, many lanes small ones.  Set by the autotuner.
 * The per-lane partner order changes with the tile, so forces differ by
 * float rounding (within the precision form's tolerance).  Any time: a tile
 * changed after MD steps drops the captured step, which the next bpimd_step
 * recaptures; positions, velocities and the thermostat counter are kept.
 * BPIMD_ERR_STATE for a single-system context, BPIMD_ERR_ARG for other values. */
int bpimd_batch_set_pair_tile(bpimd_ctx *ctx, int32_t lanes_per_particle);

/* ------------------------------------------------------------- profiling */
/* Stage timing with CUDA events recorded on the context stream around each
 * kernel of an evaluation.  Stage order:
 *   0 bead pass and pair Boltzmann factors (one launch),
 *   1 forward+backward recursions (with the prefix sums, V_B and the
 *     probability normaliser),
 *   2 connection probabilities + exterior-bead forces. */
#define BPIMD_NUM_STAGES 3

/* Start recording stage events for up to `max_evals` following evaluations
 * (older records are discarded).  Adds BPIMD_NUM_STAGES + 1 event records per
 * evaluation. */
int bpimd_profile_begin(bpimd_ctx *ctx, int max_evals);

/* Stop recording, synchronise, and write the summed device time of each stage
 * in milliseconds to stage_ms[BPIMD_NUM_STAGES] and the number of recorded
 * evaluations to *n_evals.  Either pointer may be NULL. */
int bpimd_profile_end(bpimd_ctx *ctx, double *stage_ms, int *n_evals);

/* ----------------------------------------------- allocation-free variant */
/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory at the moment they need an evaluation: a host
 * program whose memory manager owns every device allocation, a simulation loop
 * that may not call cudaMalloc/cudaFree (they can synchronise the whole
 * device and stall other streams), or an embedding with a fixed memory budget.
 *
 * Same computation and arguments as bpimd_exchange_energy_forces, without a
 * context: cfg describes the system (N, P, m, omega_P, beta, precision; the MD
 * fields are ignored), positions/V_B/forces are device pointers owned by the
 * caller, cuda_stream is a cudaStream_t (NULL = default stream) that must
 * belong to the current device (a stream of another device returns
 * BPIMD_ERR_ARG: the scratch array used is the current device's).  It allocates
 * nothing: its scratch memory is one file-scope __device__ array of 1 MiB per
 * device, which bounds the size to N <= BPIMD_NOALLOC_MAX_N (larger N returns
 * BPIMD_ERR_SIZE before any work is enqueued).
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress) and caches it; make that
 *     first call before any stream capture.
 *   - Every call on a device shares the array, which keeps the previous call's
 *     contents; calls whose work overlaps on the GPU (e.g. on two streams)
 *     race on it.  Serialise them (one stream).
 *   - Asynchronous; device-side status (non-finite inputs) is not reported:
 *     non-finite positions give non-finite outputs. */
#define BPIMD_NOALLOC_MAX_N 256
int bpimd_exchange_energy_forces_noalloc(const bpimd_config *cfg, const double *positions,
                                         double *V_B, double *forces, void *cuda_stream);

/* --------------------------------------------------- throughput probes */
/* Measurement utility for roofline figures (no counterpart in the paper):
 * enqueue one compute-bound kernel on cuda_stream (a cudaStream_t, NULL =
 * default stream) that keeps every SM busy with independent chains of
 *   kind 0: float64 fused multiply-adds (the float64 pipe),
 *   kind 1: 32 x 32 -> 64-bit integer multiply-adds (the integer pipe),
 * `iters` per chain, and return in *ops (may be NULL) the number of
 * multiply-adds it performs.  The caller times it (CUDA events on the same
 * stream) and divides.  sink: a device buffer of at least 8 * 8 * SMs bytes
 * (8-byte aligned) that the kernel writes only in a case that never occurs.
 * Asynchronous; BPIMD_ERR_ARG for another kind, iters < 1 or a bad sink. */
int bpimd_peak_probe(int32_t kind, int64_t iters, void *sink, void *cuda_stream, int64_t *ops);

/* Self-test of the device's powers of two (no counterpart in the paper; for
 * tests), both by the integer-pipe fixed-point method, x >= 0, 0 below the
 * float64 normal range: out[i] = 2^(-x[i]/2) with the exact double x double
 * argument product of the float64 Gaussian pair force (method 0, factor 1/2),
 * or 2^(-x[i]) as for the float64 pair factors (method 1).
 * x, out: device arrays of n float64.  Asynchronous on cuda_stream. */
int bpimd_pow2_selftest(int32_t method, const double *x, double *out, int32_t n, void *cuda_stream);

/* Human-readable text for a status code (static storage). */
const char *bpimd_status_string(int status);

/* Library version string (static storage). */
const char *bpimd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BPIMD_H */
