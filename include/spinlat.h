/*
 * spinlat.h -- C ABI of the GB300 (sm_103a) NEP-SPIN spin-lattice step library.
 *
 * The library advances a coupled lattice + spin system under the spin-aware
 * neuro-evolution potential of arXiv 2606.14073 and its spin-lattice integrator:
 *   - create_system(positions, spins, box, species, nep_params)   (Section 5.2.1)
 *   - step(n, dt, T, B)                                           (Sections 5.1.3, 5.2.1)
 *   - energy_forces_fields()                                      (Sections 5.1.1, 5.1.2)
 * Every step runs on the GPU: cell-list neighbour search, the 66-entry spin-aware
 * descriptor, the per-atom tanh network, its backward pass to forces, spin fields
 * and virial, and the integrator.  There is no CPU fallback; without a usable
 * CUDA device every call returns SL_ECUDA.
 *
 * Conventions
 *   units      A, fs, eV, amu, K, tesla; spins are unit vectors (one per atom).
 *   arrays     row-major, caller atom order: positions[n][3], spins[n][3] ...
 *   ownership  the caller owns every array it passes; the library copies inputs
 *              in and copies outputs out in caller order before returning.
 *              The library owns all device memory of a system.
 *   threads    a system may be used from one host thread at a time.
 *   errors     every int-returning call returns SL_OK (0) or a negative code;
 *              sl_last_error() gives a message for the calling thread.  No C++
 *              exception crosses the ABI.
 */
#ifndef SPINLAT_H
#define SPINLAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SL_OK 0
#define SL_EINVAL (-1)          /* bad argument (shape, size, box, parameter)      */
#define SL_ENOMEM (-2)          /* device or host allocation failed                */
#define SL_ENBR_OVERFLOW (-3)   /* a neighbour list outgrew its capacity           */
#define SL_ENONFINITE (-4)      /* a force or field became NaN/Inf                 */
#define SL_ETIMEOUT (-5)        /* a bounded device wait gave up                   */
#define SL_ECUDA (-6)           /* CUDA runtime error or no usable device          */
#define SL_EINTERNAL (-7)       /* a self-check of the library failed              */

#define SL_PREC_FP64 0          /* everything in FP64                               */
#define SL_PREC_MIXED 1         /* FP32 descriptors/backward, FP16 tensor-core MLP, */
                                /* FP64 state, accumulation and renormalisation     */

typedef struct sl_system sl_system;

/* NEP-SPIN model.  Shapes supported by the kernels: n_species = 2, n_ch = 5,
 * basis_k = 9 (basis size 8, Section 5.2.4), l_max = 4, n_hidden = 30, which gives
 * the 66-entry descriptor of Section 5.2.3.  Layouts:
 *   coeffs   [n_species][n_species][6][n_ch][basis_k]: [centre][neighbour species],
 *            group order R, A, EX, DMI, ANI, SIA (structural radial, structural
 *            angular, and the four pairwise magnetic sub-terms of Section 5.2.4)
 *   q_scaler [66]; w0 [n_hidden][66]; b0 [n_hidden]; w1 [n_hidden]
 *   descriptor order R(5), A(n,l)(20), O(1), EX(5), DMI(5), ANI(5), SIA(5), SA(n,l)(20)
 * E_i = sum_h w1_h tanh(sum_v w0_hv q_scaler_v q_v - b0_h) - b1. */
typedef struct {
    int32_t n_species, n_ch, l_max, basis_k;
    double rc_rad, rc_ang;           /* radial and angular cutoffs, A (rc_ang <= rc_rad) */
    int32_t n_hidden;
    const double *coeffs, *q_scaler, *w0, *b0, *w1;
    double b1;
    const double *mass_amu;          /* [n_species] */
    const double *moment_muB;        /* [n_species] magnetic moment, Bohr magnetons */
} sl_nep_params;

typedef struct {
    int32_t precision;               /* SL_PREC_FP64 or SL_PREC_MIXED                  */
    uint64_t seed;                   /* Philox key word 0 (noise)                      */
    uint64_t replica;                /* Philox key word 1 (independent replicas)       */
    double skin;                     /* neighbour skin, A (rebuild at skin/2 motion)  */
    double gamma_lattice_per_fs;     /* lattice Langevin friction                      */
    double lambda_spin;              /* Gilbert damping of the stochastic spin update  */
    int32_t midpoint_iters;          /* 0: predictor-corrector spin update; 1..64: cap of the
                                        self-consistent midpoint iteration (Section 5.1.3)  */
    int32_t nbr_cap_rad;             /* radial list capacity (candidates within rc_rad+skin) */
    int32_t nbr_cap_ang;             /* angular list capacity (within rc_ang+skin)      */
    int32_t steps_per_graph;         /* steps captured in one CUDA graph (0: no graphs) */
    void *cuda_stream;               /* cudaStream_t to run on; NULL: a library stream  */
    int32_t device;                  /* CUDA device ordinal; -1: the calling thread's current device */
    double midpoint_tol;             /* stop the midpoint iteration when every spin moved
                                        less than this between iterates (0: run the cap)   */
    int32_t anderson_depth;          /* 0: plain fixed-point iteration; 1..8: history of the
                                        regularised Anderson-accelerated iteration          */
    double anderson_reg;             /* Tikhonov weight of the Anderson least-squares
                                        problem, relative to its mean diagonal              */
} sl_options;

/* Self-consistent midpoint spin update (midpoint_iters > 0; Section 5.1.3).  The
 * lattice part of the step is unchanged.  With r_mid = (r_n + r_{n+1})/2 and
 * X_0 = Rot(S_n, omega(S_n, H_n + eta) dt), iteration m forms the midpoint spins
 * M_m = (S_n + X_m)/|S_n + X_m|, evaluates the field at (r_mid, M_m), applies
 * G_m = Rot(S_n, omega(M_m, H_m + eta) dt) and stops when max_i |G_m - X_m| <
 * midpoint_tol or at the cap; S_{n+1} = G_m, and forces and fields are evaluated at
 * (r_{n+1}, S_{n+1}) for the final kick.  X_{m+1} = G_m, or with anderson_depth > 0
 * the Anderson mix X_{m+1} = G_m - dG g, (dF^T dF + reg tr/k I) g = dF^T f_m over the
 * last k + 1 residuals f = G - X, spins renormalised.  Costs one evaluation per
 * iteration plus one; SL_ENBR_OVERFLOW also reports a midpoint configuration beyond
 * the lists' skin. */

/* Fill *opt with the defaults: FP64, seed 1234, replica 0, skin 1 A, gamma 0.01/fs,
 * lambda 0.1, caps 160/64, 10 steps per graph, library stream, current device,
 * predictor-corrector spin update (midpoint_iters 0, tol 0, Anderson depth 0,
 * regularisation 1e-10). */
void sl_default_options(sl_options *opt);

/* Create a system of n atoms on the current CUDA device.
 *   positions [n][3] A (wrapped into the box along periodic dims on entry)
 *   spins     [n][3] (normalised on entry)
 *   box[3]    orthorhombic lengths, A; along a periodic dim it must be at least
 *             2 (rc_rad + skin); along a free dim it is the binning extent
 *   periodic[3] 0/1;  species [n] in [0, n_species)
 *   velocities [n][3] A/fs, or NULL for zero
 * Forces and fields of the initial state are evaluated before returning.
 * Returns SL_OK and *out, or an error (nothing allocated on error). */
int sl_create_system(const double *positions, const double *spins, const double box[3],
                     const int32_t periodic[3], const int32_t *species, int64_t n,
                     const double *velocities, const sl_nep_params *params,
                     const sl_options *opt, sl_system **out);

/* Advance n_steps steps of dt fs at temperature T_K and field B_tesla[3]
 * (Section 5.1.3 ordering: lattice update first, spin update last).  One step:
 *   v += dt/2 F/m; r += dt/2 v; Langevin O-step on v; r += dt/2 v;
 *   spin predictor S' = Rot(S, omega(S, H + eta) dt);  F', H' at (r, S');
 *   corrector S = Rot(S, (omega(S, H + eta) + omega(S', H' + eta)) dt/2), renormalised;
 *   v += dt/2 F'/m;  (F, H) = (F', H').
 * omega(S, X) = (X + lambda S x X) / ((1 + lambda^2) hbar), eta the thermal field.
 * On SL_ENBR_OVERFLOW or SL_ENONFINITE the state is restored to that at entry. */
int sl_step(sl_system *sys, int64_t n_steps, double dt_fs, double T_K, const double B_tesla[3]);

/* Evaluate the potential at the current (positions, spins) with the field of the
 * last sl_step (zero before any step).  energy_eV: E = sum_i E_i - sum_i mu_i muB B.S_i;
 * forces [n][3] eV/A; fields [n][3] eV = -dE/dS_i (Zeeman included); virial [9] eV
 * (W_ab = -sum_i sum_j (r_ij)_a dE_i/d(r_ij)_b).  Any output may be NULL.
 * Does not change the dynamical state. */
int sl_energy_forces_fields(sl_system *sys, double *energy_eV, double *forces, double *fields,
                            double *virial);

/* Per-atom descriptors q [n][66] (unscaled) and network energies E_i [n], caller
 * order; either may be NULL.  Evaluated at the current state. */
int sl_get_descriptors(sl_system *sys, double *q, double *atom_energy);

/* Copy the state out (any pointer may be NULL), all [n][3] in caller order.
 * forces/fields are the carried values of the integrator (evaluated at the last
 * predicted spins); ref_positions are the positions the current neighbour lists
 * were built from (they fix the list segments and so the summation order). */
int sl_get_state(const sl_system *sys, double *positions, double *velocities, double *spins,
                 double *forces, double *fields, double *ref_positions, uint64_t *step);

/* Replace the state.  positions/velocities/spins may not be NULL.  If forces and
 * fields are both given they become the carried integrator values; if both are
 * NULL they are re-evaluated at the new state.  Spins off unit length by more than
 * rounding are normalised (not in the longitudinal mode, sl_set_longitudinal).  ref_positions (may be NULL): the
 * lists are rebuilt from these positions instead of the new ones.  Given the
 * forces, fields and ref_positions of sl_get_state, the continued trajectory is
 * bit-identical to the uninterrupted one, in this or in any other system. */
int sl_set_state(sl_system *sys, const double *positions, const double *velocities,
                 const double *spins, const double *forces, const double *fields,
                 const double *ref_positions, uint64_t step);

/* Neighbour candidate lists of the current build, caller indices, ascending:
 * counts_rad[n], lists_rad[n][cap] (d2 < (rc_rad+skin)^2) and counts_ang[n],
 * lists_ang[n][cap] (d2 < (rc_ang+skin)^2).  Rebuilds the lists first. */
int sl_get_neighbors(sl_system *sys, int32_t cap, int32_t *counts_rad, int32_t *lists_rad,
                     int32_t *counts_ang, int32_t *lists_ang);

/* Device bytes a system of n atoms with these options will allocate (for admission
 * control by callers that pack replicas into free device memory). */
int64_t sl_estimate_device_bytes(int64_t n, const sl_options *opt);

/* Number of atoms, precision mode, neighbour-list builds so far (device-triggered
 * rebuilds included) and kernels launched by sl_step/sl_step_profiled so far. */
int sl_get_info(const sl_system *sys, int64_t *n_atoms, int32_t *precision, int64_t *n_builds,
                int64_t *n_launches);

/* Per-atom part of the external field: B_atoms [n][3] in tesla, caller atom order,
 * copied in; the field on atom i is then B (the sl_step argument) + B_atoms[i], in
 * the Zeeman energy -mu_i mu_B B_i.S_i, the fields and the energy.  NULL removes it.
 * The paper's production protocol uses a field that steps along x (Fig. 7).
 * SL_EINVAL for a non-finite entry. */
int sl_set_atom_fields(sl_system *sys, const double *B_atoms);

/* Longitudinal moment mode (the paper's integrator includes longitudinal fluctuation of
 * the magnetic moments, Section 3; it prints no equation, so this follows the Langevin
 * form with longitudinal damping of Ma and Dudarev, Phys. Rev. B 86, 054416, 2012).
 * With enable != 0 the spin lengths |S_i| become dynamical: the energy gains the Landau
 * onsite term sum_i a_t |S_i|^2 + b_t |S_i|^4 (landau: [n_species][2] = (a, b) in eV,
 * NULL for none; it also enters -dE/dS and the energy of sl_energy_forces_fields), the
 * spin equation is dS/dt = (H/hbar) x S + (alpha/hbar) H + xi with <xi xi> = 2 alpha kB T/hbar
 * (stationary density exp(-E/kT) over R^3), and each step is the predictor-corrector:
 *   S* = Rot(S, H dt/hbar) + alpha dt/hbar H + s zeta,
 *   S_next = Rot(S, (H + H*) dt/(2 hbar)) + alpha dt/hbar (H + H*)/2 + s zeta,
 * s = sqrt(2 alpha kB T dt/hbar), zeta the spin stream's normals, no renormalisation;
 * the options' lambda_spin is not used.  sl_set_state keeps the given spin lengths.
 * enable = 0 returns to unit spins (each spin is normalised; a spin of zero length gives
 * SL_ENONFINITE).  The carried forces and fields are re-evaluated.  SL_EINVAL for
 * alpha < 0, a non-finite coefficient, or a system created with midpoint_iters > 0. */
int sl_set_longitudinal(sl_system *sys, int32_t enable, double alpha, const double *landau);

/* Coloured Suzuki-Trotter spin sweep (a splitting of the spin update into classes of spins
 * that do not see each other's fields; the paper integrates with the predictor-corrector and
 * the midpoint iteration of Section 5.1.3, this is the coloured variant of that spin update).
 * With enable != 0, each sl_step step keeps the lattice part and replaces the spin
 * predictor-corrector by: colour the atoms at the new positions (atoms closer than 2 rc_rad
 * conflict, because the field on a spin depends on every spin within 2 rc_rad through the
 * neighbours' descriptors; greedy colouring in caller index order, the smallest colour unused
 * by conflicting atoms of lower index), then for c = 0..C-1 and back C-1..0 evaluate the
 * field at the current spins and rotate every spin of colour c by half a step,
 * S <- Rot(S, omega(S, H + eta) dt/2), renormalised, with the step's thermal field eta; then
 * forces and fields at the new state and the final lattice kick.  2C + 1 evaluations per
 * step, driven from the host (no graph capture).  SL_EINVAL with the midpoint or the
 * longitudinal mode; batches and sl_step_profiled refuse systems in this mode. */
int sl_set_spin_sweep(sl_system *sys, int32_t enable);

/* The colouring of the last coloured step: colours [n] in caller order (may be NULL; then no
 * device copy), the number of colours and the evaluations made by coloured steps so far.
 * SL_EINVAL for colours != NULL before any coloured step. */
int sl_get_sweep_colours(const sl_system *sys, int32_t *colours, int32_t *n_colours, int64_t *evaluations);

/* Texture diagnostics of a film with normal normal_axis (0, 1, 2), computed on the
 * device at the current state (Fig. 7 and Section 8 follow helix and skyrmion textures
 * in a thin stripe).  The two in-plane axes a < b are cut into n_a = max(1, floor(L_a /
 * cell)) and n_b cells (atoms beyond a non-periodic edge go to the edge cell);
 * m [n_b][n_a][3] (may be NULL) receives the normalised spin sum of every column (zero
 * for an empty column) and Q (may be NULL) the Berg-Luescher lattice topological charge:
 * every plaquette gives two counter-clockwise triangles, each contributing its signed
 * solid angle 2 atan2(m1.(m2 x m3), 1 + m1.m2 + m2.m3 + m3.m1); Q = sum / 4 pi, plaquettes
 * wrapping across periodic in-plane axes only.  With m and Q both NULL only n_a, n_b
 * are returned.  Results are deterministic.  SL_EINVAL for a bad axis or cell, or more
 * than 2^28 cells. */
int sl_texture_map(sl_system *sys, int32_t normal_axis, double cell, int32_t *n_a, int32_t *n_b, double *m,
                   double *Q);

/* Autotuner of the evaluation kernels' launch shapes (atoms per block of the radial,
 * angular and backward kernels, and in mixed precision their register budgets, i.e. the
 * resident blocks per SM the compiled kernel is held to; persistent CTAs per SM of the
 * tensor-core network).
 * Times the candidate shapes with CUDA events over `repeats` evaluations of the current
 * state (which it leaves unchanged), keeps the fastest shape per kernel for this system
 * and for later systems of the process on the same device, precision and size (a
 * power-of-two bucket of n).  The per-atom arithmetic does not depend on the shapes, so
 * results are bit-identical with any choice.  chosen [4] (may be NULL): radial block,
 * angular block, backward block (threads), network CTAs per SM; eval_ms_before/after
 * (may be NULL): summed median time of the four kernel groups with the previous and the
 * chosen shapes.  SL_EINVAL for repeats outside [1, 1000]. */
int sl_autotune(sl_system *sys, int32_t repeats, int32_t *chosen, double *eval_ms_before, double *eval_ms_after);

/* The evaluation kernels' current launch configuration, cfg[8]: radial block (threads),
 * radial register budget (0: default of 4 blocks per SM, 3: 3 blocks per SM), angular
 * block, angular budget (0: default of 4 blocks per SM, 1: unconstrained), backward block,
 * backward budget (0: default of 4 blocks per SM, 3: 3 blocks per SM), network CTAs per
 * SM, 0.  landscape
 * [16] (may be NULL): the last sl_autotune's median ms of the radial, angular, network and
 * backward kernels under each of its 4 candidate shapes (candidate-major; -1 where not
 * timed: never tuned, or FP64 mode, which has 2 candidates).  Candidates: 0 half blocks and
 * 1 network CTA, 1 full blocks and 2 CTAs, 2 and 3 the same with the register-budget
 * variants.  SL_EINVAL for NULL sys or cfg. */
int sl_get_launch_config(const sl_system *sys, int32_t *cfg, double *landscape);

/* Midpoint evaluations executed by all steps so far (0 in the predictor-corrector
 * mode); the mean iteration count per step is this over the steps taken. */
int sl_get_midpoint_evaluations(const sl_system *sys, int64_t *evaluations);

/* Kernels (or kernel groups) timed by sl_step_profiled, in step order. */
#define SL_K_FIRST_HALF 0    /* kicks, drifts, Langevin, spin predictor, rebuild test     */
#define SL_K_REBUILD 1       /* binning + lists + reverse slots (early exit when not due) */
#define SL_K_COMPACT 2       /* empty: the compaction runs inside the radial kernel       */
#define SL_K_RAD_FWD 3       /* in-cutoff compaction + radial and pairwise-magnetic sums  */
#define SL_K_ANG_FWD 4       /* angular and spin-angular channels                         */
#define SL_K_NETWORK 5       /* per-atom network and its input gradient                   */
#define SL_K_BACKWARD 6      /* backward to pair records, per-atom sums                   */
#define SL_K_SECOND_HALF 7   /* gather, spin corrector or midpoint iteration, final kick  */
#define SL_NKERNELS 8

/* Same as sl_step but without CUDA graphs and with CUDA events recorded on the
 * system's stream between the kernel groups; kernel_ms[SL_NKERNELS] receives the
 * summed device time of each group over the n_steps steps. */
int sl_step_profiled(sl_system *sys, int64_t n_steps, double dt_fs, double T_K, const double B_tesla[3],
                     double *kernel_ms);

/* FMA throughput of the current device in FLOP/s (an FMA counts 2), measured with
 * dependent-chain FMA kernels on every SM: precision SL_PREC_FP64 (FP64 pipe) or
 * SL_PREC_MIXED (FP32 pipe).  Used as the ALU roofline of the descriptor kernels. */
int sl_measure_fma_peak(int32_t precision, double *flops_per_s, double *elapsed_ms);

/* Stream the system's work is ordered on (a cudaStream_t). */
void *sl_get_stream(const sl_system *sys);

void sl_destroy_system(sl_system *sys);

/* Message of the last error on the calling thread ("" if none). */
const char *sl_last_error(void);

/* ---------------------------------------------------------------- batches
 * Independent replicas (temperature/field sweeps) stepped together, in a fixed number of
 * slots.  Replicas keep their own state, RNG key and neighbour lists; a replica's trajectory
 * is bit-identical alone and in a batch, whatever else the batch holds.
 *
 * When the replicas taking part in a call share the device and the model parameters and none
 * uses the midpoint iteration, they take the fused step: each kernel of the step is ONE
 * launch over every replica (a persistent grid walking a device table of per-slot argument
 * blocks; a replica's blocks are those of its own launches).  A one-block plan kernel at the
 * start of every step builds the step's work maps from per-slot budgets of steps left, so
 * replicas with different step counts share the launches until each budget is spent, and the
 * two captured graphs (steps_per_graph steps, one step) survive admissions and retirements:
 * sl_batch_set rewrites a slot's table entry and the grids of the graphs' one-item-per-block
 * kernels, not the graphs themselves (up to the atom capacity, see sl_batch_reserve).  Otherwise the replicas run on their own streams (one fork/join graph
 * when every occupied slot takes part).
 *
 * A system must leave every batch (sl_batch_set(b, slot, NULL)) before it is destroyed.  All
 * systems of a batch share the precision mode; the coloured sweep steps alone. */
typedef struct sl_batch sl_batch;

/* k slots (1 <= k <= 4096); systems[i] may be NULL (an empty slot); no system in two slots. */
int sl_batch_create(sl_system *const *systems, int32_t k, sl_batch **out);
/* Put sys into slot (NULL: empty the slot).  SL_EINVAL for a slot outside [0, k), a precision
 * mode other than the occupied slots', or a system that already holds another slot. */
int sl_batch_set(sl_batch *b, int32_t slot, sl_system *sys);
/* n_steps[k]: steps each slot's replica takes in this call (0 = idle; must be 0 for an empty
 * slot); dt/T/B per slot.  Returns after every replica's steps are done; on a list overflow or a
 * non-finite value the failing replicas go back to their state before the call, the others
 * keep their steps, and the first error is returned. */
int sl_batch_step(sl_batch *b, const int64_t *n_steps, const double *dt_fs, const double *T_K,
                  const double *B_tesla /* [k][3] */);
/* sl_batch_step in two halves: submit queues the call's steps on the device and returns at
 * once; wait finishes them (status, restores, step counters) and returns the first error.
 * Between the two, the replicas taking part must not be used and their slots not changed
 * (SL_EINVAL); empty slots may be filled, and other systems created and used, meanwhile.
 * A second submit before the wait is SL_EINVAL; wait with nothing in flight is SL_OK. */
int sl_batch_submit(sl_batch *b, const int64_t *n_steps, const double *dt_fs, const double *T_K,
                    const double *B_tesla /* [k][3] */);
int sl_batch_wait(sl_batch *b);
/* Number of graph launches of the batch stream (fused graphs, or fork/join graphs that
 * advanced every replica together by steps_per_graph steps). */
int sl_batch_graph_launches(const sl_batch *b, int64_t *launches);
/* stats[7]: graph launches, captures of the fused graphs, fused steps executed (each advances
 * every replica with budget left by one step), kernel launches queued by the batch's calls,
 * calls that took the fused step, calls that ran the replicas on their own streams, and the
 * atom capacity the fused launches are sized for. */
int sl_batch_stats(const sl_batch *b, int64_t *stats);
/* Size the fused launches for up to `atoms` atoms over all slots (default: 65,536, raised to
 * the next power of two whenever the slots' atoms exceed it).  The captured graphs survive
 * every admission and retirement up to the capacity; growing it captures them again.  The
 * kernels of the step that take one work item per block launch only the occupied slots'
 * blocks: an admission or retirement resizes their grids in the captured graphs, so a
 * capacity above the resident atoms costs no idle blocks.  SL_EINVAL for a negative count. */
int sl_batch_reserve(sl_batch *b, int64_t atoms);
void sl_batch_destroy(sl_batch *b);

/* ---------------------------------------------------------------- no device allocation
 * Per-atom descriptors and network energies of a small system, for callers that
 * cannot allocate device memory: plugins of simulation engines that hand every
 * device byte to their own pool allocator (a cudaMalloc behind the pool's back would
 * break its accounting or fail against its reservation), and real-time loops that
 * cannot take the device-wide synchronisation cudaMalloc and cudaFree may imply.
 * The paper has no counterpart; this is a service of this library.
 *   positions4, spins4  DEVICE arrays [n][4] of double (x, y, z, unused)
 *   species             DEVICE array [n] of int32
 *   q                   DEVICE output [n][66] (unscaled descriptors) or NULL
 *   atom_energy         DEVICE output [n] (E_i of the network)
 *   box, periodic, params  host values as for sl_create_system; along a periodic
 *                       dim the box must be at least 2 rc_rad
 *   cuda_stream         cudaStream_t the work is ordered on (NULL: default stream);
 *                       the call returns after the stream has drained
 * FP64 throughout, no neighbour skin (an exact all-pairs search inside rc_rad).
 * The scratch (about 6.3 MB: lists, descriptor columns, angular sums, a status
 * word) is one fixed array compiled into the library, resident on every GPU that
 * loads it until the process exits.  No call allocates device memory; n above
 * 2048 atoms returns SL_EINVAL, more than 160 neighbours inside rc_rad returns
 * SL_ENBR_OVERFLOW, and a species value outside [0, n_species) (checked on the
 * device, where the array lives) returns SL_EINVAL.  The first call on a device
 * looks up the array's device address (and may load the library's device code);
 * make that first call before any stream capture.  Every call uses the same array, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race: serialise them. */
int sl_descriptors_energies_noalloc(const double *positions4, const double *spins4, const int32_t *species,
                                    int64_t n, const double box[3], const int32_t periodic[3],
                                    const sl_nep_params *params, double *q, double *atom_energy,
                                    void *cuda_stream);

/* ---------------------------------------------------------------- self checks
 * Host-only checks of the kernels' compile-time tables (no GPU needed):
 * max |P_l(u.v) - sum_m kappa_lm p_lm(u) p_lm(v)| and the max finite-difference
 * error of the harmonic gradients over n_samples random unit vectors. */
int sl_selftest_harmonics(int32_t n_samples, double *max_addition_err, double *max_gradient_err);

/* Device self-test of the mixed-precision radial carrier (Sections 5.2.3-5.2.4): the FP32
 * basis f_k(r) and df_k/dr, whose cutoff factor is evaluated from Taylor polynomials of sin
 * and cos, against the FP64 basis (the CUDA library's sincospi) at n_samples radii evenly
 * spread over [0, rc).  Outputs the largest absolute differences divided by the largest
 * FP64 magnitudes.  SL_EINVAL for n_samples < 1 or rc <= 0; SL_ECUDA without a device. */
int sl_selftest_carrier(int32_t n_samples, double rc, double *max_rel_err_f, double *max_rel_err_df);

/* Device self-test of the bounded waits the tensor-core network kernel uses: one thread waits
 * on a shared-memory mbarrier that nothing arrives at, gives up after max_polls polls and
 * raises the timeout status bit, which the host reads.  Returns SL_ETIMEOUT (the expected
 * outcome, the device and context stay usable), SL_OK if the wait completed, SL_EINVAL for
 * max_polls outside [1, 2^22], SL_ECUDA without a device. */
int sl_selftest_bounded_wait(int32_t max_polls);

#ifdef __cplusplus
}
#endif
#endif /* SPINLAT_H */
