// sl_internal.h -- host-side system object and kernel launchers (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sl_common.cuh"

namespace sl {

// Per-call integrator constants, written by the host before each batch of
// steps and read by the kernels (so one captured graph serves any dt, T, B).
struct StepDev {
    double dt, half_dt;
    double c_fric;              // exp(-gamma dt)
    double sig_v[NS];           // sqrt((1 - c^2) kB T ACC / m)
    double acc_m[NS];           // ACC / m  (force -> acceleration)
    double sig_eta;             // sqrt(2 lambda kB T hbar / dt)
    double lambda;              // Gilbert damping
    double wscale;              // 1 / ((1 + lambda^2) hbar)
    double zee[NS][3];          // mu_t muB B  (Zeeman field per species)
    double mom[NS];             // mu_t muB (scales the per-atom field part)
    double disp2;               // (skin/2)^2, rebuild threshold
    // longitudinal mode (variable moment lengths): precession about H/hbar (lambda = 0,
    // sig_eta = 0 above), plus the drift alpha dt/hbar H and the additive noise lng_sig zeta;
    // no renormalisation.  landau: (a, b) of the onsite energy a|S|^2 + b|S|^4 per species.
    int lng;
    double lng_drift;           // alpha dt / hbar
    double lng_sig;             // sqrt(2 alpha kB T dt / hbar)
    double landau[NS][2];
    // coloured spin sweep: the first half leaves the spins alone (they are advanced by the
    // sweep over colour classes at the new positions)
    int sts;
};

// Device control block of the self-consistent midpoint iteration.
constexpr int MID_MAX_ITERS = 64;    // largest accepted iteration cap
constexpr int AA_MAX_DEPTH = 8;      // largest accepted Anderson history
struct MidDev {
    int converged;                                   // set once the step's iteration has stopped
    int fallback;                                    // Anderson solve unusable this iteration
    unsigned long long resid[MID_MAX_ITERS];         // max_i |G_i - X_i| per iteration (FP64 bits)
    unsigned long long iters;                        // midpoint evaluations executed, all steps
    double gamma[AA_MAX_DEPTH];                      // Anderson coefficients of the current iteration
};

// Launch shapes of the evaluation kernels, chosen by sl_autotune (the defaults below
// otherwise).  The per-atom arithmetic does not depend on them, so results are the same
// for every choice.
struct LaunchCfg {
    int crad_block = 128;      // threads per block of k_crad (one atom per thread)
    int ang_block = 0;         // threads per block of k_ang_fwd (four per atom); 0: the precision's default
    int bwd_block = 0;         // threads per block of k_bwd
    int mlp_ctas_per_sm = 2;   // persistent CTAs per SM of the tensor-core network
    // register budgets of the mixed-precision kernels, as the minimum resident blocks per SM
    // the compiler holds the allocation to (0: the kernel's default budget)
    int crad_minb = 0;         // 0 (4 blocks: 128 registers) or 3 (3 blocks)
    int ang_minb = 0;          // 0 (4 blocks: 128 registers) or 1 (unconstrained)
    int bwd_minb = 0;          // 0 (4 blocks: 128 registers) or 3 (3 blocks)
};

// Where an evaluation reads positions and spins (null: the state arrays) and an
// optional device flag that makes the evaluation kernels return at once.
struct EvalAt {
    const double4 *pos = nullptr, *spin = nullptr;
    const float4 *posf = nullptr, *spinf = nullptr;
    const int *skip = nullptr;
};

struct SoloTables;   // sl_batch.h

struct Cells {
    int nc[3];
    int ncell;
    int *count = nullptr, *start = nullptr, *fill = nullptr, *atoms = nullptr, *of = nullptr;
    float4 *posf = nullptr;    // cell-ordered FP32 positions (list build)
    uint32_t *key = nullptr;   // cell-ordered species << 30 | caller index
    int *sub = nullptr;        // [ncell][8] first position of each half-width sub-cell, relative to its cell
};

struct Sys {
    uint64_t uid = 0;          // unique in the process (a batch tells its slots' systems apart by it)
    int64_t n = 0;
    int prec = 0;
    uint64_t seed = 0, replica = 0;
    double skin = 1.0, gamma = 0.01, lambda = 0.1;
    int cap = 160, cap_ang = 64;
    int steps_per_graph = 10;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;

    NepDev<double> pd;
    NepDev<float> pf;
    double mass[NS], moment[NS];
    BoxDev<double> boxd;
    BoxDev<float> boxf;
    double box[3];
    int per[3];
    double cut_r2, cut_a2;     // (rc + skin)^2, radial and angular

    // state, internal atom order (species-major, then spatial cell order)
    double4 *pos = nullptr, *vel = nullptr, *spin = nullptr, *spin_prev = nullptr;
    double4 *F = nullptr, *H = nullptr, *posref = nullptr;
    float4 *posf = nullptr, *spinf = nullptr;
    int32_t *species = nullptr, *orig = nullptr, *inv = nullptr;
    int64_t n_fe = 0;          // atoms [0, n_fe) are species 0

    // neighbour lists, atom-major rows of nbr_stride(cap) entries: nbr (internal index of
    // each candidate), rev (slot of the atom in its candidate's list; cap <= 256, one byte) and
    // nbr_hash (an 8-bit hash of each candidate's index: the reverse-slot search's filter)
    int32_t *nbr = nullptr;
    uint8_t *rev = nullptr, *nbr_hash = nullptr;
    int4 *seg = nullptr;       // per atom: ends of (ang t0, ang t1, rad t0, rad t1)
    Cells cells;

    // evaluation buffers (element type = compute precision)
    void *q = nullptr;         // [DIM][qs]: descriptor v of atom i at v * qs + i
    int64_t qs = 0;            // row stride of q: n rounded up to a multiple of 4 (16-byte rows)
    CUtensorMap qmap;          // TMA map of q (mixed precision): [DIM] rows x n atoms, 128 x 66 boxes
    void *mlp_img = nullptr;   // the network weights as the tensor-core kernel's FP16 hi/lo operand images
    void *bsum = nullptr;      // [n][NLM][BREC] angular-sum records
    void *fp = nullptr;        // [DIM][n]
    void *ei = nullptr;        // [n]
    void *pairs = nullptr;     // [cap][n] pair records (see sl_eval2.cuh)
    int32_t *clj = nullptr;    // [cap_ang + cap][n] compact in-cutoff neighbours
    uint16_t *cls = nullptr;   // [cap_ang + cap][n] candidate slot | reverse slot << 8
    int4 *cnt = nullptr;       // [n] compact row counts
    uint32_t *cmask = nullptr; // [maskw][n] in-cutoff candidate slots (the gather's walk)
    int maskw = 0;             // ceil(cap / 32)
    void *fown = nullptr;      // [n] v4: sum_j dE_i/dr_ij
    void *gii = nullptr;       // [n] v4: dE_i/dS_i
    void *wpart = nullptr;     // [9][n] per-atom virial parts
    double4 *Fo = nullptr, *Ho = nullptr;   // evaluation outputs (not the carried F, H)

    // control
    int *status = nullptr;     // device status bits
    int *rebuild = nullptr;    // device rebuild flag
    unsigned long long *d_step = nullptr;   // [2]: current step, copy for the corrector
    StepDev *d_par = nullptr;
    StepDev *h_par = nullptr;  // pinned
    int *h_status = nullptr;   // pinned
    uint64_t step = 0;
    double B[3] = {0, 0, 0};
    int64_t n_builds = 0;      // builds requested by the host
    unsigned long long *d_builds = nullptr;   // builds executed on the device
    int64_t n_launches = 0;    // kernels launched by step calls
    double *red = nullptr;     // reduction scratch (device)
    double *h_red = nullptr;   // pinned
    // host side of state transfers: the internal -> caller order permutation (fixed at
    // creation) and a pinned staging buffer of n records, allocated on first use
    std::vector<int32_t> h_orig;
    mutable double4 *h_stage = nullptr;

    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    uint64_t capture_version = 0;   // bumped whenever a captured launch would read stale pointers
    // snapshot for error recovery
    double4 *snap = nullptr;   // 5 n: pos, vel, spin, F, H

    // the system's own argument tables of the step kernels (sl_batch.h)
    SoloTables *solo = nullptr;

    // set while launch_eval evaluates at the midpoint iteration's point (the system's tables
    // hold that point)
    EvalAt at;
    LaunchCfg cfg;
    // the last sl_autotune's measured landscape: median ms of the radial, angular, network and
    // backward kernels under each of its candidate shapes (-1: not timed)
    double tune_ms[4][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}};

    // per-atom part of the external field (tesla, internal order); null: uniform field only
    double4 *Bat = nullptr;

    // texture diagnostics scratch (sl_texture.cu), grown on demand
    unsigned long long *tex_acc = nullptr;
    double4 *tex_m = nullptr;
    double *tex_part = nullptr;
    int64_t tex_cells = 0;

    // longitudinal mode (sl_set_longitudinal) and the last step arguments, kept so the
    // integrator constants can be rebuilt when the mode changes between steps
    int lng = 0;
    double lng_alpha = 0.0;
    double landau[NS][2] = {{0, 0}, {0, 0}};
    double last_dt = 1.0, last_T = 0.0;

    // coloured Suzuki-Trotter spin sweep (sl_set_spin_sweep): colour of every atom (internal
    // order, device) for the current step, and the colour count of the last step
    int sts = 0;
    int32_t *colour = nullptr;
    int32_t last_colours = 0;
    int64_t sweep_evaluations = 0;

    // self-consistent midpoint spin update (mid_iters = 0: predictor-corrector)
    int mid_iters = 0, aa_depth = 0;
    double mid_tol = 0.0, aa_reg = 1e-10;
    double4 *posmid = nullptr;   // lattice midpoint of the step
    float4 *posmidf = nullptr;
    double4 *mids = nullptr;     // midpoint spins (evaluation point of the iteration)
    float4 *midsf = nullptr;
    double4 *mx = nullptr, *mg = nullptr;        // iterate X and its image G
    double4 *aax = nullptr, *aag = nullptr;      // Anderson rings [(depth + 1)][n]
    double *aapart = nullptr;                    // Anderson partial sums [AA_BLOCKS][...]
    MidDev *md = nullptr;
};

// the system's own argument tables (sl_batch.cu): written for its current buffers (not during
// a stream capture; 0 on success), and released
int solo_refresh(Sys &s);
void solo_free(Sys &s);

// launchers (sl_neighbors.cu)
// row stride of the atom-major caller-index copy of the lists: cap rounded up to a multiple
// of 4 entries, so every row starts on a 16-byte boundary
inline int nbr_stride(int cap) { return (cap + 31) & ~31; }   // byte rows of 32-byte multiples
void nbr_setup(Sys &s);
void launch_rebuild(Sys &s, bool conditional);
// sl_eval2.cu: the system's evaluation at the state (with the virial parts when asked for), or
// at the midpoint point while s.at is set; ev (optional, 6 events): recorded before the
// radial kernel, after it, after the angular kernel, the network and the backward.
void launch_eval(Sys &s, bool want_virial, cudaEvent_t *ev = nullptr);
void eval2_init();   // dynamic shared-memory limits of the evaluation kernels (once per device)
int default_quad_block(int prec);   // threads per block of the quad kernels by default
int make_q_tensor_map(Sys &s);                   // sl_mlp_tc.cu: the TMA map of s.q; 0 on success
int make_mlp_image(Sys &s);                      // sl_mlp_tc.cu: s.mlp_img from s.pf; 0 on success
// first half, rebuild group (7), compaction with radial forward, angular forward, network, backward,
// second half
constexpr int KERNELS_PER_STEP = 1 + 8 + 2 + 1 + 1 + 1;
// sl_integrate.cu
void launch_first_half(Sys &s);
void launch_second_half(Sys &s);
void launch_second_half_nospin(Sys &s);   // gather and final kick only (midpoint mode)
void launch_sweep_rotate(Sys &s, int c);  // coloured sweep: half-step rotation of the spins of colour c
// sl_midpoint.cu: the iteration of one step between the first half and the final evaluation;
// returns the number of kernels it queued
int launch_midpoint(Sys &s);
int midpoint_kernels_per_step(const Sys &s);
size_t midpoint_scratch_doubles();
// sl_texture.cu: film texture diagnostics (in-plane magnetisation map, topological charge)
int texture_grid(const Sys &s, int normal, double cell, int *na, int *nb);
cudaError_t launch_texture(Sys &s, int normal, double cell, double *h_m, double *Q);
void launch_gather(Sys &s, bool carried);
void launch_compare_bits(Sys &s, const double4 *ref, int *diff);   // *diff |= 1 if (Fo, Ho) != ref bitwise
void launch_normalise_spins(Sys &s);
int reduce_energy_virial(Sys &s, double *E, double *W, bool want_virial);

int launch_noalloc(const NepDev<double> &P, const double4 *pos, const double4 *spin, const int32_t *species, int n,
                   const BoxDev<double> &box, double *q_out, double *e_out, cudaStream_t stream, int *status_out);
int noalloc_max_atoms();
// sl_peak.cu
int measure_fma_peak(int precision, double *flops_per_s, double *elapsed_ms);
// FP32 carrier against FP64 at n radii in [0, rc): out = {max |df|, max |d(df/dr)|, max |f|, max |df/dr|}
int selftest_carrier(int n, double rc, double out[4]);
// sl_mlp_tc.cu: a bounded mbarrier wait on a barrier nothing arrives at; *status_out gets the device status bits
int selftest_bounded_wait(int limit, int *status_out);

}  // namespace sl
