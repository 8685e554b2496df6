// sl_integrate.cu -- spin-lattice integrator kernels, force/field gather, reductions.
//
// One step (arXiv 2606.14073, Sections 3, 5.1.3, 5.2.1; the paper gives no formulas,
// this is the structure-preserving predictor-corrector reading with the spin
// update scheduled last):
//   first half  (k_first_half):  v += dt/2 F/m; r += dt/2 v; v = c v + sig_v xi;
//                                r += dt/2 v (wrapped); eta = sig_eta zeta;
//                                S' = Rot(S, omega(S, H + eta) dt)
//   evaluation  at (r, S')  (sl_eval2.cu)
//   second half (k_second_half): gather F', H'; S = Rot(S, (omega(S,H+eta) + omega(S',H'+eta)) dt/2),
//                                renormalised in FP64; v += dt/2 F'/m; (F, H) = (F', H')
// omega(S, X) = (X + lambda S x X) / ((1 + lambda^2) hbar); Rot is the exact Rodrigues
// rotation.  Longitudinal mode (variable |S|, Section 3; Langevin form with longitudinal
// damping of Ma and Dudarev 2012): lambda = 0 and eta = 0 in the rotations, each spin
// update adds alpha dt/hbar H (predictor: H; corrector: (H + H')/2) and the additive noise
// sqrt(2 alpha kB T dt/hbar) zeta, and nothing is renormalised; the Landau onsite field
// -(2a + 4b|S|^2) S joins H wherever the Zeeman field does.  xi, zeta are Philox4x64-10 normals, streams 1 and 2, counter
// (step, caller index, stream, 0), key (seed, replica): the corrector regenerates
// the predictor's eta bit for bit, so nothing is stored between the halves.
#include "sl_internal.h"
#include "sl_eval2.cuh"
#include "sl_batch.h"
#include "sl_fused.cuh"
#include "sl_spin.cuh"

namespace sl {

struct IntArgs {
    double4 *pos, *vel, *spin, *spin_prev, *F, *H, *posref;
    float4 *posf, *spinf;
    double4 *posmid;    // non-null in the midpoint mode: lattice midpoint of the step
    float4 *posmidf;
    const double4 *Bat; // non-null: per-atom part of the external field (tesla)
    const int32_t *orig;
    int64_t n, n_fe;
    BoxDev<double> bd;
    int per[3];
    const StepDev *par;
    unsigned long long *step;
    int *rebuild, *status;
    uint64_t seed, replica;
};

// Landau onsite field -(2a + 4b|S|^2) S of atom i (species t), added to H.
__device__ __forceinline__ void add_landau(const StepDev &P, int t, const double4 S, double H[3]) {
    const double m2 = S.x * S.x + S.y * S.y + S.z * S.z;
    const double k = -(2.0 * P.landau[t][0] + 4.0 * P.landau[t][1] * m2);
    H[0] += k * S.x; H[1] += k * S.y; H[2] += k * S.z;
}



template <bool MIXED>
__device__ __forceinline__ void first_half_body(const IntArgs &a, int64_t blk) {
    const int64_t i = blk * (int64_t)blockDim.x + threadIdx.x;
    const unsigned long long st = a.step[0];
    if (i == 0) a.step[1] = st;
    if (i >= a.n) return;
    const StepDev &P = *a.par;
    const int t = i < a.n_fe ? 0 : 1;
    const uint64_t id = (uint64_t)a.orig[i];
    double4 r = a.pos[i], v = a.vel[i];
    const double4 F = a.F[i], H = a.H[i], S = a.spin[i];
    const double hdt = P.half_dt, am = P.acc_m[t];
    double xi[3], ze[3];
    if constexpr (MIXED) {
        float x3[3], z3[3];
        gauss3f(st, id, 1, a.seed, a.replica, x3);
        gauss3f(st, id, 2, a.seed, a.replica, z3);
        for (int c = 0; c < 3; ++c) { xi[c] = x3[c]; ze[c] = z3[c]; }
    } else {
        gauss3(st, id, 1, a.seed, a.replica, xi);
        gauss3(st, id, 2, a.seed, a.replica, ze);
    }
    const double4 r0 = r;
    v.x += hdt * F.x * am; v.y += hdt * F.y * am; v.z += hdt * F.z * am;
    r.x += hdt * v.x; r.y += hdt * v.y; r.z += hdt * v.z;
    const double c = P.c_fric, sv = P.sig_v[t];
    v.x = c * v.x + sv * xi[0]; v.y = c * v.y + sv * xi[1]; v.z = c * v.z + sv * xi[2];
    r.x += hdt * v.x; r.y += hdt * v.y; r.z += hdt * v.z;
    if (a.posmid) {   // lattice midpoint r0 + (r - r0)/2 of the unwrapped step, then wrapped
        double m3[3] = {r0.x + 0.5 * (r.x - r0.x), r0.y + 0.5 * (r.y - r0.y), r0.z + 0.5 * (r.z - r0.z)};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (a.per[d]) m3[d] = m3[d] - a.bd.L[d] * floor(m3[d] * a.bd.invL[d]);
        a.posmid[i] = make_double4(m3[0], m3[1], m3[2], 0.0);
        a.posmidf[i] = make_float4((float)m3[0], (float)m3[1], (float)m3[2], 0.f);
    }
    if (a.per[0]) r.x = r.x - a.bd.L[0] * floor(r.x * a.bd.invL[0]);
    if (a.per[1]) r.y = r.y - a.bd.L[1] * floor(r.y * a.bd.invL[1]);
    if (a.per[2]) r.z = r.z - a.bd.L[2] * floor(r.z * a.bd.invL[2]);
    const double se = P.sig_eta;
    double Sp[3];
    if (P.sts) {   // coloured sweep: the spins are advanced at the new positions, colour by colour
        Sp[0] = S.x; Sp[1] = S.y; Sp[2] = S.z;
    } else if constexpr (MIXED) {
        float w[3], d[3];
        const float fse = (float)se;
        omega_of_f((float)S.x, (float)S.y, (float)S.z, (float)H.x + fse * (float)ze[0],
                   (float)H.y + fse * (float)ze[1], (float)H.z + fse * (float)ze[2], (float)P.lambda,
                   (float)P.wscale, w);
        rotate_delta_f((float)S.x, (float)S.y, (float)S.z, w[0], w[1], w[2], (float)P.dt, d);
        if (P.lng) {
            const float kd = (float)P.lng_drift, ks = (float)P.lng_sig;
            d[0] += kd * (float)H.x + ks * (float)ze[0];
            d[1] += kd * (float)H.y + ks * (float)ze[1];
            d[2] += kd * (float)H.z + ks * (float)ze[2];
        }
        Sp[0] = S.x + (double)d[0]; Sp[1] = S.y + (double)d[1]; Sp[2] = S.z + (double)d[2];
    } else {
        double w[3];
        omega_of(S.x, S.y, S.z, H.x + se * ze[0], H.y + se * ze[1], H.z + se * ze[2], P.lambda, P.wscale, w);
        rotate(S.x, S.y, S.z, w, P.dt, Sp);
        if (P.lng) {
            Sp[0] += P.lng_drift * H.x + P.lng_sig * ze[0];
            Sp[1] += P.lng_drift * H.y + P.lng_sig * ze[1];
            Sp[2] += P.lng_drift * H.z + P.lng_sig * ze[2];
        }
    }
    a.pos[i] = r;
    a.vel[i] = v;
    a.spin_prev[i] = S;
    a.spin[i] = make_double4(Sp[0], Sp[1], Sp[2], 0.0);
    a.posf[i] = make_float4((float)r.x, (float)r.y, (float)r.z, 0.f);
    a.spinf[i] = make_float4((float)Sp[0], (float)Sp[1], (float)Sp[2], 0.f);
    // rebuild trigger: displacement since the last build beyond skin/2
    const double4 p0 = a.posref[i];
    double dx = r.x - p0.x, dy = r.y - p0.y, dz = r.z - p0.z;
    minimg(a.bd, dx, dy, dz);
    if (dx * dx + dy * dy + dz * dz > P.disp2) *a.rebuild = 1;
}

// SPIN = false (midpoint mode): the spins were already advanced by the midpoint
// iteration; only the gather, the final kick and the carried F, H remain.
template <typename R, bool MIXED, bool SPIN = true>
__device__ __forceinline__ void second_half_body(const IntArgs &a, const GatherArgs<R> &g, int64_t blk) {
    const int64_t i = blk * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) a.step[0] = a.step[1] + 1;
    if (i >= a.n) return;
    const StepDev &P = *a.par;
    const int t = i < a.n_fe ? 0 : 1;
    const uint64_t id = (uint64_t)a.orig[i];
    const unsigned long long st = a.step[1];
    double Fs[3], Hs[3];
    gather<R>(g, i, Fs, Hs);
    Hs[0] += P.zee[t][0]; Hs[1] += P.zee[t][1]; Hs[2] += P.zee[t][2];
    if (a.Bat) {
        const double4 b = a.Bat[i];
        Hs[0] += P.mom[t] * b.x; Hs[1] += P.mom[t] * b.y; Hs[2] += P.mom[t] * b.z;
    }
    if (P.lng) add_landau(P, t, a.spin[i], Hs);
    if constexpr (!SPIN) {
        double4 v = a.vel[i];
        const double hdt = P.half_dt, am = P.acc_m[t];
        v.x += hdt * Fs[0] * am; v.y += hdt * Fs[1] * am; v.z += hdt * Fs[2] * am;
        a.vel[i] = v;
        a.F[i] = make_double4(Fs[0], Fs[1], Fs[2], 0.0);
        a.H[i] = make_double4(Hs[0], Hs[1], Hs[2], 0.0);
        if (!(isfinite(Fs[0]) && isfinite(Fs[1]) && isfinite(Fs[2]) && isfinite(Hs[0]) && isfinite(Hs[1]) &&
              isfinite(Hs[2])))
            atomicOr(a.status, ST_NONFINITE);
        return;
    }
    const double se = P.sig_eta;
    const double4 S0 = a.spin_prev[i], S1 = a.spin[i], H0 = a.H[i];
    double Sn[3];
    if constexpr (MIXED) {
        float ze[3], w0[3], w1[3], d[3];
        gauss3f(st, id, 2, a.seed, a.replica, ze);
        const float fse = (float)se, lam = (float)P.lambda, k = (float)P.wscale;
        omega_of_f((float)S0.x, (float)S0.y, (float)S0.z, (float)H0.x + fse * ze[0], (float)H0.y + fse * ze[1],
                   (float)H0.z + fse * ze[2], lam, k, w0);
        omega_of_f((float)S1.x, (float)S1.y, (float)S1.z, (float)Hs[0] + fse * ze[0], (float)Hs[1] + fse * ze[1],
                   (float)Hs[2] + fse * ze[2], lam, k, w1);
        rotate_delta_f((float)S0.x, (float)S0.y, (float)S0.z, 0.5f * (w0[0] + w1[0]), 0.5f * (w0[1] + w1[1]),
                       0.5f * (w0[2] + w1[2]), (float)P.dt, d);
        if (P.lng) {
            const float kd = (float)P.lng_drift, ks = (float)P.lng_sig;
            d[0] += kd * (0.5f * ((float)H0.x + (float)Hs[0])) + ks * ze[0];
            d[1] += kd * (0.5f * ((float)H0.y + (float)Hs[1])) + ks * ze[1];
            d[2] += kd * (0.5f * ((float)H0.z + (float)Hs[2])) + ks * ze[2];
        }
        Sn[0] = S0.x + (double)d[0]; Sn[1] = S0.y + (double)d[1]; Sn[2] = S0.z + (double)d[2];
    } else {
        double ze[3], w0[3], w1[3], w[3];
        gauss3(st, id, 2, a.seed, a.replica, ze);
        omega_of(S0.x, S0.y, S0.z, H0.x + se * ze[0], H0.y + se * ze[1], H0.z + se * ze[2], P.lambda, P.wscale, w0);
        omega_of(S1.x, S1.y, S1.z, Hs[0] + se * ze[0], Hs[1] + se * ze[1], Hs[2] + se * ze[2], P.lambda, P.wscale,
                 w1);
        w[0] = 0.5 * (w0[0] + w1[0]); w[1] = 0.5 * (w0[1] + w1[1]); w[2] = 0.5 * (w0[2] + w1[2]);
        rotate(S0.x, S0.y, S0.z, w, P.dt, Sn);
        if (P.lng) {
            Sn[0] += P.lng_drift * (0.5 * (H0.x + Hs[0])) + P.lng_sig * ze[0];
            Sn[1] += P.lng_drift * (0.5 * (H0.y + Hs[1])) + P.lng_sig * ze[1];
            Sn[2] += P.lng_drift * (0.5 * (H0.z + Hs[2])) + P.lng_sig * ze[2];
        }
    }
    if (!P.lng) {   // renormalisation in FP64 after every rotation
        const double inn = 1.0 / sqrt(Sn[0] * Sn[0] + Sn[1] * Sn[1] + Sn[2] * Sn[2]);
        Sn[0] *= inn; Sn[1] *= inn; Sn[2] *= inn;
    }
    double4 v = a.vel[i];
    const double hdt = P.half_dt, am = P.acc_m[t];
    v.x += hdt * Fs[0] * am; v.y += hdt * Fs[1] * am; v.z += hdt * Fs[2] * am;
    a.vel[i] = v;
    a.spin[i] = make_double4(Sn[0], Sn[1], Sn[2], 0.0);
    a.spinf[i] = make_float4((float)Sn[0], (float)Sn[1], (float)Sn[2], 0.f);
    a.F[i] = make_double4(Fs[0], Fs[1], Fs[2], 0.0);
    a.H[i] = make_double4(Hs[0], Hs[1], Hs[2], 0.0);
    if (!(isfinite(Fs[0]) && isfinite(Fs[1]) && isfinite(Fs[2]) && isfinite(Hs[0]) && isfinite(Hs[1]) &&
          isfinite(Hs[2])))
        atomicOr(a.status, ST_NONFINITE);
}

// The halves over an argument table (sl_batch.h: a system's own table or a batch's), one
// 256-thread block per 256 atoms of a slot.
template <typename R>
struct HalfArgs {
    IntArgs a;
    GatherArgs<R> g;
};
template <bool MIXED>
__global__ void __launch_bounds__(256) k_first_half(const IntArgs *__restrict__ tab, SlotMap sm,
                                                    const __grid_constant__ IntArgs solo) {
    one_work(tab, sm, solo, [](const IntArgs &a, int64_t blk, int64_t) { first_half_body<MIXED>(a, blk); });
}
template <typename R, bool MIXED, bool SPIN>
__global__ void __launch_bounds__(256) k_second_half(const HalfArgs<R> *__restrict__ tab, SlotMap sm,
                                                     const __grid_constant__ HalfArgs<R> solo) {
    one_work(tab, sm, solo,
             [](const HalfArgs<R> &h, int64_t blk, int64_t) { second_half_body<R, MIXED, SPIN>(h.a, h.g, blk); });
}

// Forces and fields at the current state into (Fo, Ho).
template <typename R>
__global__ void __launch_bounds__(256) k_gather_only(GatherArgs<R> g, const StepDev *par, int64_t n_fe,
                                                     double4 *Fo, double4 *Ho, int *status, const double4 *Bat,
                                                     const double4 *spin) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int t = i < n_fe ? 0 : 1;
    double Fs[3], Hs[3];
    gather<R>(g, i, Fs, Hs);
    Hs[0] += par->zee[t][0]; Hs[1] += par->zee[t][1]; Hs[2] += par->zee[t][2];
    if (Bat) {
        const double4 b = Bat[i];
        Hs[0] += par->mom[t] * b.x; Hs[1] += par->mom[t] * b.y; Hs[2] += par->mom[t] * b.z;
    }
    if (par->lng) add_landau(*par, t, spin[i], Hs);
    Fo[i] = make_double4(Fs[0], Fs[1], Fs[2], 0.0);
    Ho[i] = make_double4(Hs[0], Hs[1], Hs[2], 0.0);
    if (!(isfinite(Fs[0]) && isfinite(Fs[1]) && isfinite(Fs[2]) && isfinite(Hs[0]) && isfinite(Hs[1]) &&
          isfinite(Hs[2])))
        atomicOr(status, ST_NONFINITE);
}

// Coloured sweep sub-step: every spin of colour c is rotated by half a step about its
// field at the current configuration, S <- Rot(S, omega(S, H + eta) dt/2), renormalised in
// FP64; eta is the step's thermal field (the spin stream's normals of this step, as in the
// predictor-corrector).  The field is gathered from the pair records of the evaluation just
// made; spins of other colours are left alone.
template <typename R, bool MIXED>
__global__ void __launch_bounds__(256) k_sweep_rotate(IntArgs a, GatherArgs<R> g, const int32_t *colour, int c) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n || colour[i] != c) return;
    const StepDev &P = *a.par;
    const int t = i < a.n_fe ? 0 : 1;
    const uint64_t id = (uint64_t)a.orig[i];
    const unsigned long long st = a.step[1];
    double Fs[3], Hs[3];
    gather<R>(g, i, Fs, Hs);
    Hs[0] += P.zee[t][0]; Hs[1] += P.zee[t][1]; Hs[2] += P.zee[t][2];
    if (a.Bat) {
        const double4 b = a.Bat[i];
        Hs[0] += P.mom[t] * b.x; Hs[1] += P.mom[t] * b.y; Hs[2] += P.mom[t] * b.z;
    }
    const double4 S = a.spin[i];
    const double se = P.sig_eta;
    double Sn[3];
    if constexpr (MIXED) {
        float ze[3], w[3], d[3];
        gauss3f(st, id, 2, a.seed, a.replica, ze);
        const float fse = (float)se;
        omega_of_f((float)S.x, (float)S.y, (float)S.z, (float)Hs[0] + fse * ze[0], (float)Hs[1] + fse * ze[1],
                   (float)Hs[2] + fse * ze[2], (float)P.lambda, (float)P.wscale, w);
        rotate_delta_f((float)S.x, (float)S.y, (float)S.z, w[0], w[1], w[2], (float)P.half_dt, d);
        Sn[0] = S.x + (double)d[0]; Sn[1] = S.y + (double)d[1]; Sn[2] = S.z + (double)d[2];
    } else {
        double ze[3], w[3];
        gauss3(st, id, 2, a.seed, a.replica, ze);
        omega_of(S.x, S.y, S.z, Hs[0] + se * ze[0], Hs[1] + se * ze[1], Hs[2] + se * ze[2], P.lambda, P.wscale, w);
        rotate(S.x, S.y, S.z, w, P.half_dt, Sn);
    }
    const double inn = 1.0 / sqrt(Sn[0] * Sn[0] + Sn[1] * Sn[1] + Sn[2] * Sn[2]);
    Sn[0] *= inn; Sn[1] *= inn; Sn[2] *= inn;
    a.spin[i] = make_double4(Sn[0], Sn[1], Sn[2], 0.0);
    a.spinf[i] = make_float4((float)Sn[0], (float)Sn[1], (float)Sn[2], 0.f);
    if (!(isfinite(Hs[0]) && isfinite(Hs[1]) && isfinite(Hs[2]))) atomicOr(a.status, ST_NONFINITE);
}

static IntArgs int_args(Sys &s) {
    IntArgs a;
    a.pos = s.pos; a.vel = s.vel; a.spin = s.spin; a.spin_prev = s.spin_prev; a.F = s.F; a.H = s.H;
    a.posref = s.posref; a.posf = s.posf; a.spinf = s.spinf; a.orig = s.orig; a.n = s.n; a.n_fe = s.n_fe;
    a.bd = s.boxd;
    for (int d = 0; d < 3; ++d) a.per[d] = s.per[d];
    a.par = s.d_par; a.step = s.d_step; a.rebuild = s.rebuild; a.status = s.status;
    a.seed = s.seed; a.replica = s.replica;
    a.posmid = s.mid_iters > 0 ? s.posmid : nullptr;
    a.posmidf = s.mid_iters > 0 ? s.posmidf : nullptr;
    a.Bat = s.Bat;
    return a;
}

template <typename R>
static GatherArgs<R> gather_args(Sys &s) {
    GatherArgs<R> g;
    g.fown = (const v4<R> *)s.fown; g.gii = (const v4<R> *)s.gii; g.pd = (const PairRec<R> *)s.pairs;
    g.mask = s.cmask; g.maskw = s.maskw; g.n = s.n;
    return g;
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_first_half_t(const FusedTables &t, const Launch &L, cudaStream_t st) {
    const IntArgs *tab = L.solo ? nullptr : t.at<IntArgs>(t.o_first);
    const IntArgs so = solo_args<IntArgs>(L);
    if (t.prec == 0) k_first_half<false><<<L.grid, 256, 0, st>>>(tab, L.slots(), so);
    else k_first_half<true><<<L.grid, 256, 0, st>>>(tab, L.slots(), so);
}

template <typename R, bool MIXED>
static void second_half_t(const FusedTables &t, const Launch &L, bool spin, cudaStream_t st) {
    const HalfArgs<R> *tab = L.solo ? nullptr : t.at<HalfArgs<R>>(t.o_second);
    const HalfArgs<R> so = solo_args<HalfArgs<R>>(L);
    if (spin) k_second_half<R, MIXED, true><<<L.grid, 256, 0, st>>>(tab, L.slots(), so);
    else k_second_half<R, MIXED, false><<<L.grid, 256, 0, st>>>(tab, L.slots(), so);
}
void launch_second_half_t(const FusedTables &t, const Launch &L, bool spin, cudaStream_t st) {
    if (t.prec == 0) second_half_t<double, false>(t, L, spin, st);
    else second_half_t<float, true>(t, L, spin, st);
}

// a system's own launches, over its table
void launch_first_half(Sys &s) { launch_first_half_t(s.solo->t, solo_launch(s, FK_FIRST, SK_STEP), s.stream); }
void launch_second_half(Sys &s) {
    launch_second_half_t(s.solo->t, solo_launch(s, FK_SECOND, SK_STEP), true, s.stream);
}
void launch_second_half_nospin(Sys &s) {
    launch_second_half_t(s.solo->t, solo_launch(s, FK_SECOND, SK_STEP), false, s.stream);
}

void launch_sweep_rotate(Sys &s, int c) {
    if (s.prec == 0)
        k_sweep_rotate<double, false><<<nblk(s.n, 256), 256, 0, s.stream>>>(int_args(s), gather_args<double>(s),
                                                                            s.colour, c);
    else
        k_sweep_rotate<float, true><<<nblk(s.n, 256), 256, 0, s.stream>>>(int_args(s), gather_args<float>(s),
                                                                          s.colour, c);
}

void launch_gather(Sys &s, bool carried) {
    double4 *Fo = carried ? s.F : s.Fo, *Ho = carried ? s.H : s.Ho;
    if (s.prec == 0)
        k_gather_only<double><<<nblk(s.n, 256), 256, 0, s.stream>>>(gather_args<double>(s), s.d_par, s.n_fe, Fo, Ho,
                                                                    s.status, s.Bat, s.spin);
    else
        k_gather_only<float><<<nblk(s.n, 256), 256, 0, s.stream>>>(gather_args<float>(s), s.d_par, s.n_fe, Fo, Ho,
                                                                   s.status, s.Bat, s.spin);
}

// Sets *diff when the evaluation outputs (Fo, Ho) differ in any bit from ref ([n] forces,
// then [n] fields): the autotuner's check that launch shapes leave results unchanged.
__global__ void k_compare_bits(const double4 *__restrict__ Fo, const double4 *__restrict__ Ho,
                               const double4 *__restrict__ ref, int64_t n, int *diff) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 f = Fo[i], h = Ho[i], rf = ref[i], rh = ref[n + i];
    const bool same = __double_as_longlong(f.x) == __double_as_longlong(rf.x) &&
                      __double_as_longlong(f.y) == __double_as_longlong(rf.y) &&
                      __double_as_longlong(f.z) == __double_as_longlong(rf.z) &&
                      __double_as_longlong(h.x) == __double_as_longlong(rh.x) &&
                      __double_as_longlong(h.y) == __double_as_longlong(rh.y) &&
                      __double_as_longlong(h.z) == __double_as_longlong(rh.z);
    if (!same) atomicOr(diff, 1);
}

// ---- fused batch step (sl_batch.h)
void fused_half_sizes(int prec, size_t *first, size_t *second) {
    *first = sizeof(IntArgs);
    *second = prec == 0 ? sizeof(HalfArgs<double>) : sizeof(HalfArgs<float>);
}

void fused_put_half(Sys &s, int r, const FusedTables &t, unsigned char *img, int64_t *blocks) {
    const IntArgs a = int_args(s);
    reinterpret_cast<IntArgs *>(img + t.o_first)[r] = a;
    if (s.prec == 0) reinterpret_cast<HalfArgs<double> *>(img + t.o_second)[r] = HalfArgs<double>{a, gather_args<double>(s)};
    else reinterpret_cast<HalfArgs<float> *>(img + t.o_second)[r] = HalfArgs<float>{a, gather_args<float>(s)};
    blocks[FK_FIRST] = blocks[FK_SECOND] = nblk(s.n, 256);
}

void launch_compare_bits(Sys &s, const double4 *ref, int *diff) {
    if (s.n > 0) k_compare_bits<<<nblk(s.n, 256), 256, 0, s.stream>>>(s.Fo, s.Ho, ref, s.n, diff);
}

// Unit length for every spin (leaving the longitudinal mode), FP64.
__global__ void k_normalise_spins(double4 *spin, float4 *spinf, int64_t n, int *status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 S = spin[i];
    const double n2 = S.x * S.x + S.y * S.y + S.z * S.z;
    if (!(n2 > 0.0)) {
        atomicOr(status, ST_NONFINITE);
        return;
    }
    const double inn = 1.0 / sqrt(n2);
    spin[i] = make_double4(S.x * inn, S.y * inn, S.z * inn, 0.0);
    spinf[i] = make_float4((float)(S.x * inn), (float)(S.y * inn), (float)(S.z * inn), 0.f);
}

void launch_normalise_spins(Sys &s) {
    if (s.n > 0) k_normalise_spins<<<nblk(s.n, 256), 256, 0, s.stream>>>(s.spin, s.spinf, s.n, s.status);
}



// ------------------------------------------------------------------ reductions
// Deterministic two-level FP64 sums: fixed 256 blocks, each summing a fixed
// stride of atoms in order, then one block adding the block partials in order.
constexpr int RED_BLOCKS = 256;
constexpr int RED_VALS = 10;   // E_network + E_Zeeman, virial[9]

template <typename R>
__global__ void __launch_bounds__(256) k_reduce1(const R *__restrict__ ei, const R *__restrict__ wpart,
                                                 const double4 *__restrict__ spin, const StepDev *par, int64_t n,
                                                 int64_t n_fe, int want_virial, double *__restrict__ part,
                                                 const double4 *__restrict__ Bat) {
    __shared__ double sh[RED_VALS][256];
    double acc[RED_VALS];
#pragma unroll
    for (int v = 0; v < RED_VALS; ++v) acc[v] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int t = i < n_fe ? 0 : 1;
        const double4 S = spin[i];
        double ez = par->zee[t][0] * S.x + par->zee[t][1] * S.y + par->zee[t][2] * S.z;
        if (Bat) {
            const double4 b = Bat[i];
            ez += par->mom[t] * (b.x * S.x + b.y * S.y + b.z * S.z);
        }
        if (par->lng) {
            const double m2 = S.x * S.x + S.y * S.y + S.z * S.z;
            ez -= par->landau[t][0] * m2 + par->landau[t][1] * m2 * m2;
        }
        acc[0] += (double)ei[i] - ez;
        if (want_virial)
            for (int v = 0; v < 9; ++v) acc[1 + v] += (double)wpart[(int64_t)v * n + i];
    }
#pragma unroll
    for (int v = 0; v < RED_VALS; ++v) sh[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int v = 0; v < RED_VALS; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x < RED_VALS) part[blockIdx.x * RED_VALS + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_reduce2(const double *__restrict__ part, double *__restrict__ out) {
    if (threadIdx.x < RED_VALS) {
        double s = 0.0;
        for (int b = 0; b < RED_BLOCKS; ++b) s += part[b * RED_VALS + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

int reduce_energy_virial(Sys &s, double *E, double *W, bool want_virial) {
    double *part = s.red, *out = s.red + RED_BLOCKS * RED_VALS;
    if (s.prec == 0)
        k_reduce1<double><<<RED_BLOCKS, 256, 0, s.stream>>>((const double *)s.ei, (const double *)s.wpart, s.spin,
                                                            s.d_par, s.n, s.n_fe, want_virial, part, s.Bat);
    else
        k_reduce1<float><<<RED_BLOCKS, 256, 0, s.stream>>>((const float *)s.ei, (const float *)s.wpart, s.spin,
                                                           s.d_par, s.n, s.n_fe, want_virial, part, s.Bat);
    k_reduce2<<<1, 32, 0, s.stream>>>(part, out);
    cudaError_t e = cudaMemcpyAsync(s.h_red, out, sizeof(double) * RED_VALS, cudaMemcpyDeviceToHost, s.stream);
    if (e != cudaSuccess) return -1;
    e = cudaStreamSynchronize(s.stream);
    if (e != cudaSuccess) return -1;
    if (E) *E = s.h_red[0];
    if (W)
        for (int v = 0; v < 9; ++v) W[v] = s.h_red[1 + v];
    return 0;
}

}  // namespace sl
