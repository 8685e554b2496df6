// sl_nep.cu -- NEP-SPIN descriptor, network and backward kernels (one thread per atom).
//
// Descriptor of atom i (arXiv 2606.14073, Sections 5.1.1-5.1.2; 66 entries, Section 5.2.3):
//   R_n  = sum_j g^R_n(r_ij)                           radial, r < rc_rad
//   X_n  = sum_j g^X_n(r_ij) phi_X(S_i, S_j, u_ij)      X = EX, DMI, ANI, SIA (Section 5.2.4)
//   A_nl = sum_m kappa_lm B_nlm^2,   B_nlm  = sum_j g^A_n(r_ij) p_lm(u_ij)           r < rc_ang
//   SA_nl = sum_m kappa_lm BS_nlm^2, BS_nlm = sum_j g^A_n(r_ij) (S_i.S_j) p_lm(u_ij)
//   O = |S_i|^2
// with g^G_n = sum_k c^G_{n k t_i t_j} f_k (shared Chebyshev carrier, Section 5.2.4).
// The angular channels use the harmonic (addition-theorem) form: one pass over
// neighbours per channel n instead of the pair double sum.
//
// Three kernels:
//   k_fwd   q[66][n] and the 240 angular sums B, BS (kept for the backward);
//   k_mlp   E_i and Fp = dE_i/dq_i (CUDA-core version; the tensor-core one is in sl_mlp_tc.cu);
//   k_bwd   per neighbour slot: dE_i/dr_ij and dE_i/dS_j, and per atom sum_j dE_i/dr_ij,
//           dE_i/dS_i and the virial part -sum_j r_ij (x) dE_i/dr_ij.
// Forces and fields are then gathered (sl_integrate.cu) without atomics:
//   F_k = sum_j (dE_k/dr_kj - dE_j/dr_jk),  H_k = -dE_k/dS_k - sum_j dE_j/dS_k + Zeeman.
//
// Atoms are stored species-major, so a warp almost always has one centre species;
// the neighbour list is segmented by neighbour species, so inside a segment both
// species are compile-time constants and every coefficient is a constant operand.
#include <mutex>

#include "sl_internal.h"

namespace sl {

template <typename R> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <typename R> using v2 = typename V2<R>::t;

template <typename R>
struct EvalArgs {
    const v4<R> *pos;
    const v4<R> *spin;
    const int32_t *nbr;
    const int4 *seg;
    int64_t n, n_fe;
    BoxDev<R> box;
    R *q, *bsum, *fp, *ei;
    v4<R> *pd0;
    v2<R> *pd1;
    v4<R> *fown, *gii;
    R *wpart;
    int want_virial;
};

template <typename R>
__device__ __forceinline__ R tanh_(R x);
template <>
__device__ __forceinline__ float tanh_<float>(float x) { return tanhf(x); }
template <>
__device__ __forceinline__ double tanh_<double>(double x) { return tanh(x); }

// ------------------------------------------------------------------ forward
template <typename R, int TI, int TJ>
__device__ __forceinline__ void fwd_radial(const NepDev<R> &P, const EvalArgs<R> &a, int64_t i, const v4<R> &pi,
                                           const v4<R> &si, int s0, int s1, R qr[NCH], R qx[4][NCH]) {
    R b0[NK], b1[NK], b2[NK], b3[NK], b4[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) { b0[k] = b1[k] = b2[k] = b3[k] = b4[k] = R(0); }
    for (int s = s0; s < s1; ++s) {
        const int j = a.nbr[(int64_t)s * a.n + i];
        const v4<R> pj = a.pos[j];
        R dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        minimg(a.box, dx, dy, dz);
        const R d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < P.rc_r2) {
            const v4<R> sj = a.spin[j];
            const R ir = rsqrt_(d2), r = d2 * ir;
            const R ux = dx * ir, uy = dy * ir, uz = dz * ir;
            R f[NK];
            carrier_f(r, P.inv_rc_r, f);
            const R sij = si.x * sj.x + si.y * sj.y + si.z * sj.z;
            const R siu = si.x * ux + si.y * uy + si.z * uz;
            const R sju = sj.x * ux + sj.y * uy + sj.z * uz;
            const R dmi = (si.y * sj.z - si.z * sj.y) * ux + (si.z * sj.x - si.x * sj.z) * uy +
                          (si.x * sj.y - si.y * sj.x) * uz;
            const R ani = siu * sju, sia = siu * siu;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                b0[k] += f[k];
                b1[k] += f[k] * sij;
                b2[k] += f[k] * dmi;
                b3[k] += f[k] * ani;
                b4[k] += f[k] * sia;
            }
        }
    }
#pragma unroll
    for (int n = 0; n < NCH; ++n) {
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            qr[n] += P.c[TI][TJ][G_R][n][k] * b0[k];
            qx[0][n] += P.c[TI][TJ][G_EX][n][k] * b1[k];
            qx[1][n] += P.c[TI][TJ][G_DMI][n][k] * b2[k];
            qx[2][n] += P.c[TI][TJ][G_ANI][n][k] * b3[k];
            qx[3][n] += P.c[TI][TJ][G_SIA][n][k] * b4[k];
        }
    }
}

template <typename R, int TI, int TJ>
__device__ __forceinline__ void fwd_angular(const NepDev<R> &P, const EvalArgs<R> &a, int64_t i, const v4<R> &pi,
                                            const v4<R> &si, int n, int s0, int s1, R B[NLM], R BS[NLM]) {
    for (int s = s0; s < s1; ++s) {
        const int j = a.nbr[(int64_t)s * a.n + i];
        const v4<R> pj = a.pos[j];
        R dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        minimg(a.box, dx, dy, dz);
        const R d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < P.rc_a2) {
            const v4<R> sj = a.spin[j];
            const R ir = rsqrt_(d2), r = d2 * ir;
            R f[NK];
            carrier_f(r, P.inv_rc_a, f);
            R g = R(0);
#pragma unroll
            for (int k = 0; k < NK; ++k) g += P.c[TI][TJ][G_A][n][k] * f[k];
            const R gs = g * (si.x * sj.x + si.y * sj.y + si.z * sj.z);
            R p[NLM];
            harm_p(dx * ir, dy * ir, dz * ir, p);
#pragma unroll
            for (int lm = 0; lm < NLM; ++lm) {
                B[lm] += g * p[lm];
                BS[lm] += gs * p[lm];
            }
        }
    }
}

template <typename R, int TI>
__device__ __forceinline__ void fwd_atom(const NepDev<R> &P, const EvalArgs<R> &a, int64_t i) {
    const v4<R> pi = a.pos[i], si = a.spin[i];
    const int4 sg = a.seg[i];
    const int64_t N = a.n;
    R qr[NCH], qx[4][NCH];
#pragma unroll
    for (int n = 0; n < NCH; ++n) { qr[n] = R(0); qx[0][n] = qx[1][n] = qx[2][n] = qx[3][n] = R(0); }
    fwd_radial<R, TI, 0>(P, a, i, pi, si, 0, sg.x, qr, qx);
    fwd_radial<R, TI, 1>(P, a, i, pi, si, sg.x, sg.y, qr, qx);
    fwd_radial<R, TI, 0>(P, a, i, pi, si, sg.y, sg.z, qr, qx);
    fwd_radial<R, TI, 1>(P, a, i, pi, si, sg.z, sg.w, qr, qx);
#pragma unroll
    for (int n = 0; n < NCH; ++n) {
        a.q[(Q_R + n) * N + i] = qr[n];
        a.q[(Q_EX + n) * N + i] = qx[0][n];
        a.q[(Q_DMI + n) * N + i] = qx[1][n];
        a.q[(Q_ANI + n) * N + i] = qx[2][n];
        a.q[(Q_SIA + n) * N + i] = qx[3][n];
    }
    a.q[Q_O * N + i] = si.x * si.x + si.y * si.y + si.z * si.z;
#pragma unroll 1
    for (int n = 0; n < NCH; ++n) {
        R B[NLM], BS[NLM];
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) { B[lm] = R(0); BS[lm] = R(0); }
        fwd_angular<R, TI, 0>(P, a, i, pi, si, n, 0, sg.x, B, BS);
        fwd_angular<R, TI, 1>(P, a, i, pi, si, n, sg.x, sg.y, B, BS);
        R qa[4] = {R(0), R(0), R(0), R(0)}, qs[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
            const R kap = R(harm_kappa(lm));
            qa[harm_l(lm) - 1] += kap * B[lm] * B[lm];
            qs[harm_l(lm) - 1] += kap * BS[lm] * BS[lm];
            a.bsum[(int64_t)(n * NLM + lm) * N + i] = B[lm];
            a.bsum[(int64_t)(NCH * NLM + n * NLM + lm) * N + i] = BS[lm];
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            a.q[(int64_t)(Q_A + n * 4 + l) * N + i] = qa[l];
            a.q[(int64_t)(Q_SA + n * 4 + l) * N + i] = qs[l];
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(128) k_fwd(const __grid_constant__ NepDev<R> P, const EvalArgs<R> a) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    if (i < a.n_fe) fwd_atom<R, 0>(P, a, i);
    else fwd_atom<R, 1>(P, a, i);
}

// ------------------------------------------------------------------ network
// E_i = sum_h w1_h tanh(z_h) - b1, z_h = sum_v W0_hv s_v q_v - b0_h;
// Fp_v = s_v sum_h w1_h (1 - tanh^2 z_h) W0_hv.
template <typename R>
__global__ void __launch_bounds__(128) k_mlp(const __grid_constant__ NepDev<R> P, const R *__restrict__ q,
                                             R *__restrict__ fp, R *__restrict__ ei, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    R x[DIM];
#pragma unroll
    for (int v = 0; v < DIM; ++v) x[v] = q[(int64_t)v * n + i] * P.scal[v];
    R t[NH];
    R E = -P.b1;
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        R z = -P.b0[h];
#pragma unroll
        for (int v = 0; v < DIM; ++v) z += P.w0[h][v] * x[v];
        const R th = tanh_(z);
        E += P.w1[h] * th;
        t[h] = P.w1[h] * (R(1) - th * th);
    }
#pragma unroll
    for (int v = 0; v < DIM; ++v) {
        R s = R(0);
#pragma unroll
        for (int h = 0; h < NH; ++h) s += t[h] * P.w0[h][v];
        fp[(int64_t)v * n + i] = s * P.scal[v];
    }
    ei[i] = E;
}

// ------------------------------------------------------------------ backward
template <typename R, int TI, int TJ, int LM>
__device__ __forceinline__ void bwd_lm(const R *__restrict__ sB, int bd, R ux, R uy, R uz, R ir, R sij,
                                       const R g[NCH], const R dg[NCH], R &accu, R &avx, R &avy, R &avz, R &cj) {
    R p, gx, gy, gz;
    harm_one<R, LM>(ux, uy, uz, p, gx, gy, gz);
    R aA = R(0), aS = R(0), bA = R(0), bS = R(0);
#pragma unroll
    for (int n = 0; n < NCH; ++n) {
        const R ba = sB[(n * NLM + LM) * bd];
        const R bs = sB[(NCH * NLM + n * NLM + LM) * bd];
        aA += ba * g[n];
        aS += bs * g[n];
        bA += ba * dg[n];
        bS += bs * dg[n];
    }
    const R av = aA + sij * aS, bv = bA + sij * bS;
    accu += p * (bv - R(harm_l(LM)) * ir * av);
    avx += av * gx;
    avy += av * gy;
    avz += av * gz;
    cj += aS * p;
}

template <typename R, int TI, int TJ, int LM>
__device__ __forceinline__ void bwd_lm_all(const R *__restrict__ sB, int bd, R ux, R uy, R uz, R ir, R sij,
                                           const R g[NCH], const R dg[NCH], R &accu, R &avx, R &avy, R &avz, R &cj) {
    bwd_lm<R, TI, TJ, LM>(sB, bd, ux, uy, uz, ir, sij, g, dg, accu, avx, avy, avz, cj);
    if constexpr (LM + 1 < NLM) bwd_lm_all<R, TI, TJ, LM + 1>(sB, bd, ux, uy, uz, ir, sij, g, dg, accu, avx, avy, avz, cj);
}

template <typename R>
struct BwdAcc {
    R fx, fy, fz;            // sum_j dE_i/dr_ij
    R hx, hy, hz;            // dE_i/dS_i
    R w[9];                  // -sum_j r_ij (x) dE_i/dr_ij
};

template <typename R, int TI, int TJ, bool ANG>
__device__ __forceinline__ void bwd_seg(const NepDev<R> &P, const EvalArgs<R> &a, int64_t i, const v4<R> &pi,
                                        const v4<R> &si, const R FR[NCH], const R FX[4][NCH], const R *sB, int bd,
                                        int s0, int s1, BwdAcc<R> &acc) {
    // precontracted radial coefficients  C^G_k = sum_n Fp^G_n c^G_{n k t_i t_j}
    R C0[NK], C1[NK], C2[NK], C3[NK], C4[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        R s0_ = R(0), s1_ = R(0), s2_ = R(0), s3_ = R(0), s4_ = R(0);
#pragma unroll
        for (int n = 0; n < NCH; ++n) {
            s0_ += FR[n] * P.c[TI][TJ][G_R][n][k];
            s1_ += FX[0][n] * P.c[TI][TJ][G_EX][n][k];
            s2_ += FX[1][n] * P.c[TI][TJ][G_DMI][n][k];
            s3_ += FX[2][n] * P.c[TI][TJ][G_ANI][n][k];
            s4_ += FX[3][n] * P.c[TI][TJ][G_SIA][n][k];
        }
        C0[k] = s0_; C1[k] = s1_; C2[k] = s2_; C3[k] = s3_; C4[k] = s4_;
    }
    const int64_t N = a.n;
    for (int s = s0; s < s1; ++s) {
        const int j = a.nbr[(int64_t)s * N + i];
        const v4<R> pj = a.pos[j];
        R dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        minimg(a.box, dx, dy, dz);
        const R d2 = dx * dx + dy * dy + dz * dz;
        R Dx = R(0), Dy = R(0), Dz = R(0), Gx = R(0), Gy = R(0), Gz = R(0);
        if (d2 < P.rc_r2) {
            const v4<R> sj = a.spin[j];
            const R ir = rsqrt_(d2), r = d2 * ir;
            const R ux = dx * ir, uy = dy * ir, uz = dz * ir;
            R f[NK], df[NK];
            carrier_fd(r, P.inv_rc_r, f, df);
            R h0 = 0, h1 = 0, h2 = 0, h3 = 0, h4 = 0, e0 = 0, e1 = 0, e2 = 0, e3 = 0, e4 = 0;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                e0 += C0[k] * df[k];
                h1 += C1[k] * f[k]; e1 += C1[k] * df[k];
                h2 += C2[k] * f[k]; e2 += C2[k] * df[k];
                h3 += C3[k] * f[k]; e3 += C3[k] * df[k];
                h4 += C4[k] * f[k]; e4 += C4[k] * df[k];
            }
            (void)h0;
            const R sij = si.x * sj.x + si.y * sj.y + si.z * sj.z;
            const R siu = si.x * ux + si.y * uy + si.z * uz;
            const R sju = sj.x * ux + sj.y * uy + sj.z * uz;
            const R wx = si.y * sj.z - si.z * sj.y, wy = si.z * sj.x - si.x * sj.z, wz = si.x * sj.y - si.y * sj.x;
            const R wu = wx * ux + wy * uy + wz * uz;
            const R rad = e0 + e1 * sij + e2 * wu + e3 * siu * sju + e4 * siu * siu;
            // tangential parts (v - (v.u) u) / r of the spin-function gradients
            const R cSi = (h3 * sju + R(2) * h4 * siu) * ir;   // coefficient of P_perp S_i
            const R cSj = h3 * siu * ir;                       // coefficient of P_perp S_j
            const R cW = h2 * ir;                              // coefficient of P_perp (S_i x S_j)
            const R along = rad - cSi * siu - cSj * sju - cW * wu;
            Dx = along * ux + cSi * si.x + cSj * sj.x + cW * wx;
            Dy = along * uy + cSi * si.y + cSj * sj.y + cW * wy;
            Dz = along * uz + cSi * si.z + cSj * sj.z + cW * wz;
            // dE_i/dS_j = h_EX S_i + h_DMI (u x S_i) + h_ANI (S_i.u) u
            Gx = h1 * si.x + h2 * (uy * si.z - uz * si.y) + h3 * siu * ux;
            Gy = h1 * si.y + h2 * (uz * si.x - ux * si.z) + h3 * siu * uy;
            Gz = h1 * si.z + h2 * (ux * si.y - uy * si.x) + h3 * siu * uz;
            // dE_i/dS_i += h_EX S_j + h_DMI (S_j x u) + h_ANI (S_j.u) u + 2 h_SIA (S_i.u) u
            const R cu = h3 * sju + R(2) * h4 * siu;
            acc.hx += h1 * sj.x + h2 * (sj.y * uz - sj.z * uy) + cu * ux;
            acc.hy += h1 * sj.y + h2 * (sj.z * ux - sj.x * uz) + cu * uy;
            acc.hz += h1 * sj.z + h2 * (sj.x * uy - sj.y * ux) + cu * uz;
            if constexpr (ANG) {
                if (d2 < P.rc_a2) {
                    carrier_fd(r, P.inv_rc_a, f, df);
                    R g[NCH], dg[NCH];
#pragma unroll
                    for (int n = 0; n < NCH; ++n) {
                        R s_ = R(0), t_ = R(0);
#pragma unroll
                        for (int k = 0; k < NK; ++k) {
                            s_ += P.c[TI][TJ][G_A][n][k] * f[k];
                            t_ += P.c[TI][TJ][G_A][n][k] * df[k];
                        }
                        g[n] = s_;
                        dg[n] = t_;
                    }
                    R accu = R(0), avx = R(0), avy = R(0), avz = R(0), cj = R(0);
                    bwd_lm_all<R, TI, TJ, 0>(sB, bd, ux, uy, uz, ir, sij, g, dg, accu, avx, avy, avz, cj);
                    Dx += accu * ux + ir * avx;
                    Dy += accu * uy + ir * avy;
                    Dz += accu * uz + ir * avz;
                    Gx += cj * si.x; Gy += cj * si.y; Gz += cj * si.z;
                    acc.hx += cj * sj.x; acc.hy += cj * sj.y; acc.hz += cj * sj.z;
                }
            }
            acc.fx += Dx; acc.fy += Dy; acc.fz += Dz;
            if (a.want_virial) {
                acc.w[0] -= dx * Dx; acc.w[1] -= dx * Dy; acc.w[2] -= dx * Dz;
                acc.w[3] -= dy * Dx; acc.w[4] -= dy * Dy; acc.w[5] -= dy * Dz;
                acc.w[6] -= dz * Dx; acc.w[7] -= dz * Dy; acc.w[8] -= dz * Dz;
            }
        }
        v4<R> e0v;
        e0v.x = Dx; e0v.y = Dy; e0v.z = Dz; e0v.w = Gx;
        v2<R> e1v;
        e1v.x = Gy; e1v.y = Gz;
        a.pd0[(int64_t)s * N + i] = e0v;
        a.pd1[(int64_t)s * N + i] = e1v;
    }
}

template <typename R, int TI>
__device__ __forceinline__ void bwd_atom(const NepDev<R> &P, const EvalArgs<R> &a, int64_t i, R *sB, int bd) {
    const int64_t N = a.n;
    const v4<R> pi = a.pos[i], si = a.spin[i];
    const int4 sg = a.seg[i];
    // adjoints of the angular sums: dE/dB_nlm = 2 kappa_lm Fp(A_nl) B_nlm, same for BS with Fp(SA_nl)
#pragma unroll 1
    for (int n = 0; n < NCH; ++n) {
        R fa[4], fs[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            fa[l] = a.fp[(int64_t)(Q_A + n * 4 + l) * N + i];
            fs[l] = a.fp[(int64_t)(Q_SA + n * 4 + l) * N + i];
        }
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
            const R k2 = R(2.0 * harm_kappa(lm));
            sB[(n * NLM + lm) * bd] = k2 * fa[harm_l(lm) - 1] * a.bsum[(int64_t)(n * NLM + lm) * N + i];
            sB[(NCH * NLM + n * NLM + lm) * bd] =
                k2 * fs[harm_l(lm) - 1] * a.bsum[(int64_t)(NCH * NLM + n * NLM + lm) * N + i];
        }
    }
    R FR[NCH], FX[4][NCH];
#pragma unroll
    for (int n = 0; n < NCH; ++n) {
        FR[n] = a.fp[(int64_t)(Q_R + n) * N + i];
        FX[0][n] = a.fp[(int64_t)(Q_EX + n) * N + i];
        FX[1][n] = a.fp[(int64_t)(Q_DMI + n) * N + i];
        FX[2][n] = a.fp[(int64_t)(Q_ANI + n) * N + i];
        FX[3][n] = a.fp[(int64_t)(Q_SIA + n) * N + i];
    }
    const R fo = R(2) * a.fp[(int64_t)Q_O * N + i];
    BwdAcc<R> acc;
    acc.fx = acc.fy = acc.fz = R(0);
    acc.hx = fo * si.x; acc.hy = fo * si.y; acc.hz = fo * si.z;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc.w[t] = R(0);
    bwd_seg<R, TI, 0, true>(P, a, i, pi, si, FR, FX, sB, bd, 0, sg.x, acc);
    bwd_seg<R, TI, 1, true>(P, a, i, pi, si, FR, FX, sB, bd, sg.x, sg.y, acc);
    bwd_seg<R, TI, 0, false>(P, a, i, pi, si, FR, FX, sB, bd, sg.y, sg.z, acc);
    bwd_seg<R, TI, 1, false>(P, a, i, pi, si, FR, FX, sB, bd, sg.z, sg.w, acc);
    v4<R> fo4, go4;
    fo4.x = acc.fx; fo4.y = acc.fy; fo4.z = acc.fz; fo4.w = R(0);
    go4.x = acc.hx; go4.y = acc.hy; go4.z = acc.hz; go4.w = R(0);
    a.fown[i] = fo4;
    a.gii[i] = go4;
    if (a.want_virial) {
#pragma unroll
        for (int t = 0; t < 9; ++t) a.wpart[(int64_t)t * N + i] = acc.w[t];
    }
}

template <typename R>
__global__ void k_bwd(const __grid_constant__ NepDev<R> P, const EvalArgs<R> a) {
    extern __shared__ unsigned char smem_raw[];
    R *sB = reinterpret_cast<R *>(smem_raw) + threadIdx.x;
    const int bd = blockDim.x;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    if (i < a.n_fe) bwd_atom<R, 0>(P, a, i, sB, bd);
    else bwd_atom<R, 1>(P, a, i, sB, bd);
}

// ------------------------------------------------------------------ launch
template <typename R>
static EvalArgs<R> make_args(Sys &s, bool want_virial);

template <>
EvalArgs<double> make_args<double>(Sys &s, bool want_virial) {
    EvalArgs<double> a;
    a.pos = s.pos; a.spin = s.spin; a.box = s.boxd;
    a.nbr = s.nbr; a.seg = s.seg; a.n = s.n; a.n_fe = s.n_fe;
    a.q = (double *)s.q; a.bsum = (double *)s.bsum; a.fp = (double *)s.fp; a.ei = (double *)s.ei;
    a.pd0 = (double4 *)s.pd0; a.pd1 = (double2 *)s.pd1; a.fown = (double4 *)s.fown; a.gii = (double4 *)s.gii;
    a.wpart = (double *)s.wpart; a.want_virial = want_virial;
    return a;
}

template <>
EvalArgs<float> make_args<float>(Sys &s, bool want_virial) {
    EvalArgs<float> a;
    a.pos = s.posf; a.spin = s.spinf; a.box = s.boxf;
    a.nbr = s.nbr; a.seg = s.seg; a.n = s.n; a.n_fe = s.n_fe;
    a.q = (float *)s.q; a.bsum = (float *)s.bsum; a.fp = (float *)s.fp; a.ei = (float *)s.ei;
    a.pd0 = (float4 *)s.pd0; a.pd1 = (float2 *)s.pd1; a.fown = (float4 *)s.fown; a.gii = (float4 *)s.gii;
    a.wpart = (float *)s.wpart; a.want_virial = want_virial;
    return a;
}

template <typename R>
static constexpr int bwd_block() { return sizeof(R) == 8 ? 32 : 64; }

template <typename R>
static void eval_impl(Sys &s, const NepDev<R> &P, bool want_virial, cudaEvent_t *ev) {
    const EvalArgs<R> a = make_args<R>(s, want_virial);
    const unsigned nb = (unsigned)((s.n + 127) / 128);
    if (ev) cudaEventRecord(ev[0], s.stream);
    k_fwd<R><<<nb, 128, 0, s.stream>>>(P, a);
    if (ev) cudaEventRecord(ev[1], s.stream);
    k_mlp<R><<<nb, 128, 0, s.stream>>>(P, (const R *)s.q, (R *)s.fp, (R *)s.ei, s.n);
    if (ev) cudaEventRecord(ev[2], s.stream);
    const int bd = bwd_block<R>();
    const size_t sm = (size_t)NB * bd * sizeof(R);
    k_bwd<R><<<(unsigned)((s.n + bd - 1) / bd), bd, sm, s.stream>>>(P, a);
    if (ev) cudaEventRecord(ev[3], s.stream);
}

// Kernel attributes are set once per process, before any stream capture.
void eval_init() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_bwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(NB * bwd_block<float>() * sizeof(float)));
    cudaFuncSetAttribute(k_bwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(NB * bwd_block<double>() * sizeof(double)));
    done = true;
}

void launch_eval(Sys &s, bool want_virial, cudaEvent_t *ev) {
    if (s.n == 0) return;
    if (s.prec == 0) eval_impl<double>(s, s.pd, want_virial, ev);
    else eval_impl<float>(s, s.pf, want_virial, ev);
}

size_t eval_bytes(const Sys &s) {
    const size_t r = s.prec == 0 ? 8 : 4;
    const size_t n = (size_t)s.n;
    return r * n * (2 * DIM + NB + 1 + 9) + r * 4 * n * 2 + r * 6 * n * (size_t)s.cap;
}


// ------------------------------------------------------------------ no-allocation variant
// Descriptors and network energies of a small system in ONE kernel whose scratch
// (neighbour lists, list segments, descriptor columns, angular sums, a status
// word) lives in a fixed file-scope device array instead of memory the caller or
// the library allocates.  For callers that may not allocate device memory (see
// sl_descriptors_energies_noalloc in spinlat.h).  Computes in FP64.
namespace noalloc {

constexpr int MAX_ATOMS = 2048;
constexpr int MAX_NBR = 160;   // neighbours inside rc_rad per atom
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t OFF_NBR = 0;
constexpr size_t OFF_SEG = align256(OFF_NBR + sizeof(int32_t) * MAX_ATOMS * MAX_NBR);
constexpr size_t OFF_Q = align256(OFF_SEG + sizeof(int4) * MAX_ATOMS);
constexpr size_t OFF_B = align256(OFF_Q + sizeof(double) * DIM * MAX_ATOMS);
constexpr size_t OFF_STATUS = align256(OFF_B + sizeof(double) * NB * MAX_ATOMS);
constexpr size_t BYTES = align256(OFF_STATUS + sizeof(int));

// ~6.3 MB, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_scratch[BYTES];

__global__ void __launch_bounds__(128) k_eval_noalloc(const __grid_constant__ NepDev<double> P,
                                                      const double4 *__restrict__ pos,
                                                      const double4 *__restrict__ spin,
                                                      const int32_t *__restrict__ species, int n, BoxDev<double> box,
                                                      unsigned char *scratch, double *__restrict__ q_out,
                                                      double *__restrict__ e_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t *nbr = reinterpret_cast<int32_t *>(scratch + OFF_NBR);
    int4 *seg = reinterpret_cast<int4 *>(scratch + OFF_SEG);
    double *q = reinterpret_cast<double *>(scratch + OFF_Q);
    double *bsum = reinterpret_cast<double *>(scratch + OFF_B);
    int *status = reinterpret_cast<int *>(scratch + OFF_STATUS);
    // brute-force neighbours inside rc_rad, inserted in (segment, index) order
    // straight into this atom's scratch column (slot-major, stride n)
    const double4 pi = pos[i];
    int m = 0;
    bool overflow = false;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        const double4 pj = pos[j];
        double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        minimg(box, dx, dy, dz);
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (!(d2 < P.rc_r2)) continue;
        if (m >= MAX_NBR) { overflow = true; continue; }
        const int key = ((d2 < P.rc_a2 ? 0 : 2) + species[j]) * MAX_ATOMS + j;
        int v = m - 1;
        while (v >= 0) {
            const int jv = nbr[(int64_t)v * n + i];
            const double4 pv = pos[jv];
            double ex = pv.x - pi.x, ey = pv.y - pi.y, ez = pv.z - pi.z;
            minimg(box, ex, ey, ez);
            const int kv = (((ex * ex + ey * ey + ez * ez) < P.rc_a2 ? 0 : 2) + species[jv]) * MAX_ATOMS + jv;
            if (kv <= key) break;
            nbr[(int64_t)(v + 1) * n + i] = jv;
            --v;
        }
        nbr[(int64_t)(v + 1) * n + i] = j;
        ++m;
    }
    if (overflow) atomicOr(status, ST_NBR_OVERFLOW);
    int ends[4] = {0, 0, 0, 0};
    for (int s = 0; s < m; ++s) {
        const int j = nbr[(int64_t)s * n + i];
        const double4 pj = pos[j];
        double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        minimg(box, dx, dy, dz);
        const int sg = ((dx * dx + dy * dy + dz * dz) < P.rc_a2 ? 0 : 2) + species[j];
        for (int t = sg; t < 4; ++t) ends[t] = s + 1;
    }
    for (int t = 1; t < 4; ++t) ends[t] = max(ends[t], ends[t - 1]);
    seg[i] = make_int4(ends[0], ends[1], ends[2], ends[3]);
    // descriptor through the same per-atom code as k_fwd
    EvalArgs<double> a;
    a.pos = pos; a.spin = spin; a.nbr = nbr; a.seg = seg; a.n = n; a.n_fe = 0; a.box = box;
    a.q = q; a.bsum = bsum;
    if (species[i] == 0) fwd_atom<double, 0>(P, a, i);
    else fwd_atom<double, 1>(P, a, i);
    // network energy E_i = sum_h w1_h tanh(sum_v W0_hv s_v q_v - b0_h) - b1
    double x[DIM];
#pragma unroll
    for (int v = 0; v < DIM; ++v) {
        x[v] = q[(int64_t)v * n + i];
        if (q_out) q_out[(int64_t)i * DIM + v] = x[v];
        x[v] *= P.scal[v];
    }
    double E = -P.b1;
#pragma unroll 1
    for (int h = 0; h < NH; ++h) {
        double z = -P.b0[h];
#pragma unroll
        for (int v = 0; v < DIM; ++v) z += P.w0[h][v] * x[v];
        E += P.w1[h] * tanh(z);
    }
    e_out[i] = E;
}

}  // namespace noalloc

// Device address of the scratch array for the current device, looked up once per
// device (host code cannot use the symbol itself as a device address).
int noalloc_scratch(void **out) {
    static std::mutex mu;
    static void *addr[128] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return -1;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, noalloc::g_scratch) != cudaSuccess || !p) return -1;
        addr[dev] = p;
    }
    *out = addr[dev];
    return 0;
}

int launch_noalloc(const NepDev<double> &P, const double4 *pos, const double4 *spin, const int32_t *species, int n,
                   const BoxDev<double> &box, double *q_out, double *e_out, cudaStream_t stream, int *status_out) {
    void *scratch = nullptr;
    if (noalloc_scratch(&scratch)) return -1;
    int *status = reinterpret_cast<int *>(static_cast<unsigned char *>(scratch) + noalloc::OFF_STATUS);
    if (cudaMemsetAsync(status, 0, sizeof(int), stream) != cudaSuccess) return -1;
    noalloc::k_eval_noalloc<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(
        P, pos, spin, species, n, box, static_cast<unsigned char *>(scratch), q_out, e_out);
    if (cudaGetLastError() != cudaSuccess) return -1;
    int st = 0;
    if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return -1;
    *status_out = st;
    return 0;
}

int noalloc_max_atoms() { return noalloc::MAX_ATOMS; }

}  // namespace sl
