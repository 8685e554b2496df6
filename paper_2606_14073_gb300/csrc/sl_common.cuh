// sl_common.cuh -- shared device definitions of the NEP-SPIN GB300 library.
//
// Model shape fixed at compile time (the FeGe network of arXiv 2606.14073):
// 2 species, 5 channels, 9 Chebyshev terms (basis size 8, Section 5.2.4),
// l_max = 4 (24 real solid harmonics), 30 hidden units, 66-entry descriptor
// (Section 5.2.3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sl {

constexpr int NS = 2;     // species
constexpr int NCH = 5;    // radial channels n = 0..4
constexpr int NK = 9;     // Chebyshev terms k = 0..8
constexpr int NH = 30;    // hidden units
constexpr int NLM = 24;   // real solid harmonics, l = 1..4
constexpr int DIM = 66;   // descriptor length
constexpr int NB = 2 * NCH * NLM;   // 240 angular sums kept for the backward pass
// The angular sums are stored atom-major as one 12-entry record per harmonic lm:
// (B_0lm, BS_0lm, B_1lm, BS_1lm, ..., B_4lm, BS_4lm, 0, 0), 48 bytes in FP32 (three
// 16-byte words), the layout the backward kernel keeps its adjoints in.
constexpr int BREC = 12;
constexpr int NBREC = NLM * BREC;   // 288 stored entries per atom

// coefficient groups
constexpr int G_R = 0, G_A = 1, G_EX = 2, G_DMI = 3, G_ANI = 4, G_SIA = 5;
// descriptor offsets: R(5) A(n,l)(20) O(1) EX(5) DMI(5) ANI(5) SIA(5) SA(n,l)(20)
constexpr int Q_R = 0, Q_A = 5, Q_O = 25, Q_EX = 26, Q_DMI = 31, Q_ANI = 36, Q_SIA = 41, Q_SA = 46;

// physical constants (CODATA 2018)
constexpr double KB = 8.617333262e-5;     // eV/K
constexpr double HBAR = 0.6582119569;     // eV fs
constexpr double MUB = 5.7883818060e-5;   // eV/T
constexpr double ACC = 9.6485332e-3;      // (eV/A/amu) -> A/fs^2

// Model parameters in the compute precision R.  Passed by value as a
// __grid_constant__ kernel parameter (about 13 KB in FP32, 26 KB in FP64): with
// the centre and neighbour species known at compile time every coefficient is a
// constant-bank operand of the FMA that uses it.
template <typename R>
struct NepDev {
    R c[NS][NS][6][NCH][NK];   // [centre][neighbour][group][n][k]
    R scal[DIM];
    R w0[NH][DIM];
    R b0[NH];
    R w1[NH];
    R b1;
    R rc_r, rc_a, inv_rc_r, inv_rc_a, rc_r2, rc_a2;
};

// Orthorhombic box; invL = 0 along free dimensions disables the minimum image.
template <typename R>
struct BoxDev {
    R L[3];
    R invL[3];
};

template <typename R> struct V4;
template <> struct V4<float> { using t = float4; };
template <> struct V4<double> { using t = double4; };
template <typename R> using v4 = typename V4<R>::t;

// Loads through the read-only (non-coherent) path, for data the calling kernel never writes.
// The kernels read their argument blocks from tables, so the compiler cannot prove that by
// itself from the pointers.
__device__ __forceinline__ float4 ro(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ int4 ro(const int4 *p) { return __ldg(p); }
__device__ __forceinline__ uchar4 ro(const uchar4 *p) { return __ldg(p); }
__device__ __forceinline__ int ro(const int *p) { return __ldg(p); }
__device__ __forceinline__ unsigned ro(const unsigned *p) { return __ldg(p); }
__device__ __forceinline__ unsigned short ro(const unsigned short *p) { return __ldg(p); }
__device__ __forceinline__ float ro(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ro(const double *p) { return __ldg(p); }
__device__ __forceinline__ double4 ro(const double4 *p) {
    const double2 lo = __ldg(reinterpret_cast<const double2 *>(p)), hi = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return make_double4(lo.x, lo.y, hi.x, hi.y);
}

// Stores typed as global-memory stores.  The kernels read their argument blocks from shared
// memory; a store through a plain (generic) pointer might, as far as the compiler can tell,
// land there, and every argument would be read again after it.
__device__ __forceinline__ void stg(int *p, int v) { __stwb(p, v); }
__device__ __forceinline__ void stg(unsigned short *p, unsigned short v) { __stwb(p, v); }
__device__ __forceinline__ void stg(float *p, float v) { __stwb(p, v); }
__device__ __forceinline__ void stg(double *p, double v) { __stwb(p, v); }
__device__ __forceinline__ void stg(float4 *p, const float4 &v) { __stwb(p, v); }
__device__ __forceinline__ void stg(int4 *p, const int4 &v) { __stwb(p, v); }
__device__ __forceinline__ void stg(double4 *p, const double4 &v) {
    __stwb(reinterpret_cast<double2 *>(p), make_double2(v.x, v.y));
    __stwb(reinterpret_cast<double2 *>(p) + 1, make_double2(v.z, v.w));
}

template <typename R>
__device__ __forceinline__ R rint_(R x);
template <>
__device__ __forceinline__ float rint_<float>(float x) { return rintf(x); }
template <>
__device__ __forceinline__ double rint_<double>(double x) { return rint(x); }

template <typename R>
__device__ __forceinline__ void minimg(const BoxDev<R> &b, R &dx, R &dy, R &dz) {
    dx -= b.L[0] * rint_(dx * b.invL[0]);
    dy -= b.L[1] * rint_(dy * b.invL[1]);
    dz -= b.L[2] * rint_(dz * b.invL[2]);
}

template <typename R>
__device__ __forceinline__ R rsqrt_(R x);
template <>
__device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }


template <typename R>
__device__ __forceinline__ R fma_(R a, R b, R c);
template <>
__device__ __forceinline__ float fma_<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_<double>(double a, double b, double c) { return fma(a, b, c); }

// Cutoff half f_c/2 = (1 + cos(pi t))/4 (t = r/rc in [0, 1)) and d(f_c/2)/dr.
// FP64: the CUDA library's cospi / sincospi.  FP32: written as cos^2(w)/2 with w = pi t/2 in
// [0, pi/2] (no cancellation near t = 1) and d/dr = -(pi/2)/rc sin(w) cos(w), with sin w and
// cos w from their Taylor series at 0 through w^11 and w^12 (Horner in w^2): the first
// omitted terms are below (pi/2)^13/13! = 5.7e-8 and (pi/2)^14/14! = 6.4e-9 on the range.
__device__ __forceinline__ void sincos_halfpi_taylor(float t, float &s, float &c) {
    const float w = 1.57079632679489662f * t;
    const float w2 = w * w;
    constexpr float i2 = 1.f / 2.f, i4 = 1.f / 24.f, i6 = 1.f / 720.f, i8 = 1.f / 40320.f,
                    i10 = 1.f / 3628800.f, i12 = 1.f / 479001600.f;
    constexpr float i3 = 1.f / 6.f, i5 = 1.f / 120.f, i7 = 1.f / 5040.f, i9 = 1.f / 362880.f,
                    i11 = 1.f / 39916800.f;
    c = fmaf(w2, fmaf(w2, fmaf(w2, fmaf(w2, fmaf(w2, fmaf(w2, i12, -i10), i8), -i6), i4), -i2), 1.f);
    s = w * fmaf(w2, fmaf(w2, fmaf(w2, fmaf(w2, fmaf(w2, -i11, i9), -i7), i5), -i3), 1.f);
}

template <typename R>
__device__ __forceinline__ R cut_half(R t);
template <>
__device__ __forceinline__ float cut_half<float>(float t) {
    float s, c;
    sincos_halfpi_taylor(t, s, c);
    return 0.5f * c * c;
}
template <>
__device__ __forceinline__ double cut_half<double>(double t) { return 0.25 * (1.0 + cospi(t)); }

template <typename R>
__device__ __forceinline__ void cut_half_d(R t, R inv_rc, R &fch, R &dfch);
template <>
__device__ __forceinline__ void cut_half_d<float>(float t, float inv_rc, float &fch, float &dfch) {
    float s, c;
    sincos_halfpi_taylor(t, s, c);
    fch = 0.5f * c * c;
    dfch = -1.57079632679489662f * inv_rc * (s * c);
}
template <>
__device__ __forceinline__ void cut_half_d<double>(double t, double inv_rc, double &fch, double &dfch) {
    double sn, cs;
    sincospi(t, &sn, &cs);
    fch = 0.25 * (1.0 + cs);
    dfch = -0.785398163397448309616 * inv_rc * sn;   // d(f_c/2)/dr = -(pi/4)/rc sin
}

// Radial carrier (Sections 5.2.3-5.2.4): f_c = (1 + cos(pi r/rc))/2,
// x = 2 (r/rc - 1)^2 - 1, T_{k+1} = 2 x T_k - T_{k-1}, f_k = (T_k + 1) f_c / 2.
template <typename R>
__device__ __forceinline__ void carrier_f(R r, R inv_rc, R f[NK]) {
    const R t = r * inv_rc;
    const R fch = cut_half(t);   // f_c / 2
    const R y = t - R(1);
    const R x = R(2) * y * y - R(1);
    R tm = R(1), tc = x;
    f[0] = R(2) * fch;
    f[1] = fma_(x, fch, fch);                          // (T_1 + 1) f_c/2 with one rounding
#pragma unroll
    for (int k = 2; k < NK; ++k) {
        const R tn = R(2) * x * tc - tm;
        f[k] = fma_(tn, fch, fch);
        tm = tc;
        tc = tn;
    }
}

// Carrier and its r-derivative; dT_k/dx = k U_{k-1}, U_{k+1} = 2 x U_k - U_{k-1}.
template <typename R>
__device__ __forceinline__ void carrier_fd(R r, R inv_rc, R f[NK], R df[NK]) {
    const R t = r * inv_rc;
    R fch, dfch;
    cut_half_d(t, inv_rc, fch, dfch);
    const R y = t - R(1);
    const R x = R(2) * y * y - R(1);
    const R dxr = R(4) * y * inv_rc;
    const R dxf = dxr * fch;
    R tm = R(1), tc = x, um = R(1), uc = R(2) * x;   // T_0, T_1, U_0, U_1
    f[0] = R(2) * fch;
    df[0] = R(2) * dfch;
    f[1] = fma_(x, fch, fch);
    df[1] = dxf + fma_(x, dfch, dfch);                // dT_1/dx = U_0 = 1
#pragma unroll
    for (int k = 2; k < NK; ++k) {
        const R tn = R(2) * x * tc - tm;
        f[k] = fma_(tn, fch, fch);
        df[k] = fma_(R(k) * uc, dxf, fma_(tn, dfch, dfch));   // k U_{k-1}
        const R un = R(2) * x * uc - um;
        tm = tc; tc = tn; um = uc; uc = un;
    }
}

// Real solid harmonics p_lm (homogeneous polynomials of degree l) with weights
// kappa_lm such that P_l(u.v) = sum_m kappa_lm p_lm(u) p_lm(v) for unit u, v
// (addition theorem with kappa_lm = 4 pi N_lm^2 / (2l+1), N_lm the usual
// normalisation of the real spherical harmonic).  Order: l = 1 (x, y, z);
// l = 2 (xy, yz, xz, x^2-y^2, 3z^2-r^2); l = 3 (7 terms); l = 4 (9 terms).
__host__ __device__ constexpr int harm_l(int lm) { return lm < 3 ? 1 : lm < 8 ? 2 : lm < 15 ? 3 : 4; }
__host__ __device__ constexpr double harm_kappa(int lm) {
    constexpr double k[NLM] = {1.0, 1.0, 1.0,
                               3.0, 3.0, 3.0, 0.75, 0.25,
                               0.625, 15.0, 0.375, 0.25, 0.375, 3.75, 0.625,
                               8.75, 4.375, 1.25, 0.625, 0.015625, 0.625, 0.3125, 4.375, 0.546875};
    return k[lm];
}

template <typename R>
__host__ __device__ __forceinline__ void harm_p(R x, R y, R z, R p[NLM]) {
    const R x2 = x * x, y2 = y * y, z2 = z * z, r2 = x2 + y2 + z2;
    p[0] = x; p[1] = y; p[2] = z;
    p[3] = x * y; p[4] = y * z; p[5] = x * z; p[6] = x2 - y2; p[7] = R(2) * z2 - x2 - y2;
    p[8] = y * (R(3) * x2 - y2);
    p[9] = x * y * z;
    p[10] = y * (R(4) * z2 - x2 - y2);
    p[11] = z * (R(2) * z2 - R(3) * x2 - R(3) * y2);
    p[12] = x * (R(4) * z2 - x2 - y2);
    p[13] = z * (x2 - y2);
    p[14] = x * (x2 - R(3) * y2);
    p[15] = x * y * (x2 - y2);
    p[16] = y * z * (R(3) * x2 - y2);
    p[17] = x * y * (R(6) * z2 - x2 - y2);
    p[18] = y * z * (R(4) * z2 - R(3) * x2 - R(3) * y2);
    p[19] = R(35) * z2 * z2 - R(30) * z2 * r2 + R(3) * r2 * r2;
    p[20] = x * z * (R(4) * z2 - R(3) * x2 - R(3) * y2);
    p[21] = (x2 - y2) * (R(6) * z2 - x2 - y2);
    p[22] = x * z * (x2 - R(3) * y2);
    p[23] = x2 * x2 - R(6) * x2 * y2 + y2 * y2;
}

// One harmonic and its Euclidean gradient (LM a compile-time index).
template <typename R, int LM>
__host__ __device__ __forceinline__ void harm_one(R x, R y, R z, R &p, R &gx, R &gy, R &gz) {
    const R x2 = x * x, y2 = y * y, z2 = z * z;
    if constexpr (LM == 0) { p = x; gx = 1; gy = 0; gz = 0; }
    else if constexpr (LM == 1) { p = y; gx = 0; gy = 1; gz = 0; }
    else if constexpr (LM == 2) { p = z; gx = 0; gy = 0; gz = 1; }
    else if constexpr (LM == 3) { p = x * y; gx = y; gy = x; gz = 0; }
    else if constexpr (LM == 4) { p = y * z; gx = 0; gy = z; gz = y; }
    else if constexpr (LM == 5) { p = x * z; gx = z; gy = 0; gz = x; }
    else if constexpr (LM == 6) { p = x2 - y2; gx = R(2) * x; gy = R(-2) * y; gz = 0; }
    else if constexpr (LM == 7) { p = R(2) * z2 - x2 - y2; gx = R(-2) * x; gy = R(-2) * y; gz = R(4) * z; }
    else if constexpr (LM == 8) { p = y * (R(3) * x2 - y2); gx = R(6) * x * y; gy = R(3) * (x2 - y2); gz = 0; }
    else if constexpr (LM == 9) { p = x * y * z; gx = y * z; gy = x * z; gz = x * y; }
    else if constexpr (LM == 10) {
        p = y * (R(4) * z2 - x2 - y2); gx = R(-2) * x * y; gy = R(4) * z2 - x2 - R(3) * y2; gz = R(8) * y * z;
    } else if constexpr (LM == 11) {
        p = z * (R(2) * z2 - R(3) * x2 - R(3) * y2); gx = R(-6) * x * z; gy = R(-6) * y * z;
        gz = R(6) * z2 - R(3) * x2 - R(3) * y2;
    } else if constexpr (LM == 12) {
        p = x * (R(4) * z2 - x2 - y2); gx = R(4) * z2 - R(3) * x2 - y2; gy = R(-2) * x * y; gz = R(8) * x * z;
    } else if constexpr (LM == 13) { p = z * (x2 - y2); gx = R(2) * x * z; gy = R(-2) * y * z; gz = x2 - y2; }
    else if constexpr (LM == 14) { p = x * (x2 - R(3) * y2); gx = R(3) * (x2 - y2); gy = R(-6) * x * y; gz = 0; }
    else if constexpr (LM == 15) {
        p = x * y * (x2 - y2); gx = y * (R(3) * x2 - y2); gy = x * (x2 - R(3) * y2); gz = 0;
    } else if constexpr (LM == 16) {
        p = y * z * (R(3) * x2 - y2); gx = R(6) * x * y * z; gy = R(3) * z * (x2 - y2); gz = y * (R(3) * x2 - y2);
    } else if constexpr (LM == 17) {
        p = x * y * (R(6) * z2 - x2 - y2); gx = y * (R(6) * z2 - R(3) * x2 - y2);
        gy = x * (R(6) * z2 - x2 - R(3) * y2); gz = R(12) * x * y * z;
    } else if constexpr (LM == 18) {
        p = y * z * (R(4) * z2 - R(3) * x2 - R(3) * y2); gx = R(-6) * x * y * z;
        gy = z * (R(4) * z2 - R(3) * x2 - R(9) * y2); gz = y * (R(12) * z2 - R(3) * x2 - R(3) * y2);
    } else if constexpr (LM == 19) {
        const R r2 = x2 + y2 + z2;
        p = R(35) * z2 * z2 - R(30) * z2 * r2 + R(3) * r2 * r2;
        gx = x * (R(12) * r2 - R(60) * z2); gy = y * (R(12) * r2 - R(60) * z2); gz = z * (R(80) * z2 - R(48) * r2);
    } else if constexpr (LM == 20) {
        p = x * z * (R(4) * z2 - R(3) * x2 - R(3) * y2); gx = z * (R(4) * z2 - R(9) * x2 - R(3) * y2);
        gy = R(-6) * x * y * z; gz = x * (R(12) * z2 - R(3) * x2 - R(3) * y2);
    } else if constexpr (LM == 21) {
        p = (x2 - y2) * (R(6) * z2 - x2 - y2); gx = x * (R(12) * z2 - R(4) * x2);
        gy = y * (R(4) * y2 - R(12) * z2); gz = R(12) * z * (x2 - y2);
    } else if constexpr (LM == 22) {
        p = x * z * (x2 - R(3) * y2); gx = R(3) * z * (x2 - y2); gy = R(-6) * x * y * z; gz = x * (x2 - R(3) * y2);
    } else {
        p = x2 * x2 - R(6) * x2 * y2 + y2 * y2; gx = R(4) * x * (x2 - R(3) * y2);
        gy = R(4) * y * (y2 - R(3) * x2); gz = 0;
    }
}

// All 24 harmonics and gradients through harm_one (the form the backward kernel uses).
template <typename R, int LM = 0>
__host__ __device__ __forceinline__ void harm_all(R x, R y, R z, R p[NLM], R g[NLM][3]) {
    harm_one<R, LM>(x, y, z, p[LM], g[LM][0], g[LM][1], g[LM][2]);
    if constexpr (LM + 1 < NLM) harm_all<R, LM + 1>(x, y, z, p, g);
}

// ------------------------------------------------------------------ Philox
// Philox4x64-10 (Salmon et al., SC'11): counter (step, atom, stream, 0),
// key (seed, replica).
__device__ __forceinline__ void philox4x64_10(uint64_t &c0, uint64_t &c1, uint64_t &c2, uint64_t &c3,
                                              uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
}

// Three standard normals (Box-Muller on 53-bit uniforms u1 in (0,1], u2 in [0,1)).
__device__ __forceinline__ void gauss3(uint64_t step, uint64_t atom, uint64_t stream, uint64_t seed,
                                       uint64_t replica, double z[3]) {
    uint64_t c0 = step, c1 = atom, c2 = stream, c3 = 0;
    philox4x64_10(c0, c1, c2, c3, seed, replica);
    const double two53 = 1.0 / 9007199254740992.0;
    const double u1 = ((double)(c0 >> 11) + 1.0) * two53, u2 = (double)(c1 >> 11) * two53;
    const double u3 = ((double)(c2 >> 11) + 1.0) * two53, u4 = (double)(c3 >> 11) * two53;
    double s, c;
    const double rho1 = sqrt(-2.0 * log(u1));
    sincospi(2.0 * u2, &s, &c);
    z[0] = rho1 * c;
    z[1] = rho1 * s;
    const double rho2 = sqrt(-2.0 * log(u3));
    z[2] = rho2 * cospi(2.0 * u4);
}

// Three standard normals in FP32 from the same Philox block: 24-bit uniforms
// u1 in (0,1], u2 in [0,1), Box-Muller (the reduced-precision integrator's noise).
__device__ __forceinline__ void gauss3f(uint64_t step, uint64_t atom, uint64_t stream, uint64_t seed,
                                        uint64_t replica, float z[3]) {
    uint64_t c0 = step, c1 = atom, c2 = stream, c3 = 0;
    philox4x64_10(c0, c1, c2, c3, seed, replica);
    const float two24 = 1.0f / 16777216.0f;
    const float u1 = ((float)(c0 >> 40) + 1.0f) * two24, u2 = (float)(c1 >> 40) * two24;
    const float u3 = ((float)(c2 >> 40) + 1.0f) * two24, u4 = (float)(c3 >> 40) * two24;
    float s, c;
    const float rho1 = sqrtf(-2.0f * logf(u1));
    sincospif(2.0f * u2, &s, &c);
    z[0] = rho1 * c;
    z[1] = rho1 * s;
    z[2] = sqrtf(-2.0f * logf(u3)) * cospif(2.0f * u4);
}

// Device status bits.
constexpr int ST_NBR_OVERFLOW = 1;
constexpr int ST_NONFINITE = 2;
constexpr int ST_TIMEOUT = 4;
constexpr int ST_MID_RANGE = 8;     // midpoint configuration beyond the neighbour-list skin
constexpr int ST_BAD_SPECIES = 16;  // a species value outside [0, NS) (no-allocation entry point)

}  // namespace sl
