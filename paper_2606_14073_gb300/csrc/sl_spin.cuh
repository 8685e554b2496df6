// sl_spin.cuh -- spin-update helpers shared by the integrator (sl_integrate.cu) and the
// self-consistent midpoint iteration (sl_midpoint.cu): the damped precession vector,
// the exact Rodrigues rotation (FP64, and an FP32 increment form), and the
// atomics-free force/field gather over an atom's own pair records.
#pragma once

#include "sl_common.cuh"
#include "sl_eval2.cuh"

namespace sl {

template <typename R>
struct GatherArgs {
    const v4<R> *fown, *gii;
    const PairRec<R> *pd;
    const uint32_t *mask;   // in-cutoff candidate slots, [maskw][n]
    int maskw;
    int64_t n;
};

__device__ __forceinline__ void omega_of(double sx, double sy, double sz, double hx, double hy, double hz,
                                         double lam, double k, double w[3]) {
    w[0] = (hx + lam * (sy * hz - sz * hy)) * k;
    w[1] = (hy + lam * (sz * hx - sx * hz)) * k;
    w[2] = (hz + lam * (sx * hy - sy * hx)) * k;
}

__device__ __forceinline__ void rotate(double sx, double sy, double sz, const double w[3], double dt, double out[3]) {
    const double wn2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    if (wn2 == 0.0) { out[0] = sx; out[1] = sy; out[2] = sz; return; }
    const double wn = sqrt(wn2);
    const double ax = w[0] / wn, ay = w[1] / wn, az = w[2] / wn;
    double s, c;
    sincos(wn * dt, &s, &c);
    const double as = ax * sx + ay * sy + az * sz;
    const double cx = ay * sz - az * sy, cy = az * sx - ax * sz, cz = ax * sy - ay * sx;
    out[0] = sx * c + cx * s + ax * as * (1.0 - c);
    out[1] = sy * c + cy * s + ay * as * (1.0 - c);
    out[2] = sz * c + cz * s + az * as * (1.0 - c);
}

// Rotation increment dS = Rot(S, w dt) - S in FP32 (added to the FP64 spin by the
// caller): dS = (a x S) sin(th) - 2 sin^2(th/2) (S - a (a.S)), th = |w| dt.
__device__ __forceinline__ void rotate_delta_f(float sx, float sy, float sz, float wx, float wy, float wz, float dt,
                                               float d[3]) {
    const float wn2 = wx * wx + wy * wy + wz * wz;
    if (wn2 == 0.0f) { d[0] = d[1] = d[2] = 0.0f; return; }
    const float iw = rsqrtf(wn2);
    const float ax = wx * iw, ay = wy * iw, az = wz * iw;
    float sh, ch;
    sincosf(0.5f * wn2 * iw * dt, &sh, &ch);
    const float sn = 2.0f * sh * ch, omc = 2.0f * sh * sh;
    const float as = ax * sx + ay * sy + az * sz;
    d[0] = (ay * sz - az * sy) * sn - omc * (sx - ax * as);
    d[1] = (az * sx - ax * sz) * sn - omc * (sy - ay * as);
    d[2] = (ax * sy - ay * sx) * sn - omc * (sz - az * as);
}

__device__ __forceinline__ void omega_of_f(float sx, float sy, float sz, float hx, float hy, float hz, float lam,
                                           float k, float w[3]) {
    w[0] = (hx + lam * (sy * hz - sz * hy)) * k;
    w[1] = (hy + lam * (sz * hx - sx * hz)) * k;
    w[2] = (hz + lam * (sx * hy - sy * hx)) * k;
}

// F_k = sum_j dE_k/dr_kj - sum_j dE_j/dr_jk, H_k = -dE_k/dS_k - sum_j dE_j/dS_k: the
// records (dE_j/dr_jk, dE_j/dS_k) sit in k's own in-cutoff candidate slots.  The slots
// are walked in order by the whole warp at once, so the records that neighbouring atoms
// read at one slot are neighbours in memory (slot-major layout).
template <typename R>
__device__ __forceinline__ void gather(const GatherArgs<R> &g, int64_t k, double F[3], double H[3]) {
    const v4<R> fo = ro(g.fown + k), gi = ro(g.gii + k);
    R fx = fo.x, fy = fo.y, fz = fo.z, hx = -gi.x, hy = -gi.y, hz = -gi.z;
    const int64_t N = g.n;
#pragma unroll 1
    for (int w = 0; w < g.maskw; ++w) {
        const uint32_t word = ro(g.mask + (int64_t)w * N + k);
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
            if ((word >> b) & 1u) {
                const PairRec<R> *e = g.pd + (int64_t)(w * 32 + b) * N + k;
                const v4<R> ea = ro(&e->a), eb = ro(&e->b);
                fx -= ea.x; fy -= ea.y; fz -= ea.z;
                hx -= ea.w; hy -= eb.x; hz -= eb.y;
            }
        }
    }
    F[0] = (double)fx; F[1] = (double)fy; F[2] = (double)fz;
    H[0] = (double)hx; H[1] = (double)hy; H[2] = (double)hz;
}

}  // namespace sl
