// sl_midpoint.cu -- self-consistent midpoint spin update (arXiv 2606.14073, Section 5.1.3).
//
// The paper augments the explicit predictor-corrector with an optional iteration: from
// the beginning-of-step spins, form a midpoint configuration, re-evaluate force and
// field there, re-apply the one-step update, until a convergence criterion or an
// iteration cap; an accelerated fixed-point variant with regularisation is optional.
// The reading taken here (the same as the FP64 CPU oracle's):
//   r_mid = r_n + (r_{n+1} - r_n)/2      lattice midpoint (written by the first half)
//   X_0   = Rot(S_n, omega(S_n, H_n + eta) dt)      the explicit predictor
//   for m < cap:
//     M_m = (S_n + X_m)/|S_n + X_m|                 midpoint spins      (k_mid_prep)
//     H_m = H(r_mid, M_m)                           evaluation kernels, early exit once stopped
//     G_m = Rot(S_n, omega(M_m, H_m + eta) dt)      (k_mid_update; eta regenerated bit for bit)
//     stop when max_i |G_m,i - X_m,i| < tol or m + 1 = cap            (k_mid_check)
//     X_{m+1} = G_m, or the regularised Anderson mix                  (k_aa_dots/solve/mix)
//   S_{n+1} = G_m renormalised in FP64                                (k_mid_final)
// then the usual evaluation at (r_{n+1}, S_{n+1}) and the final kick.  Every decision
// is taken on the device (flags in MidDev), so a step stays one captured graph.
#include <cstddef>

#include "sl_internal.h"
#include "sl_eval2.cuh"
#include "sl_spin.cuh"

namespace sl {
namespace {

constexpr int AA_BLOCKS = 256;                                 // fixed: deterministic partial sums
constexpr int AA_VALS = AA_MAX_DEPTH * AA_MAX_DEPTH + AA_MAX_DEPTH;

struct MidArgs {
    const double4 *spin_prev;          // S_n
    double4 *spin;                     // state spins: X_0 on entry, S_{n+1} at the end
    float4 *spinf;
    double4 *mids;                     // midpoint spins M_m
    float4 *midsf;
    double4 *X, *G;                    // iterate and its image
    double4 *Xh, *Gh;                  // Anderson rings [(depth + 1)][n]
    double *part;                      // [AA_BLOCKS][AA_VALS]
    const double4 *posmid, *posref;
    const double4 *Bat;                // per-atom part of the external field, or null
    const int32_t *orig;
    int64_t n, n_fe;
    BoxDev<double> bd;
    const StepDev *par;
    const unsigned long long *step;    // step[1]: the step being taken
    int *status;
    MidDev *md;
    uint64_t seed, replica;
    int cap, depth;
    double tol, reg;
};

__global__ void k_mid_start(MidDev *md, int cap) {
    if (threadIdx.x == 0) {
        md->converged = 0;
        md->fallback = 0;
    }
    for (int m = threadIdx.x; m < cap; m += blockDim.x) md->resid[m] = 0ull;
}

__global__ void __launch_bounds__(256) k_mid_prep(MidArgs a, int m) {
    if (a.md->converged) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double4 S0 = a.spin_prev[i];
    double4 X;
    if (m == 0) {
        X = a.spin[i];
        a.X[i] = X;
        // the lists were built for positions within skin/2 of posref; so must the midpoint be
        const double4 p = a.posmid[i], q = a.posref[i];
        double dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
        minimg(a.bd, dx, dy, dz);
        if (dx * dx + dy * dy + dz * dz > a.par->disp2) atomicOr(a.status, ST_MID_RANGE);
    } else {
        X = a.X[i];
    }
    const double mx = S0.x + X.x, my = S0.y + X.y, mz = S0.z + X.z;
    const double inv = 1.0 / sqrt(mx * mx + my * my + mz * mz);
    a.mids[i] = make_double4(mx * inv, my * inv, mz * inv, 0.0);
    a.midsf[i] = make_float4((float)(mx * inv), (float)(my * inv), (float)(mz * inv), 0.f);
}

template <typename R, bool MIXED>
__global__ void __launch_bounds__(256) k_mid_update(MidArgs a, GatherArgs<R> g, int m) {
    if (a.md->converged) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const StepDev &P = *a.par;
    const int t = i < a.n_fe ? 0 : 1;
    double Fs[3], Hs[3];
    gather<R>(g, i, Fs, Hs);
    Hs[0] += P.zee[t][0]; Hs[1] += P.zee[t][1]; Hs[2] += P.zee[t][2];
    if (a.Bat) {
        const double4 b = a.Bat[i];
        Hs[0] += P.mom[t] * b.x; Hs[1] += P.mom[t] * b.y; Hs[2] += P.mom[t] * b.z;
    }
    if (!(isfinite(Hs[0]) && isfinite(Hs[1]) && isfinite(Hs[2]))) atomicOr(a.status, ST_NONFINITE);
    const double4 S0 = a.spin_prev[i], M = a.mids[i], X = a.X[i];
    const unsigned long long st = a.step[1];
    const uint64_t id = (uint64_t)a.orig[i];
    const double se = P.sig_eta;
    double Gn[3];
    if constexpr (MIXED) {
        float ze[3], w[3], d[3];
        gauss3f(st, id, 2, a.seed, a.replica, ze);
        const float fse = (float)se;
        omega_of_f((float)M.x, (float)M.y, (float)M.z, (float)Hs[0] + fse * ze[0], (float)Hs[1] + fse * ze[1],
                   (float)Hs[2] + fse * ze[2], (float)P.lambda, (float)P.wscale, w);
        rotate_delta_f((float)S0.x, (float)S0.y, (float)S0.z, w[0], w[1], w[2], (float)P.dt, d);
        Gn[0] = S0.x + (double)d[0]; Gn[1] = S0.y + (double)d[1]; Gn[2] = S0.z + (double)d[2];
    } else {
        double ze[3], w[3];
        gauss3(st, id, 2, a.seed, a.replica, ze);
        omega_of(M.x, M.y, M.z, Hs[0] + se * ze[0], Hs[1] + se * ze[1], Hs[2] + se * ze[2], P.lambda, P.wscale, w);
        rotate(S0.x, S0.y, S0.z, w, P.dt, Gn);
    }
    const double4 G = make_double4(Gn[0], Gn[1], Gn[2], 0.0);
    a.G[i] = G;
    const double ex = G.x - X.x, ey = G.y - X.y, ez = G.z - X.z;
    const double d = sqrt(ex * ex + ey * ey + ez * ez);
    // non-negative doubles order like their bit patterns: the maximum is order-free
    atomicMax(&a.md->resid[m], (unsigned long long)__double_as_longlong(d));
    if (a.depth == 0) {
        a.X[i] = G;
    } else {
        const int64_t slot = m % (a.depth + 1);
        a.Xh[slot * a.n + i] = X;
        a.Gh[slot * a.n + i] = G;
    }
}

__global__ void k_mid_check(MidDev *md, int m, int cap, double tol) {
    if (md->converged) return;
    md->iters += 1ull;
    const double d = __longlong_as_double((long long)md->resid[m]);
    if (d < tol || m + 1 == cap) md->converged = 1;
}

// ---------------------------------------------------------------- Anderson mix
// f_j = G_j - X_j; column q of dF is f_{m-k+q+1} - f_{m-k+q} (ring slots), k = min(m, depth).
__device__ __forceinline__ void ring_cols(int m, int k, int depth, int q, int &ja, int &jb) {
    ja = (m - k + q + 1) % (depth + 1);
    jb = (m - k + q) % (depth + 1);
}

__global__ void __launch_bounds__(256) k_aa_dots(MidArgs a, int m) {
    if (a.md->converged) return;
    const int k = m < a.depth ? m : a.depth;
    if (k == 0) return;
    __shared__ double red[256];
    double acc[AA_VALS];
    for (int v = 0; v < k * k + k; ++v) acc[v] = 0.0;
    const int64_t cur = m % (a.depth + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double4 gm = a.Gh[cur * a.n + i], xm = a.Xh[cur * a.n + i];
        const double fm[3] = {gm.x - xm.x, gm.y - xm.y, gm.z - xm.z};
        double dF[AA_MAX_DEPTH][3];
        for (int q = 0; q < k; ++q) {
            int ja, jb;
            ring_cols(m, k, a.depth, q, ja, jb);
            const double4 ga = a.Gh[ja * a.n + i], xa = a.Xh[ja * a.n + i];
            const double4 gb = a.Gh[jb * a.n + i], xb = a.Xh[jb * a.n + i];
            dF[q][0] = (ga.x - xa.x) - (gb.x - xb.x);
            dF[q][1] = (ga.y - xa.y) - (gb.y - xb.y);
            dF[q][2] = (ga.z - xa.z) - (gb.z - xb.z);
        }
        for (int q = 0; q < k; ++q) {
            for (int c = 0; c < 3; ++c) acc[k * k + q] += dF[q][c] * fm[c];
            for (int r = 0; r < k; ++r)
                for (int c = 0; c < 3; ++c) acc[q * k + r] += dF[q][c] * dF[r][c];
        }
    }
    // fixed-order tree reduction per value
    for (int v = 0; v < k * k + k; ++v) {
        red[threadIdx.x] = acc[v];
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.part[(int64_t)blockIdx.x * AA_VALS + v] = red[0];
        __syncthreads();
    }
}

__global__ void k_aa_solve(MidArgs a, int m) {
    if (a.md->converged) return;
    const int k = m < a.depth ? m : a.depth;
    if (k == 0) return;
    __shared__ double sum[AA_VALS];
    for (int v = threadIdx.x; v < k * k + k; v += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < AA_BLOCKS; ++b) s += a.part[(int64_t)b * AA_VALS + v];
        sum[v] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double A[AA_MAX_DEPTH * AA_MAX_DEPTH], y[AA_MAX_DEPTH];
    double tr = 0.0;
    for (int q = 0; q < k; ++q) {
        y[q] = sum[k * k + q];
        for (int r = 0; r < k; ++r) A[q * k + r] = sum[q * k + r];
        tr += A[q * k + q];
    }
    int ok = tr > 0.0;
    const double delta = a.reg * tr / k;
    for (int q = 0; q < k; ++q) A[q * k + q] += delta;
    // Cholesky A = L L^T in place, then L z = y, L^T g = z
    for (int j = 0; j < k && ok; ++j) {
        double d = A[j * k + j];
        for (int q = 0; q < j; ++q) d -= A[j * k + q] * A[j * k + q];
        if (!(d > 0.0)) { ok = 0; break; }
        d = sqrt(d);
        A[j * k + j] = d;
        for (int i = j + 1; i < k; ++i) {
            double v = A[i * k + j];
            for (int q = 0; q < j; ++q) v -= A[i * k + q] * A[j * k + q];
            A[i * k + j] = v / d;
        }
    }
    if (ok) {
        for (int i = 0; i < k; ++i) {
            double v = y[i];
            for (int q = 0; q < i; ++q) v -= A[i * k + q] * y[q];
            y[i] = v / A[i * k + i];
        }
        for (int i = k - 1; i >= 0; --i) {
            double v = y[i];
            for (int q = i + 1; q < k; ++q) v -= A[q * k + i] * y[q];
            y[i] = v / A[i * k + i];
        }
        for (int q = 0; q < k; ++q) a.md->gamma[q] = y[q];
    }
    a.md->fallback = ok ? 0 : 1;
}

__global__ void __launch_bounds__(256) k_aa_mix(MidArgs a, int m) {
    if (a.md->converged) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int k = m < a.depth ? m : a.depth;
    const double4 G = a.G[i];
    if (k == 0 || a.md->fallback) {
        a.X[i] = G;
        return;
    }
    double x = G.x, y = G.y, z = G.z;
    for (int q = 0; q < k; ++q) {
        int ja, jb;
        ring_cols(m, k, a.depth, q, ja, jb);
        const double gq = a.md->gamma[q];
        const double4 ga = a.Gh[ja * a.n + i], gb = a.Gh[jb * a.n + i];
        x -= gq * (ga.x - gb.x);
        y -= gq * (ga.y - gb.y);
        z -= gq * (ga.z - gb.z);
    }
    const double inv = 1.0 / sqrt(x * x + y * y + z * z);
    a.X[i] = make_double4(x * inv, y * inv, z * inv, 0.0);
}

__global__ void __launch_bounds__(256) k_mid_final(MidArgs a) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double4 G = a.G[i];
    const double inv = 1.0 / sqrt(G.x * G.x + G.y * G.y + G.z * G.z);
    const double sx = G.x * inv, sy = G.y * inv, sz = G.z * inv;
    a.spin[i] = make_double4(sx, sy, sz, 0.0);
    a.spinf[i] = make_float4((float)sx, (float)sy, (float)sz, 0.f);
}

MidArgs mid_args(Sys &s) {
    MidArgs a;
    a.spin_prev = s.spin_prev; a.spin = s.spin; a.spinf = s.spinf;
    a.mids = s.mids; a.midsf = s.midsf; a.X = s.mx; a.G = s.mg; a.Xh = s.aax; a.Gh = s.aag; a.part = s.aapart;
    a.posmid = s.posmid; a.posref = s.posref; a.Bat = s.Bat; a.orig = s.orig; a.n = s.n; a.n_fe = s.n_fe; a.bd = s.boxd;
    a.par = s.d_par; a.step = s.d_step; a.status = s.status; a.md = s.md; a.seed = s.seed; a.replica = s.replica;
    a.cap = s.mid_iters; a.depth = s.aa_depth; a.tol = s.mid_tol; a.reg = s.aa_reg;
    return a;
}

template <typename R>
GatherArgs<R> mid_gather_args(Sys &s) {
    GatherArgs<R> g;
    g.fown = (const v4<R> *)s.fown; g.gii = (const v4<R> *)s.gii; g.pd = (const PairRec<R> *)s.pairs;
    g.mask = s.cmask; g.maskw = s.maskw; g.n = s.n;
    return g;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int midpoint_kernels_per_step(const Sys &s) {
    if (s.mid_iters <= 0) return 0;
    return 1 + s.mid_iters * (1 + 4 + 1 + 1 + (s.aa_depth > 0 ? 3 : 0)) + 1;
}

size_t midpoint_scratch_doubles() { return (size_t)AA_BLOCKS * AA_VALS; }

int launch_midpoint(Sys &s) {
    if (s.mid_iters <= 0 || s.n == 0) return 0;
    const MidArgs a = mid_args(s);
    const unsigned nb = nblk(s.n, 256);
    k_mid_start<<<1, 64, 0, s.stream>>>(s.md, s.mid_iters);
    EvalAt at;
    at.pos = s.posmid; at.posf = s.posmidf; at.spin = s.mids; at.spinf = s.midsf;
    at.skip = reinterpret_cast<const int *>(reinterpret_cast<const char *>(s.md) + offsetof(MidDev, converged));
    for (int m = 0; m < s.mid_iters; ++m) {
        k_mid_prep<<<nb, 256, 0, s.stream>>>(a, m);
        s.at = at;
        launch_eval(s, false);
        s.at = EvalAt();
        if (s.prec == 0) k_mid_update<double, false><<<nb, 256, 0, s.stream>>>(a, mid_gather_args<double>(s), m);
        else k_mid_update<float, true><<<nb, 256, 0, s.stream>>>(a, mid_gather_args<float>(s), m);
        k_mid_check<<<1, 1, 0, s.stream>>>(s.md, m, s.mid_iters, s.mid_tol);
        if (s.aa_depth > 0) {
            k_aa_dots<<<AA_BLOCKS, 256, 0, s.stream>>>(a, m);
            k_aa_solve<<<1, 64, 0, s.stream>>>(a, m);
            k_aa_mix<<<nb, 256, 0, s.stream>>>(a, m);
        }
    }
    k_mid_final<<<nb, 256, 0, s.stream>>>(a);
    return midpoint_kernels_per_step(s);
}

}  // namespace sl
