/*
 * nepspin_oracle.c -- plain FP64 CPU oracle for the NEP-SPIN spin-lattice step.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark are the only callers; the product (CUDA) path never loads
 * this library and shares no code, header, table or constant generator with it.
 *
 * What it computes (arXiv 2606.14073, Sections 3, 5.1.1-5.1.3, 5.2.1):
 *   E(R,S) = sum_i E_i(q_i) + E_Zeeman,  q_i the 66-entry spin-aware NEP descriptor,
 *   F_i = -dE/dr_i,  H_i = -dE/dS_i (unconstrained R^3 gradient, Zeeman included),
 *   virial W_ab = -sum_i sum_j (r_ij)_a dE_i/d(r_ij)_b,
 * and the spin-lattice integrator step (velocity-Verlet halves, lattice Langevin
 * O-step, predictor-corrector spin rotation with the spin update last).
 *
 * The paper prints no formulas for the descriptor, the network or the integrator.
 * The readings taken here (each also listed in the design notes):
 *  - radial carrier (Section 5.2.3, 5.2.4: Chebyshev T_k/U_k recurrences, basis
 *    size 8 = 9 terms): f_c(r) = (1+cos(pi r/rc))/2, x = 2(r/rc-1)^2-1,
 *    f_k = (T_k(x)+1) f_c / 2, k = 0..K-1, dT_k/dx = k U_{k-1};
 *  - group radial functions g^G_n = sum_k c^G_{n k t_i t_j} f_k for the groups
 *    G = R (structural radial), A (structural angular), and the four pairwise
 *    magnetic sub-terms EX, DMI, ANI, SIA named in Section 5.2.4;
 *  - descriptor, 66 entries for 5 channels (Section 5.2.3 gives 66 Fp entries):
 *      [R(5), A(n,l)(20), O(1), EX(5), DMI(5), ANI(5), SIA(5), SA(n,l)(20)]
 *    R_n   = sum_j g^R_n(r_ij)                                  (r < rc_R)
 *    A_nl  = sum_{j,k} g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_jik), j = k included,
 *            l = 1..4                                           (r < rc_A)
 *    O     = |S_i|^2                             (onsite group, Section 5.1.2)
 *    X_n   = sum_j g^X_n(r_ij) phi_X, phi_EX = S_i.S_j, phi_DMI = (S_i x S_j).u,
 *            phi_ANI = (S_i.u)(S_j.u), phi_SIA = (S_i.u)^2      (pairwise group)
 *    SA_nl = sum_{j,k} g^A_n(r_ij)(S_i.S_j) g^A_n(r_ik)(S_i.S_k) P_l(cos theta_jik)
 *            (spin-weighted angular group, Section 5.1.2)
 *  - network (Section 5.2.3 "ANN", one hidden tanh layer):
 *      E_i = sum_h w1_h tanh(sum_v W0_hv s_v q_v - b0_h) - b1;
 *  - Zeeman: E_Z = -sum_i mu_i mu_B B_i.S_i, B_i = B + (optional per-atom part);
 *  - optional Landau onsite energy for variable moment lengths (longitudinal
 *    fluctuation, Section 3): E_L = sum_i a_t |S_i|^2 + b_t |S_i|^4 per species t.
 * The angular channels are evaluated here as the plain Legendre double sum over
 * neighbour pairs (their definition), not through spherical harmonics.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared
 * (-ffp-contract=off keeps the neighbour distance test bit-defined).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_G_R 0
#define OR_G_A 1
#define OR_G_EX 2
#define OR_G_DMI 3
#define OR_G_ANI 4
#define OR_G_SIA 5
#define OR_NGROUP 6
#define OR_LMAX 4
#define OR_MAXCH 8
#define OR_MAXK 16
#define OR_MAXH 64
#define OR_MAXD (1 + 13 * OR_MAXCH)

/* Physical constants (CODATA 2018). */
#define OR_KB 8.617333262e-5          /* eV / K              */
#define OR_HBAR 0.6582119569          /* eV fs               */
#define OR_MUB 5.7883818060e-5        /* eV / T              */
#define OR_ACC 9.6485332e-3           /* (eV/A/amu) -> A/fs^2 */

typedef struct {
    int32_t n_species;     /* number of species (2: Fe, Ge)          */
    int32_t n_ch;          /* radial channels n = 0..n_ch-1 (5)      */
    int32_t basis_k;       /* Chebyshev terms k = 0..basis_k-1 (9)   */
    int32_t n_hidden;      /* hidden tanh units (30)                 */
    double rc_rad, rc_ang; /* cutoffs, A                             */
    const double *coeffs;  /* [ns][ns][6][n_ch][basis_k]             */
    const double *q_scaler;/* [D]                                    */
    const double *w0;      /* [n_hidden][D]                          */
    const double *b0;      /* [n_hidden]                             */
    const double *w1;      /* [n_hidden]                             */
    double b1;
    const double *mass_amu;   /* [ns] */
    const double *moment_muB; /* [ns] */
    const double *B_atoms;    /* [n][3] per-atom external field, T, added to the uniform B;
                                 NULL: none (the same field on every atom)          */
    const double *landau;     /* [ns][2] (a, b) of E_L = a|S|^2 + b|S|^4, eV; NULL: none */
} or_params;

/* Landau onsite energy of atom i and its field -dE_L/dS_i. */
static double landau_at(const or_params *P, int t, const double S[3], double h[3]) {
    if (!P->landau) { h[0] = h[1] = h[2] = 0.0; return 0.0; }
    const double a = P->landau[2 * t], b = P->landau[2 * t + 1];
    const double m2 = S[0] * S[0] + S[1] * S[1] + S[2] * S[2];
    const double k = -(2.0 * a + 4.0 * b * m2);
    for (int c = 0; c < 3; ++c) h[c] = k * S[c];
    return a * m2 + b * m2 * m2;
}

/* External field on atom i: the uniform B plus the atom's own part. */
static void field_at(const or_params *P, const double B[3], int64_t i, double out[3]) {
    for (int c = 0; c < 3; ++c) out[c] = B[c] + (P->B_atoms ? P->B_atoms[3 * i + c] : 0.0);
}

typedef struct {
    double gamma_lattice;  /* 1/fs, Langevin friction of the lattice O-step   */
    double lambda_spin;    /* Gilbert damping of the stochastic spin update  */
    uint64_t seed;         /* Philox key word 0                              */
    uint64_t replica;      /* Philox key word 1                              */
    int32_t midpoint_iters;   /* 0: predictor-corrector; > 0: cap of the midpoint iteration */
    int32_t anderson_depth;   /* 0: plain fixed-point iteration; > 0: Anderson history     */
    double midpoint_tol;      /* stop when max_i |G_i - X_i| < tol (0: always the cap)      */
    double anderson_reg;      /* Tikhonov weight, relative to the mean diagonal              */
    int32_t longitudinal;     /* 1: variable moment lengths (no renormalisation)            */
    double alpha_long;        /* dimensionless damping of the longitudinal mode              */
    int32_t st_sweep;         /* 1: coloured Suzuki-Trotter spin sweep instead of the
                                 predictor-corrector spin update                            */
} or_dynamics;

static int or_dim(int n_ch) { return 1 + 13 * n_ch; }
static int iR(int n) { return n; }
static int iA(int nch, int n, int l) { return nch + n * OR_LMAX + (l - 1); }
static int iO(int nch) { return nch + OR_LMAX * nch; }
static int iX(int nch, int g, int n) { return iO(nch) + 1 + (g - OR_G_EX) * nch + n; }
static int iSA(int nch, int n, int l) { return iO(nch) + 1 + 4 * nch + n * OR_LMAX + (l - 1); }

/* ------------------------------------------------------------------ Philox */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds, the key bumped by the
 * Weyl constants between rounds.  Multipliers and Weyl constants as published. */
static void or_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        or_mulhilo64(M0, c0, &hi0, &lo0);
        or_mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Four standard normals for (step, atom, stream) under key (seed, replica):
 * Box-Muller on 53-bit uniforms u1 in (0,1], u2 in [0,1). */
void or_gauss4(uint64_t step, uint64_t atom, uint64_t stream, uint64_t seed, uint64_t replica,
               double out[4]) {
    uint64_t ctr[4] = {step, atom, stream, 0}, key[2] = {seed, replica}, x[4];
    or_philox4x64_10(ctr, key, x);
    const double two53 = 1.0 / 9007199254740992.0;
    for (int p = 0; p < 2; ++p) {
        double u1 = ((double)(x[2 * p] >> 11) + 1.0) * two53;
        double u2 = (double)(x[2 * p + 1] >> 11) * two53;
        double rho = sqrt(-2.0 * log(u1));
        out[2 * p] = rho * cos(2.0 * M_PI * u2);
        out[2 * p + 1] = rho * sin(2.0 * M_PI * u2);
    }
}

/* --------------------------------------------------------------- carrier */
/* Chebyshev polynomials of the first kind T_k(x) and their x-derivatives
 * k U_{k-1}(x), from the two three-term recurrences. */
void or_chebyshev(double x, int K, double *T, double *dT) {
    double U[OR_MAXK + 1];
    T[0] = 1.0;
    if (K > 1) T[1] = x;
    for (int k = 2; k < K; ++k) T[k] = 2.0 * x * T[k - 1] - T[k - 2];
    U[0] = 1.0;
    U[1] = 2.0 * x;
    for (int k = 2; k < K; ++k) U[k] = 2.0 * x * U[k - 1] - U[k - 2];
    dT[0] = 0.0;
    for (int k = 1; k < K; ++k) dT[k] = (double)k * U[k - 1];
}

/* Radial basis f_k(r) and df_k/dr for cutoff rc (zero beyond rc). */
void or_carrier(double r, double rc, int K, double *f, double *df) {
    if (r >= rc) {
        for (int k = 0; k < K; ++k) { f[k] = 0.0; df[k] = 0.0; }
        return;
    }
    double fc = 0.5 * (1.0 + cos(M_PI * r / rc));
    double dfc = -0.5 * M_PI / rc * sin(M_PI * r / rc);
    double y = r / rc - 1.0;
    double x = 2.0 * y * y - 1.0;
    double dxdr = 4.0 * y / rc;
    double T[OR_MAXK], dT[OR_MAXK];
    or_chebyshev(x, K, T, dT);
    for (int k = 0; k < K; ++k) {
        f[k] = 0.5 * (T[k] + 1.0) * fc;
        df[k] = 0.5 * dT[k] * dxdr * fc + 0.5 * (T[k] + 1.0) * dfc;
    }
}

/* Legendre polynomials P_l and P_l' for l = 1..4. */
static double leg(int l, double x) {
    switch (l) {
    case 1: return x;
    case 2: return 0.5 * (3.0 * x * x - 1.0);
    case 3: return 0.5 * (5.0 * x * x * x - 3.0 * x);
    default: return 0.125 * (35.0 * x * x * x * x - 30.0 * x * x + 3.0);
    }
}
static double dleg(int l, double x) {
    switch (l) {
    case 1: return 1.0;
    case 2: return 3.0 * x;
    case 3: return 0.5 * (15.0 * x * x - 3.0);
    default: return 0.125 * (140.0 * x * x * x - 60.0 * x);
    }
}

/* ------------------------------------------------------------ neighbours */
/* Minimum-image separation r_j - r_i and its squared length.  The operation order
 * is the bit-exact definition of the neighbour test:
 *   t = x_j - x_i;  t = t - L * rint(t / L)  (periodic dims only);
 *   d2 = (dx*dx + dy*dy) + dz*dz. */
static double sep(const double *pos, int64_t i, int64_t j, const double *box, const int32_t *per,
                  double d[3]) {
    for (int a = 0; a < 3; ++a) {
        double t = pos[3 * j + a] - pos[3 * i + a];
        if (per[a]) {
            double q = rint(t / box[a]);
            double s = box[a] * q;
            t = t - s;
        }
        d[a] = t;
    }
    double xx = d[0] * d[0];
    double yy = d[1] * d[1];
    double zz = d[2] * d[2];
    double s = xx + yy;
    return s + zz;
}

typedef struct {
    int64_t *off;   /* [n+1] */
    int32_t *idx;   /* [off[n]] neighbour j, ascending */
} or_nlist;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* All pairs with d2 < cut^2, by brute force (method 0) or by a cell list (method 1).
 * Lists are ascending in j.  Returns 0, or -1 on allocation failure. */
static int build_nlist(int64_t n, const double *pos, const double *box, const int32_t *per,
                       double cut, int method, or_nlist *out) {
    const double cut2 = cut * cut;
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    int nc[3] = {1, 1, 1};
    int64_t *cell_start = NULL, *cell_atoms = NULL;
    int32_t *cell_of = NULL;
    if (method == 1) {
        for (int a = 0; a < 3; ++a) {
            nc[a] = (int)floor(box[a] / (cut * (1.0 + 1e-9)));
            if (nc[a] < 1) nc[a] = 1;
        }
        int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
        cell_start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
        cell_atoms = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        if (!cell_start || !cell_atoms || !cell_of) return -1;
        for (int64_t i = 0; i < n; ++i) {
            int c[3];
            for (int a = 0; a < 3; ++a) {
                double w = box[a] / nc[a];
                double x = pos[3 * i + a];
                if (per[a]) x = x - box[a] * floor(x / box[a]);
                int ci = (int)floor(x / w);
                if (ci < 0) ci = 0;
                if (ci >= nc[a]) ci = nc[a] - 1;
                c[a] = ci;
            }
            cell_of[i] = (int32_t)((c[2] * nc[1] + c[1]) * nc[0] + c[0]);
            cell_start[cell_of[i] + 1]++;
        }
        for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
        if (!fill) return -1;
        memcpy(fill, cell_start, sizeof(int64_t) * (size_t)ncell);
        for (int64_t i = 0; i < n; ++i) cell_atoms[fill[cell_of[i]]++] = i;
        free(fill);
    }
    /* two passes: count, then fill */
    int32_t **tmp = (int32_t **)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t *));
    if (!tmp) return -1;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t capn = 64, m = 0;
        int32_t *lst = (int32_t *)malloc(sizeof(int32_t) * (size_t)capn);
        double d[3];
        if (method == 0) {
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                if (sep(pos, i, j, box, per, d) < cut2) {
                    if (m == capn) { capn *= 2; lst = (int32_t *)realloc(lst, sizeof(int32_t) * (size_t)capn); }
                    lst[m++] = (int32_t)j;
                }
            }
        } else {
            int ci[3];
            int32_t cc = cell_of[i];
            ci[0] = cc % nc[0]; ci[1] = (cc / nc[0]) % nc[1]; ci[2] = cc / (nc[0] * nc[1]);
            int lo[3], hi[3];
            for (int a = 0; a < 3; ++a) {
                if (per[a] && nc[a] < 3) { lo[a] = 0; hi[a] = nc[a] - 1; }
                else if (per[a]) { lo[a] = ci[a] - 1; hi[a] = ci[a] + 1; }
                else { lo[a] = ci[a] > 0 ? ci[a] - 1 : 0; hi[a] = ci[a] < nc[a] - 1 ? ci[a] + 1 : nc[a] - 1; }
            }
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) {
                        int wx = (x % nc[0] + nc[0]) % nc[0];
                        int wy = (y % nc[1] + nc[1]) % nc[1];
                        int wz = (z % nc[2] + nc[2]) % nc[2];
                        int64_t c = ((int64_t)wz * nc[1] + wy) * nc[0] + wx;
                        for (int64_t p = cell_start[c]; p < cell_start[c + 1]; ++p) {
                            int64_t j = cell_atoms[p];
                            if (j == i) continue;
                            if (sep(pos, i, j, box, per, d) < cut2) {
                                if (m == capn) { capn *= 2; lst = (int32_t *)realloc(lst, sizeof(int32_t) * (size_t)capn); }
                                lst[m++] = (int32_t)j;
                            }
                        }
                    }
            qsort(lst, (size_t)m, sizeof(int32_t), cmp_i32);
        }
        if (!lst) fail = 1;
        tmp[i] = lst;
        cnt[i + 1] = m;
    }
    free(cell_start); free(cell_atoms); free(cell_of);
    if (fail) return -1;
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    out->off = cnt;
    out->idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
    if (!out->idx) return -1;
    for (int64_t i = 0; i < n; ++i) {
        memcpy(out->idx + cnt[i], tmp[i], sizeof(int32_t) * (size_t)(cnt[i + 1] - cnt[i]));
        free(tmp[i]);
    }
    free(tmp);
    return 0;
}

static void free_nlist(or_nlist *l) { free(l->off); free(l->idx); l->off = NULL; l->idx = NULL; }

/* Neighbour sets {j : d2(i,j) < cut^2}, ascending, written as counts[n] and
 * lists[n][cap].  Returns 0, -1 (allocation) or -2 (a count above cap). */
int or_neighbors(int64_t n, const double *pos, const double *box, const int32_t *per, double cut,
                 int method, int32_t cap, int32_t *counts, int32_t *lists) {
    or_nlist nl;
    if (build_nlist(n, pos, box, per, cut, method, &nl)) return -1;
    int rc = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t m = nl.off[i + 1] - nl.off[i];
        counts[i] = (int32_t)m;
        if (m > cap) { rc = -2; m = cap; }
        memcpy(lists + i * (int64_t)cap, nl.idx + nl.off[i], sizeof(int32_t) * (size_t)m);
    }
    free_nlist(&nl);
    return rc;
}

/* ------------------------------------------------------- per-atom model */
static double coef(const or_params *P, int ti, int tj, int g, int n, int k) {
    int64_t o = ((((int64_t)ti * P->n_species + tj) * OR_NGROUP + g) * P->n_ch + n) * P->basis_k + k;
    return P->coeffs[o];
}

typedef struct {
    double E;          /* E_i (network output)                                  */
    double q[OR_MAXD]; /* descriptor                                            */
    double Fp[OR_MAXD];/* dE_i/dq_i                                             */
} or_atom;

/* Descriptor of atom i over its in-cutoff radial neighbours nb[0..m) (with the
 * angular ones, r < rc_ang, a subset).  If want_grad, also the network output,
 * Fp, and the derivatives D[a] = dE_i/dr_ij, G[a] = dE_i/dS_j (a over nb) and
 * Gii = dE_i/dS_i. */
static void atom_eval(const or_params *P, int64_t i, const int32_t *nb, int64_t m, const double *pos,
                      const double *spin, const int32_t *species, const double *box, const int32_t *per,
                      int want_grad, or_atom *A, double *D, double *G, double *Gii) {
    const int NC = P->n_ch, K = P->basis_k, Dm = or_dim(NC), NH = P->n_hidden;
    const int ti = species[i];
    const double *Si = spin + 3 * i;
    double *q = A->q;
    for (int v = 0; v < Dm; ++v) q[v] = 0.0;

    /* per-neighbour scratch */
    double (*u)[3] = malloc(sizeof(double[3]) * (size_t)(m > 0 ? m : 1));
    double *r = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double (*g)[OR_NGROUP][OR_MAXCH] = malloc(sizeof(double[OR_NGROUP][OR_MAXCH]) * (size_t)(m > 0 ? m : 1));
    double (*dg)[OR_NGROUP][OR_MAXCH] = malloc(sizeof(double[OR_NGROUP][OR_MAXCH]) * (size_t)(m > 0 ? m : 1));
    int *ang = malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    double *sdot = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double (*phi)[4] = malloc(sizeof(double[4]) * (size_t)(m > 0 ? m : 1));

    const double rcA2 = P->rc_ang * P->rc_ang;
    for (int64_t a = 0; a < m; ++a) {
        int64_t j = nb[a];
        int tj = species[j];
        double d[3];
        double d2 = sep(pos, i, j, box, per, d);
        r[a] = sqrt(d2);
        for (int c = 0; c < 3; ++c) u[a][c] = d[c] / r[a];
        const double *Sj = spin + 3 * j;
        double f[OR_MAXK], df[OR_MAXK];
        or_carrier(r[a], P->rc_rad, K, f, df);
        for (int gg = 0; gg < OR_NGROUP; ++gg) {
            if (gg == OR_G_A) continue;
            for (int n = 0; n < NC; ++n) {
                double s = 0.0, ds = 0.0;
                for (int k = 0; k < K; ++k) {
                    s += coef(P, ti, tj, gg, n, k) * f[k];
                    ds += coef(P, ti, tj, gg, n, k) * df[k];
                }
                g[a][gg][n] = s;
                dg[a][gg][n] = ds;
            }
        }
        double siu = Si[0] * u[a][0] + Si[1] * u[a][1] + Si[2] * u[a][2];
        double sju = Sj[0] * u[a][0] + Sj[1] * u[a][1] + Sj[2] * u[a][2];
        double cx[3] = {Si[1] * Sj[2] - Si[2] * Sj[1], Si[2] * Sj[0] - Si[0] * Sj[2], Si[0] * Sj[1] - Si[1] * Sj[0]};
        sdot[a] = Si[0] * Sj[0] + Si[1] * Sj[1] + Si[2] * Sj[2];
        phi[a][0] = sdot[a];                                           /* EX  */
        phi[a][1] = cx[0] * u[a][0] + cx[1] * u[a][1] + cx[2] * u[a][2]; /* DMI */
        phi[a][2] = siu * sju;                                         /* ANI */
        phi[a][3] = siu * siu;                                         /* SIA */
        for (int n = 0; n < NC; ++n) {
            q[iR(n)] += g[a][OR_G_R][n];
            for (int x = 0; x < 4; ++x) q[iX(NC, OR_G_EX + x, n)] += g[a][OR_G_EX + x][n] * phi[a][x];
        }
        ang[a] = d2 < rcA2;
        if (ang[a]) {
            or_carrier(r[a], P->rc_ang, K, f, df);
            for (int n = 0; n < NC; ++n) {
                double s = 0.0, ds = 0.0;
                for (int k = 0; k < K; ++k) {
                    s += coef(P, ti, tj, OR_G_A, n, k) * f[k];
                    ds += coef(P, ti, tj, OR_G_A, n, k) * df[k];
                }
                g[a][OR_G_A][n] = s;
                dg[a][OR_G_A][n] = ds;
            }
        } else {
            for (int n = 0; n < NC; ++n) { g[a][OR_G_A][n] = 0.0; dg[a][OR_G_A][n] = 0.0; }
        }
    }
    q[iO(NC)] = Si[0] * Si[0] + Si[1] * Si[1] + Si[2] * Si[2];
    /* angular channels as the Legendre double sum over ordered neighbour pairs */
    for (int64_t a = 0; a < m; ++a) {
        if (!ang[a]) continue;
        for (int64_t b = 0; b < m; ++b) {
            if (!ang[b]) continue;
            double c = (a == b) ? 1.0 : u[a][0] * u[b][0] + u[a][1] * u[b][1] + u[a][2] * u[b][2];
            for (int l = 1; l <= OR_LMAX; ++l) {
                double Pl = leg(l, c);
                for (int n = 0; n < NC; ++n) {
                    double gg = g[a][OR_G_A][n] * g[b][OR_G_A][n];
                    q[iA(NC, n, l)] += gg * Pl;
                    q[iSA(NC, n, l)] += gg * sdot[a] * sdot[b] * Pl;
                }
            }
        }
    }
    if (!want_grad) goto done;

    /* network: E_i = sum_h w1_h tanh(z_h) - b1, z_h = sum_v W0_hv s_v q_v - b0_h */
    {
        double th[OR_MAXH];
        double E = -P->b1;
        for (int h = 0; h < NH; ++h) {
            double z = -P->b0[h];
            for (int v = 0; v < Dm; ++v) z += P->w0[(int64_t)h * Dm + v] * P->q_scaler[v] * q[v];
            th[h] = tanh(z);
            E += P->w1[h] * th[h];
        }
        A->E = E;
        for (int v = 0; v < Dm; ++v) {
            double s = 0.0;
            for (int h = 0; h < NH; ++h) s += P->w1[h] * (1.0 - th[h] * th[h]) * P->w0[(int64_t)h * Dm + v];
            A->Fp[v] = s * P->q_scaler[v];
        }
    }
    const double *Fp = A->Fp;
    for (int c = 0; c < 3; ++c) Gii[c] = 2.0 * Fp[iO(NC)] * Si[c];
    for (int64_t a = 0; a < m; ++a) {
        int64_t j = nb[a];
        const double *Sj = spin + 3 * j;
        double *Da = D + 3 * a, *Ga = G + 3 * a;
        const double *ua = u[a];
        double ra = r[a];
        for (int c = 0; c < 3; ++c) { Da[c] = 0.0; Ga[c] = 0.0; }
        double siu = Si[0] * ua[0] + Si[1] * ua[1] + Si[2] * ua[2];
        double sju = Sj[0] * ua[0] + Sj[1] * ua[1] + Sj[2] * ua[2];
        double w[3] = {Si[1] * Sj[2] - Si[2] * Sj[1], Si[2] * Sj[0] - Si[0] * Sj[2], Si[0] * Sj[1] - Si[1] * Sj[0]};
        double wu = w[0] * ua[0] + w[1] * ua[1] + w[2] * ua[2];
        double uxsi[3] = {ua[1] * Si[2] - ua[2] * Si[1], ua[2] * Si[0] - ua[0] * Si[2], ua[0] * Si[1] - ua[1] * Si[0]};
        double sjxu[3] = {Sj[1] * ua[2] - Sj[2] * ua[1], Sj[2] * ua[0] - Sj[0] * ua[2], Sj[0] * ua[1] - Sj[1] * ua[0]};
        /* gradients of the pair spin functions with respect to r_ij */
        double gDMI[3], gANI[3], gSIA[3];
        for (int c = 0; c < 3; ++c) {
            double pSi = Si[c] - siu * ua[c], pSj = Sj[c] - sju * ua[c];
            gDMI[c] = (w[c] - wu * ua[c]) / ra;
            gANI[c] = (sju * pSi + siu * pSj) / ra;
            gSIA[c] = 2.0 * siu * pSi / ra;
        }
        double radial = 0.0; /* coefficient of u */
        for (int n = 0; n < NC; ++n) {
            double FR = Fp[iR(n)];
            double FEX = Fp[iX(NC, OR_G_EX, n)], FDMI = Fp[iX(NC, OR_G_DMI, n)];
            double FANI = Fp[iX(NC, OR_G_ANI, n)], FSIA = Fp[iX(NC, OR_G_SIA, n)];
            radial += FR * dg[a][OR_G_R][n];
            radial += FEX * dg[a][OR_G_EX][n] * phi[a][0];
            radial += FDMI * dg[a][OR_G_DMI][n] * phi[a][1];
            radial += FANI * dg[a][OR_G_ANI][n] * phi[a][2];
            radial += FSIA * dg[a][OR_G_SIA][n] * phi[a][3];
            for (int c = 0; c < 3; ++c) {
                Da[c] += FDMI * g[a][OR_G_DMI][n] * gDMI[c] + FANI * g[a][OR_G_ANI][n] * gANI[c] +
                         FSIA * g[a][OR_G_SIA][n] * gSIA[c];
                Ga[c] += FEX * g[a][OR_G_EX][n] * Si[c] + FDMI * g[a][OR_G_DMI][n] * uxsi[c] +
                         FANI * g[a][OR_G_ANI][n] * siu * ua[c];
                Gii[c] += FEX * g[a][OR_G_EX][n] * Sj[c] + FDMI * g[a][OR_G_DMI][n] * sjxu[c] +
                          FANI * g[a][OR_G_ANI][n] * sju * ua[c] + FSIA * g[a][OR_G_SIA][n] * 2.0 * siu * ua[c];
            }
        }
        for (int c = 0; c < 3; ++c) Da[c] += radial * ua[c];
    }
    /* angular channels, differentiated in their Legendre double-sum form */
    for (int64_t a = 0; a < m; ++a) {
        if (!ang[a]) continue;
        double *Da = D + 3 * a, *Ga = G + 3 * a;
        const double *Sa = spin + 3 * nb[a];
        for (int64_t b = 0; b < m; ++b) {
            if (!ang[b]) continue;
            double c = (a == b) ? 1.0 : u[a][0] * u[b][0] + u[a][1] * u[b][1] + u[a][2] * u[b][2];
            double dc[3];
            for (int x = 0; x < 3; ++x) dc[x] = (u[b][x] - c * u[a][x]) / r[a];
            for (int l = 1; l <= OR_LMAX; ++l) {
                double Pl = leg(l, c), dPl = dleg(l, c);
                for (int n = 0; n < NC; ++n) {
                    double FA = Fp[iA(NC, n, l)], FS = Fp[iSA(NC, n, l)];
                    double ga = g[a][OR_G_A][n], gb = g[b][OR_G_A][n], dga = dg[a][OR_G_A][n];
                    double sab = sdot[a] * sdot[b];
                    double radial = 2.0 * (FA + FS * sab) * dga * gb * Pl;
                    double angular = 2.0 * (FA + FS * sab) * ga * gb * dPl;
                    for (int x = 0; x < 3; ++x) {
                        Da[x] += radial * u[a][x] + angular * dc[x];
                        Ga[x] += 2.0 * FS * ga * gb * sdot[b] * Pl * Si[x];
                        Gii[x] += 2.0 * FS * ga * gb * sdot[b] * Pl * Sa[x];
                    }
                }
            }
        }
    }
done:
    free(u); free(r); free(g); free(dg); free(ang); free(sdot); free(phi);
}

/* ---------------------------------------------------------- evaluations */
static int check_params(const or_params *P) {
    if (P->n_ch < 1 || P->n_ch > OR_MAXCH || P->basis_k < 2 || P->basis_k > OR_MAXK ||
        P->n_hidden < 1 || P->n_hidden > OR_MAXH || P->n_species < 1 || P->rc_ang > P->rc_rad)
        return -3;
    return 0;
}

/* Descriptors q[n][D] of every atom. */
int or_descriptors(int64_t n, const double *pos, const double *spin, const int32_t *species,
                   const double *box, const int32_t *per, const or_params *P, double *q_out) {
    if (check_params(P)) return -3;
    or_nlist nl;
    if (build_nlist(n, pos, box, per, P->rc_rad, n > 2000 ? 1 : 0, &nl)) return -1;
    const int Dm = or_dim(P->n_ch);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        or_atom A;
        atom_eval(P, i, nl.idx + nl.off[i], nl.off[i + 1] - nl.off[i], pos, spin, species, box, per, 0,
                  &A, NULL, NULL, NULL);
        memcpy(q_out + i * Dm, A.q, sizeof(double) * (size_t)Dm);
    }
    free_nlist(&nl);
    return 0;
}

/* Energy, per-atom network energies, forces, fields and virial of the whole system.
 * Any of Ei, F, H, W may be NULL. */
int or_evaluate(int64_t n, const double *pos, const double *spin, const int32_t *species,
                const double *box, const int32_t *per, const or_params *P, const double B[3],
                double *E_out, double *Ei, double *F, double *H, double *W) {
    if (check_params(P)) return -3;
    or_nlist nl;
    if (build_nlist(n, pos, box, per, P->rc_rad, n > 2000 ? 1 : 0, &nl)) return -1;
    const int64_t npair = nl.off[n];
    double *D = malloc(sizeof(double) * 3 * (size_t)(npair > 0 ? npair : 1));
    double *G = malloc(sizeof(double) * 3 * (size_t)(npair > 0 ? npair : 1));
    double *Gs = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *Ea = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!D || !G || !Gs || !Ea) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        or_atom A;
        int64_t o = nl.off[i];
        atom_eval(P, i, nl.idx + o, nl.off[i + 1] - o, pos, spin, species, box, per, 1, &A, D + 3 * o,
                  G + 3 * o, Gs + 3 * i);
        Ea[i] = A.E;
    }
    /* assembly: F_i += D_ij, F_j -= D_ij; H_j -= G_ij; H_i -= G_ii; W -= r_ij (x) D_ij */
    double Wl[9] = {0};
    double Etot = 0.0;
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    if (H) memset(H, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        Etot += Ea[i];
        double zee = P->moment_muB[species[i]] * OR_MUB, Bi[3];
        field_at(P, B, i, Bi);
        Etot -= zee * (Bi[0] * spin[3 * i] + Bi[1] * spin[3 * i + 1] + Bi[2] * spin[3 * i + 2]);
        double hl[3];
        Etot += landau_at(P, species[i], spin + 3 * i, hl);
        if (H)
            for (int c = 0; c < 3; ++c) H[3 * i + c] += -Gs[3 * i + c] + zee * Bi[c] + hl[c];
        for (int64_t p = nl.off[i]; p < nl.off[i + 1]; ++p) {
            int64_t j = nl.idx[p];
            if (F)
                for (int c = 0; c < 3; ++c) { F[3 * i + c] += D[3 * p + c]; F[3 * j + c] -= D[3 * p + c]; }
            if (H)
                for (int c = 0; c < 3; ++c) H[3 * j + c] -= G[3 * p + c];
            if (W) {
                double d[3];
                sep(pos, i, j, box, per, d);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) Wl[3 * a + b] -= d[a] * D[3 * p + b];
            }
        }
    }
    if (E_out) *E_out = Etot;
    if (Ei) memcpy(Ei, Ea, sizeof(double) * (size_t)n);
    if (W) memcpy(W, Wl, sizeof(double) * 9);
    free(D); free(G); free(Gs); free(Ea);
    free_nlist(&nl);
    return 0;
}

/* Forces and fields of the atoms listed in sample[0..m) only: every centre whose
 * energy depends on a sampled atom (the sampled atom and its radial neighbours)
 * is evaluated, nothing else.  Ei_out (optional) gets the sampled atoms' E_i. */
int or_evaluate_subset(int64_t n, const double *pos, const double *spin, const int32_t *species,
                       const double *box, const int32_t *per, const or_params *P, const double B[3],
                       int64_t m, const int64_t *sample, double *F_out, double *H_out, double *Ei_out) {
    if (check_params(P)) return -3;
    or_nlist nl;
    if (build_nlist(n, pos, box, per, P->rc_rad, n > 2000 ? 1 : 0, &nl)) return -1;
    /* centres needed */
    char *need = calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *slot = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!need || !slot) return -1;
    for (int64_t s = 0; s < m; ++s) {
        int64_t k = sample[s];
        need[k] = 1;
        for (int64_t p = nl.off[k]; p < nl.off[k + 1]; ++p) need[nl.idx[p]] = 1;
    }
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) slot[i] = need[i] ? nc++ : -1;
    int64_t *centres = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t *poff = malloc(sizeof(int64_t) * (size_t)(nc + 1));
    for (int64_t i = 0; i < n; ++i) if (need[i]) centres[slot[i]] = i;
    poff[0] = 0;
    for (int64_t c = 0; c < nc; ++c) poff[c + 1] = poff[c] + (nl.off[centres[c] + 1] - nl.off[centres[c]]);
    double *D = malloc(sizeof(double) * 3 * (size_t)(poff[nc] > 0 ? poff[nc] : 1));
    double *G = malloc(sizeof(double) * 3 * (size_t)(poff[nc] > 0 ? poff[nc] : 1));
    double *Gs = malloc(sizeof(double) * 3 * (size_t)(nc > 0 ? nc : 1));
    double *Ea = malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c) {
        int64_t i = centres[c];
        or_atom A;
        atom_eval(P, i, nl.idx + nl.off[i], nl.off[i + 1] - nl.off[i], pos, spin, species, box, per, 1, &A,
                  D + 3 * poff[c], G + 3 * poff[c], Gs + 3 * c);
        Ea[c] = A.E;
    }
    for (int64_t s = 0; s < m; ++s) {
        int64_t k = sample[s], ck = slot[k];
        double f[3] = {0, 0, 0}, h[3];
        double zee = P->moment_muB[species[k]] * OR_MUB, Bk[3];
        field_at(P, B, k, Bk);
        double hl[3];
        landau_at(P, species[k], spin + 3 * k, hl);
        for (int c = 0; c < 3; ++c) h[c] = -Gs[3 * ck + c] + zee * Bk[c] + hl[c];
        /* own pairs */
        for (int64_t p = nl.off[k], a = 0; p < nl.off[k + 1]; ++p, ++a)
            for (int c = 0; c < 3; ++c) f[c] += D[3 * (poff[ck] + a) + c];
        /* pairs (j -> k) of each neighbour j */
        for (int64_t p = nl.off[k]; p < nl.off[k + 1]; ++p) {
            int64_t j = nl.idx[p], cj = slot[j];
            for (int64_t q = nl.off[j], a = 0; q < nl.off[j + 1]; ++q, ++a) {
                if (nl.idx[q] != k) continue;
                for (int c = 0; c < 3; ++c) {
                    f[c] -= D[3 * (poff[cj] + a) + c];
                    h[c] -= G[3 * (poff[cj] + a) + c];
                }
            }
        }
        for (int c = 0; c < 3; ++c) { F_out[3 * s + c] = f[c]; H_out[3 * s + c] = h[c]; }
        if (Ei_out) Ei_out[s] = Ea[ck];
    }
    free(need); free(slot); free(centres); free(poff); free(D); free(G); free(Gs); free(Ea);
    free_nlist(&nl);
    return 0;
}

/* ----------------------------------------------------------- integrator */
/* Precession vector of the damped spin equation dS/dt = omega x S with
 * omega = (H' + lambda S x H') / ((1 + lambda^2) hbar), H' = H + eta. */
static void omega_of(const double S[3], const double Hp[3], double lam, double w[3]) {
    double sxh[3] = {S[1] * Hp[2] - S[2] * Hp[1], S[2] * Hp[0] - S[0] * Hp[2], S[0] * Hp[1] - S[1] * Hp[0]};
    double k = 1.0 / ((1.0 + lam * lam) * OR_HBAR);
    for (int c = 0; c < 3; ++c) w[c] = (Hp[c] + lam * sxh[c]) * k;
}

/* Exact rotation of S by angle |w| dt about w/|w| (Rodrigues). */
void or_rotate(const double S[3], const double w[3], double dt, double out[3]) {
    double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (wn == 0.0) { out[0] = S[0]; out[1] = S[1]; out[2] = S[2]; return; }
    double a[3] = {w[0] / wn, w[1] / wn, w[2] / wn};
    double th = wn * dt, c = cos(th), s = sin(th);
    double axs[3] = {a[1] * S[2] - a[2] * S[1], a[2] * S[0] - a[0] * S[2], a[0] * S[1] - a[1] * S[0]};
    double as = a[0] * S[0] + a[1] * S[1] + a[2] * S[2];
    for (int k = 0; k < 3; ++k) out[k] = S[k] * c + axs[k] * s + a[k] * as * (1.0 - c);
}

/* Largest Anderson history the oracle accepts. */
#define OR_AA_MAX 8

/* Solve the k x k symmetric positive definite system A g = b in place (Cholesky). */
static int spd_solve(int k, double *A, double *b) {
    for (int j = 0; j < k; ++j) {
        double d = A[j * k + j];
        for (int q = 0; q < j; ++q) d -= A[j * k + q] * A[j * k + q];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        A[j * k + j] = d;
        for (int i = j + 1; i < k; ++i) {
            double v = A[i * k + j];
            for (int q = 0; q < j; ++q) v -= A[i * k + q] * A[j * k + q];
            A[i * k + j] = v / d;
        }
    }
    for (int i = 0; i < k; ++i) {   /* L y = b */
        double v = b[i];
        for (int q = 0; q < i; ++q) v -= A[i * k + q] * b[q];
        b[i] = v / A[i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {   /* L^T g = y */
        double v = b[i];
        for (int q = i + 1; q < k; ++q) v -= A[q * k + i] * b[q];
        b[i] = v / A[i * k + i];
    }
    return 0;
}

static void normalise3(double *v) {
    double nn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= nn; v[1] /= nn; v[2] /= nn;
}

/* The midpoint iteration of one step (see or_run).  On entry spin holds the explicit
 * predictor X_0, S0 the spins at the start of the step and pmid the lattice midpoint;
 * on return spin holds the new spins and (Fs, Hs) the forces and fields at (pos, spin). */
static int midpoint_spins(int64_t n, const double *pos, const double *pmid, double *spin, const int32_t *species, const double *box,
                          const int32_t *per, const or_params *P, const or_dynamics *dyn, double dt,
                          const double B[3], const double *S0, const double *eta, double *Fs, double *Hs,
                          int64_t *iters) {
    const size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
    const int depth = dyn->anderson_depth;
    const double lam = dyn->lambda_spin;
    double *X = malloc(sizeof(double) * n3), *G = malloc(sizeof(double) * n3), *Mid = malloc(sizeof(double) * n3);
    double *Xh = malloc(sizeof(double) * n3 * (size_t)(depth + 1));   /* history of X_j (ring) */
    double *Gh = malloc(sizeof(double) * n3 * (size_t)(depth + 1));   /* history of G_j (ring) */
    int rc = 0;
    if (!X || !G || !Mid || !Xh || !Gh) { rc = -1; goto out; }
    memcpy(X, spin, sizeof(double) * 3 * (size_t)n);
    for (int m = 0; m < dyn->midpoint_iters; ++m) {
        for (int64_t i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) Mid[3 * i + c] = S0[3 * i + c] + X[3 * i + c];
            normalise3(Mid + 3 * i);
        }
        rc = or_evaluate(n, pmid, Mid, species, box, per, P, B, NULL, NULL, Fs, Hs, NULL);
        if (rc) goto out;
        *iters += 1;
        double dmax = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double Hp[3], w[3], d2 = 0.0;
            for (int c = 0; c < 3; ++c) Hp[c] = Hs[3 * i + c] + eta[3 * i + c];
            omega_of(Mid + 3 * i, Hp, lam, w);
            or_rotate(S0 + 3 * i, w, dt, G + 3 * i);
            for (int c = 0; c < 3; ++c) d2 += (G[3 * i + c] - X[3 * i + c]) * (G[3 * i + c] - X[3 * i + c]);
            if (sqrt(d2) > dmax) dmax = sqrt(d2);
        }
        if (dmax < dyn->midpoint_tol || m + 1 == dyn->midpoint_iters) break;
        if (depth == 0) {
            memcpy(X, G, sizeof(double) * 3 * (size_t)n);
            continue;
        }
        /* Anderson mix over the last k + 1 iterates */
        const int slot = m % (depth + 1);
        memcpy(Xh + (size_t)slot * n3, X, sizeof(double) * 3 * (size_t)n);
        memcpy(Gh + (size_t)slot * n3, G, sizeof(double) * 3 * (size_t)n);
        const int k = m < depth ? m : depth;
        if (k == 0) {
            memcpy(X, G, sizeof(double) * 3 * (size_t)n);
            continue;
        }
        double A[OR_AA_MAX * OR_AA_MAX], b[OR_AA_MAX];
        /* column q: dF_q = f_{m-k+q+1} - f_{m-k+q}, f_j = G_j - X_j */
        for (int q = 0; q < k; ++q) {
            b[q] = 0.0;
            for (int r = 0; r < k; ++r) A[q * k + r] = 0.0;
        }
        for (size_t e = 0; e < 3 * (size_t)n; ++e) {
            double fm = G[e] - X[e];
            double dF[OR_AA_MAX];
            for (int q = 0; q < k; ++q) {
                const int ja = (m - k + q + 1) % (depth + 1), jb = (m - k + q) % (depth + 1);
                const double fa = Gh[(size_t)ja * n3 + e] - Xh[(size_t)ja * n3 + e];
                const double fb = Gh[(size_t)jb * n3 + e] - Xh[(size_t)jb * n3 + e];
                dF[q] = fa - fb;
            }
            for (int q = 0; q < k; ++q) {
                b[q] += dF[q] * fm;
                for (int r = 0; r < k; ++r) A[q * k + r] += dF[q] * dF[r];
            }
        }
        double tr = 0.0;
        for (int q = 0; q < k; ++q) tr += A[q * k + q];
        const double delta = dyn->anderson_reg * tr / k;
        for (int q = 0; q < k; ++q) A[q * k + q] += delta;
        if (!(tr > 0.0) || spd_solve(k, A, b)) {   /* no usable history: plain step */
            memcpy(X, G, sizeof(double) * 3 * (size_t)n);
            continue;
        }
        for (size_t e = 0; e < 3 * (size_t)n; ++e) {
            double v = G[e];
            for (int q = 0; q < k; ++q) {
                const int ja = (m - k + q + 1) % (depth + 1), jb = (m - k + q) % (depth + 1);
                v -= b[q] * (Gh[(size_t)ja * n3 + e] - Gh[(size_t)jb * n3 + e]);
            }
            X[e] = v;
        }
        for (int64_t i = 0; i < n; ++i) normalise3(X + 3 * i);
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) spin[3 * i + c] = G[3 * i + c];
        normalise3(spin + 3 * i);
    }
    rc = or_evaluate(n, pos, spin, species, box, per, P, B, NULL, NULL, Fs, Hs, NULL);
out:
    free(X); free(G); free(Mid); free(Xh); free(Gh);
    return rc;
}

/* Colouring for the coloured spin sweep: atoms i and j conflict when their minimum-image
 * distance is below 2 rc (d^2 < (2 rc)^2, the neighbour-list arithmetic), since the field on a
 * spin depends on every spin within 2 rc through the neighbours' descriptors.  Greedy in
 * index order: colour(i) = the smallest c >= 0 used by no conflicting j < i.  Returns the
 * number of colours (>= 1 when n > 0), or a negative code. */
int or_colour(int64_t n, const double *pos, const double *box, const int32_t *per, double rc,
              int32_t *colour) {
    if (n == 0) return 0;
    or_nlist nl;
    if (build_nlist(n, pos, box, per, 2.0 * rc, n > 2000 ? 1 : 0, &nl)) return -1;
    int64_t cap = 64;
    unsigned char *used = (unsigned char *)calloc((size_t)cap, 1);
    if (!used) return -1;
    int32_t ncol = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = nl.off[i]; p < nl.off[i + 1]; ++p) {
            int32_t j = nl.idx[p];
            if (j < i) {
                if (colour[j] >= cap) {
                    int64_t nc2 = 2 * (int64_t)colour[j] + 2;
                    unsigned char *u2 = (unsigned char *)realloc(used, (size_t)nc2);
                    if (!u2) { free(used); free_nlist(&nl); return -1; }
                    memset(u2 + cap, 0, (size_t)(nc2 - cap));
                    used = u2;
                    cap = nc2;
                }
                used[colour[j]] = 1;
            }
        }
        int32_t c = 0;
        while (c < cap && used[c]) ++c;
        colour[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
        for (int64_t p = nl.off[i]; p < nl.off[i + 1]; ++p) {
            int32_t j = nl.idx[p];
            if (j < i) used[colour[j]] = 0;
        }
    }
    free(used);
    free_nlist(&nl);
    return ncol;
}

/* Advance (pos, vel, spin) by n_steps steps of dt (fs) at temperature T (K) and
 * field B (T).  F and H carry the forces and fields of the current state between
 * calls (have_fh = 0: they are evaluated first).  One step, from (r, v, S, F, H):
 *   v += dt/2 F/m;  r += dt/2 v;  v = c v + sqrt((1-c^2) kT/m) xi  (c = exp(-gamma dt));
 *   r += dt/2 v (wrapped);  eta = sqrt(2 lambda kT hbar/dt) zeta;
 *   Sstar = Rot(S, omega(S, H+eta) dt);  (Fstar, Hstar) at (r, Sstar);
 *   S <- Rot(S, (omega(S, H+eta) + omega(Sstar, Hstar+eta)) dt/2), renormalised;
 *   v += dt/2 Fstar/m;  (F, H) <- (Fstar, Hstar).
 * xi is Philox stream 1, zeta stream 2, counter (step, atom, stream, 0), key (seed, replica).
 *
 * Self-consistent midpoint spin update (Section 5.1.3; dyn->midpoint_iters > 0).  The
 * lattice part is unchanged; r_mid = r_start + (r - r_start)/2 is the lattice midpoint
 * of the step (unwrapped displacement, then wrapped).  With X_0 = Rot(S, omega(S, H+eta) dt)
 * the explicit predictor, iteration m (m < midpoint_iters) takes
 *   M_m = (S + X_m) / |S + X_m|            the midpoint spins,
 *   H_m = H(r_mid, M_m)                    force and field re-evaluated at the midpoint
 *                                          configuration (r_mid, M_m),
 *   G_m = Rot(S, omega(M_m, H_m+eta) dt)   the one-step update re-applied,
 * and stops when d_m = max_i |G_m,i - X_m,i| < midpoint_tol or at the cap; then
 * S <- G_m renormalised, (F, H) are evaluated at (r, S) and v += dt/2 F/m.  The next
 * iterate is X_{m+1} = G_m (plain fixed-point iteration) or, with anderson_depth > 0,
 * the regularised Anderson mix (Anderson 1965; Walker and Ni 2011, undamped form):
 *   f_j = G_j - X_j;  dF, dG = differences of the last k+1 f_j, G_j (k = min(depth, m));
 *   (dF^T dF + delta I) g = dF^T f_m,  delta = anderson_reg * trace(dF^T dF) / k;
 *   X_{m+1} = G_m - dG g, each spin renormalised.
 * *iters_used (if not NULL) receives the number of midpoint evaluations over all steps.
 *
 * Longitudinal mode (dyn->longitudinal = 1; the moment length |S_i| is free, Section 3).
 * The spin equation is the Langevin form with longitudinal fluctuations of Ma and
 * Dudarev (Phys. Rev. B 86, 054416, 2012), in this file's precession convention:
 *   dS/dt = (H/hbar) x S + (alpha/hbar) H + xi,  <xi_a(t) xi_b(t')> = 2 alpha kT/hbar delta_ab delta(t-t'),
 * whose stationary density is exp(-E/kT) over R^3.  The step keeps the lattice part and
 * the predictor-corrector structure (Heun on the spin equation, the same noise in both):
 *   Sstar = Rot(S, H dt/hbar) + alpha dt/hbar H + sqrt(2 alpha kT dt/hbar) zeta;
 *   S <- Rot(S, (H + Hstar) dt/(2 hbar)) + alpha dt/hbar (H + Hstar)/2 + sqrt(2 alpha kT dt/hbar) zeta,
 * with no renormalisation; lambda_spin is not used.  Not combined with the midpoint mode.
 *
 * Coloured Suzuki-Trotter spin sweep (dyn->st_sweep = 1; a splitting of the spin update
 * into colour classes of mutually independent spins).  The lattice part is unchanged; at
 * the new positions r the atoms are coloured (or_colour, conflict radius 2 rc_rad) and the
 * spins are advanced by a symmetric sweep over the C colours, c = 0..C-1 then C-1..0: each
 * sub-step evaluates H at (r, S) and rotates every spin of colour c by half a step,
 *   S_i <- Rot(S_i, omega(S_i, H_i + eta_i) dt/2), renormalised,
 * with the step's eta as in the predictor-corrector; then (F, H) at (r, S) and v += dt/2 F/m.
 * 2C + 1 evaluations per step.  Not combined with the midpoint or the longitudinal mode. */
int or_run(int64_t n, double *pos, double *vel, double *spin, const int32_t *species, const double *box,
           const int32_t *per, const or_params *P, const or_dynamics *dyn, int64_t n_steps, double dt,
           double T, const double B[3], uint64_t step0, double *F, double *H, int have_fh,
           int64_t *iters_used) {
    if (check_params(P)) return -3;
    if (dyn->midpoint_iters < 0 || dyn->anderson_depth < 0 || dyn->anderson_depth > OR_AA_MAX ||
        !(dyn->midpoint_tol >= 0.0) || !(dyn->anderson_reg >= 0.0))
        return -3;
    const int lng = dyn->longitudinal != 0;
    if (lng && (dyn->midpoint_iters > 0 || !(dyn->alpha_long >= 0.0))) return -3;
    const int sts = dyn->st_sweep != 0;
    if (sts && (dyn->midpoint_iters > 0 || lng)) return -3;
    int32_t *colour = NULL;
    if (sts && !(colour = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1)))) return -1;
    if (iters_used) *iters_used = 0;
    int rc;
    if (!have_fh) {
        rc = or_evaluate(n, pos, spin, species, box, per, P, B, NULL, NULL, F, H, NULL);
        if (rc) return rc;
    }
    double *S0 = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *eta = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *Fs = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *Hs = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *pmid = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!S0 || !eta || !Fs || !Hs || !pmid) return -1;
    const double cfric = exp(-dyn->gamma_lattice * dt);
    const double lam = lng ? 0.0 : dyn->lambda_spin;
    const double sig_eta = lng ? ((T > 0.0 && dyn->alpha_long > 0.0) ? sqrt(2.0 * dyn->alpha_long * OR_KB * T * dt / OR_HBAR) : 0.0)
                               : ((T > 0.0 && lam > 0.0) ? sqrt(2.0 * lam * OR_KB * T * OR_HBAR / dt) : 0.0);
    const double kdrift = lng ? dyn->alpha_long * dt / OR_HBAR : 0.0;   /* longitudinal drift per unit field */
    for (int64_t s = 0; s < n_steps; ++s) {
        uint64_t step = step0 + (uint64_t)s;
        for (int64_t i = 0; i < n; ++i) {
            double m = P->mass_amu[species[i]];
            double sig_v = sqrt((1.0 - cfric * cfric) * OR_KB * T * OR_ACC / m);
            double xi[4], ze[4];
            or_gauss4(step, (uint64_t)i, 1, dyn->seed, dyn->replica, xi);
            or_gauss4(step, (uint64_t)i, 2, dyn->seed, dyn->replica, ze);
            for (int c = 0; c < 3; ++c) {
                double *x = pos + 3 * i + c, *v = vel + 3 * i + c;
                const double x0 = *x;
                *v += 0.5 * dt * F[3 * i + c] * OR_ACC / m;
                *x += 0.5 * dt * *v;
                *v = cfric * *v + sig_v * xi[c];
                *x += 0.5 * dt * *v;
                double xm = x0 + 0.5 * (*x - x0);     /* lattice midpoint of the step */
                if (per[c]) {
                    *x = *x - box[c] * floor(*x / box[c]);
                    xm = xm - box[c] * floor(xm / box[c]);
                }
                pmid[3 * i + c] = xm;
                eta[3 * i + c] = sig_eta * ze[c];
            }
            double Hp[3], w[3];
            if (sts) {   /* the spins wait for the colour sweep at the new positions */
                for (int c = 0; c < 3; ++c) S0[3 * i + c] = spin[3 * i + c];
                continue;
            }
            if (lng) {   /* eta is the additive noise displacement here */
                for (int c = 0; c < 3; ++c) S0[3 * i + c] = spin[3 * i + c];
                omega_of(S0 + 3 * i, H + 3 * i, 0.0, w);
                or_rotate(S0 + 3 * i, w, dt, spin + 3 * i);
                for (int c = 0; c < 3; ++c) spin[3 * i + c] += kdrift * H[3 * i + c] + eta[3 * i + c];
                continue;
            }
            for (int c = 0; c < 3; ++c) { S0[3 * i + c] = spin[3 * i + c]; Hp[c] = H[3 * i + c] + eta[3 * i + c]; }
            omega_of(S0 + 3 * i, Hp, lam, w);
            or_rotate(S0 + 3 * i, w, dt, spin + 3 * i);
        }
        if (dyn->midpoint_iters > 0) {
            int64_t it = 0;
            rc = midpoint_spins(n, pos, pmid, spin, species, box, per, P, dyn, dt, B, S0, eta, Fs, Hs, &it);
            if (iters_used) *iters_used += it;
            if (rc) break;
            for (int64_t i = 0; i < n; ++i) {
                double m = P->mass_amu[species[i]];
                for (int c = 0; c < 3; ++c) {
                    vel[3 * i + c] += 0.5 * dt * Fs[3 * i + c] * OR_ACC / m;
                    F[3 * i + c] = Fs[3 * i + c];
                    H[3 * i + c] = Hs[3 * i + c];
                }
            }
            continue;
        }
        if (sts) {
            const int ncol = or_colour(n, pos, box, per, P->rc_rad, colour);
            if (ncol < 0) { rc = -1; break; }
            for (int pass = 0; pass < 2 * ncol && !rc; ++pass) {
                const int32_t c = pass < ncol ? pass : 2 * ncol - 1 - pass;
                rc = or_evaluate(n, pos, spin, species, box, per, P, B, NULL, NULL, Fs, Hs, NULL);
                for (int64_t i = 0; i < n && !rc; ++i) {
                    if (colour[i] != c) continue;
                    double Hp[3], w[3], Sn[3];
                    for (int q = 0; q < 3; ++q) Hp[q] = Hs[3 * i + q] + eta[3 * i + q];
                    omega_of(spin + 3 * i, Hp, lam, w);
                    or_rotate(spin + 3 * i, w, 0.5 * dt, Sn);
                    normalise3(Sn);
                    for (int q = 0; q < 3; ++q) spin[3 * i + q] = Sn[q];
                }
            }
            if (rc) break;
            rc = or_evaluate(n, pos, spin, species, box, per, P, B, NULL, NULL, Fs, Hs, NULL);
            if (rc) break;
            for (int64_t i = 0; i < n; ++i) {
                double m = P->mass_amu[species[i]];
                for (int q = 0; q < 3; ++q) {
                    vel[3 * i + q] += 0.5 * dt * Fs[3 * i + q] * OR_ACC / m;
                    F[3 * i + q] = Fs[3 * i + q];
                    H[3 * i + q] = Hs[3 * i + q];
                }
            }
            continue;
        }
        rc = or_evaluate(n, pos, spin, species, box, per, P, B, NULL, NULL, Fs, Hs, NULL);
        if (rc) break;
        for (int64_t i = 0; i < n; ++i) {
            double m = P->mass_amu[species[i]];
            double Hp0[3], Hp1[3], w0[3], w1[3], w[3], Snew[3];
            if (lng) {
                double Hb[3];
                for (int c = 0; c < 3; ++c) Hb[c] = 0.5 * (H[3 * i + c] + Hs[3 * i + c]);
                omega_of(S0 + 3 * i, Hb, 0.0, w);
                or_rotate(S0 + 3 * i, w, dt, Snew);
                for (int c = 0; c < 3; ++c) {
                    spin[3 * i + c] = Snew[c] + kdrift * Hb[c] + eta[3 * i + c];
                    vel[3 * i + c] += 0.5 * dt * Fs[3 * i + c] * OR_ACC / m;
                    F[3 * i + c] = Fs[3 * i + c];
                    H[3 * i + c] = Hs[3 * i + c];
                }
                continue;
            }
            for (int c = 0; c < 3; ++c) {
                Hp0[c] = H[3 * i + c] + eta[3 * i + c];
                Hp1[c] = Hs[3 * i + c] + eta[3 * i + c];
            }
            omega_of(S0 + 3 * i, Hp0, lam, w0);
            omega_of(spin + 3 * i, Hp1, lam, w1);
            for (int c = 0; c < 3; ++c) w[c] = 0.5 * (w0[c] + w1[c]);
            or_rotate(S0 + 3 * i, w, dt, Snew);
            double nn = sqrt(Snew[0] * Snew[0] + Snew[1] * Snew[1] + Snew[2] * Snew[2]);
            for (int c = 0; c < 3; ++c) {
                spin[3 * i + c] = Snew[c] / nn;
                vel[3 * i + c] += 0.5 * dt * Fs[3 * i + c] * OR_ACC / m;
                F[3 * i + c] = Fs[3 * i + c];
                H[3 * i + c] = Hs[3 * i + c];
            }
        }
    }
    free(S0); free(eta); free(Fs); free(Hs); free(pmid); free(colour);
    return rc;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads used by the following calls (for timing the oracle on one core). */
void or_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
