// sl_eval2.cu -- NEP-SPIN evaluation: compacted radial kernels and quad-per-atom angular kernels.
//
// Same mathematics as the descriptor of arXiv 2606.14073 (Sections 5.1.1-5.1.2, 5.2.3-5.2.4)
// described in sl_nep.cu; this file maps it onto the GPU differently:
//
//   k_crad     one thread per atom, one pass over the candidate list (which carries a
//              skin): compacts the pairs inside the cutoffs into angular rows
//              (r < rc_ang) and radial-only rows (rc_ang <= r < rc_rad), each grouped by
//              neighbour species, and accumulates the radial and pairwise-magnetic basis
//              sums over them, contracted with the coefficients once per neighbour
//              species (q^R, q^EX, q^DMI, q^ANI, q^SIA, q^O).
//   k_ang_fwd  four lanes per atom.  Each lane stages one angular pair (carrier, g_n,
//              spin weight, the 24 solid harmonics) in shared memory; then every lane
//              accumulates B_nlm, BS_nlm for its 6 harmonics over the staged pairs.
//   k_bwd      four lanes per atom, lanes over pairs.  The angular adjoints
//              dE/dB_nlm = 2 kappa_lm Fp B_nlm and the precontracted radial
//              coefficients of the atom sit in shared memory; each lane takes whole
//              pairs (angular rows first, then radial-only rows) and writes the pair
//              record (dE_i/dr_ij, dE_i/dS_j) straight into the slot the neighbour j
//              will read (its own list slot of i); the per-atom sums (dE_i/dr_i side,
//              dE_i/dS_i, virial) are reduced over the quad.
// The force/field gather (sl_integrate.cu) then reads, for atom k, the records of
// its in-cutoff slots only.
#include <cstddef>
#include <mutex>

#include "sl_internal.h"
#include "sl_eval2.cuh"
#include "sl_batch.h"
#include "sl_fused.cuh"

namespace sl {

// ------------------------------------------------------------------ helpers
// Two independent multiply-adds per instruction where the hardware has them (FP32 pairs:
// the packed FMA of sm_100 and later; each component rounds like fmaf), plain FMAs in FP64.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <typename R>
__device__ __forceinline__ v2<R> pair2(R x, R y) {
    v2<R> v;
    v.x = x;
    v.y = y;
    return v;
}
// g_n = sum_k c_nk f_k and dg_n = sum_k c_nk df_k together, two multiply-adds per instruction
// The carrier of sl_common.cuh with the T_k and U_k recurrences advanced together.
template <typename R>
__device__ __forceinline__ void carrier_fd2(R r, R inv_rc, R f[NK], R df[NK]) {
    const R t = r * inv_rc;
    R fch, dfch;
    cut_half_d(t, inv_rc, fch, dfch);
    const R y = t - R(1);
    const R x = R(2) * y * y - R(1);
    const R dxr = R(4) * y * inv_rc;
    const R x2 = R(2) * x;
    const R dxf = dxr * fch;
    v2<R> tum = pair2<R>(R(1), R(1)), tuc = pair2<R>(x, x2);   // (T_0, U_0), (T_1, U_1)
    f[0] = R(2) * fch;
    df[0] = R(2) * dfch;
    f[1] = fma_(x, fch, fch);
    df[1] = dxf + fma_(x, dfch, dfch);
#pragma unroll
    for (int k = 2; k < NK; ++k) {
        const v2<R> tun = fma2(pair2<R>(x2, x2), tuc, pair2<R>(-tum.x, -tum.y));
        f[k] = fma_(tun.x, fch, fch);
        df[k] = fma_(R(k) * tuc.y, dxf, fma_(tun.x, dfch, dfch));
        tum = tuc;
        tuc = tun;
    }
}

template <typename R, int TI, int TJ, int G>
__device__ __forceinline__ void contract_k2(const NepDev<R> &P, const R f[NK], const R df[NK], R g[NCH], R dg[NCH]) {
#pragma unroll
    for (int n = 0; n < NCH; ++n) {
        v2<R> s = pair2<R>(R(0), R(0));
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const R c = P.c[TI][TJ][G][n][k];
            s = fma2(pair2<R>(c, c), pair2<R>(f[k], df[k]), s);
        }
        g[n] = s.x;
        dg[n] = s.y;
    }
}

template <typename R, int TI, int TJ, int G>
__device__ __forceinline__ void contract_k(const NepDev<R> &P, const R f[NK], R g[NCH]) {
#pragma unroll
    for (int n = 0; n < NCH; ++n) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < NK; ++k) s += P.c[TI][TJ][G][n][k] * f[k];
        g[n] = s;
    }
}

template <typename R>
__device__ __forceinline__ void sep(const BoxDev<R> &b, const v4<R> &pi, const v4<R> &pj, R &dx, R &dy, R &dz) {
    dx = pj.x - pi.x;
    dy = pj.y - pi.y;
    dz = pj.z - pi.z;
    minimg(b, dx, dy, dz);
}

// per-lane constants of harmonic lm = ql + 4 m (ql = lane in quad)
__device__ __forceinline__ int lm_of(int ql, int m) { return ql + 4 * m; }
__device__ __forceinline__ int l_of_lm(int lm) { return lm < 3 ? 1 : lm < 8 ? 2 : lm < 15 ? 3 : 4; }
template <typename R>
__device__ __forceinline__ R kappa_of_lm(int lm) {
    // kappa_lm of the addition theorem, selected at run time (the quad lane picks its harmonics)
    switch (lm) {
    case 0: case 1: case 2: return R(1.0);
    case 3: case 4: case 5: return R(3.0);
    case 6: return R(0.75);
    case 7: return R(0.25);
    case 8: return R(0.625);
    case 9: return R(15.0);
    case 10: return R(0.375);
    case 11: return R(0.25);
    case 12: return R(0.375);
    case 13: return R(3.75);
    case 14: return R(0.625);
    case 15: return R(8.75);
    case 16: return R(4.375);
    case 17: return R(1.25);
    case 18: return R(0.625);
    case 19: return R(0.015625);
    case 20: return R(0.625);
    case 21: return R(0.3125);
    case 22: return R(4.375);
    default: return R(0.546875);
    }
}

// ------------------------------------------------------------------ k_crad
// One thread per atom, per neighbour species:
//  A. the angular candidates (within rc_ang + skin of the list build, so nearly all inside
//     rc_rad): compaction and the radial and pairwise-magnetic basis sums in one pass;
//  B. the radial-shell candidates (rc_ang + skin .. rc_rad + skin at the build, fewer than
//     half inside rc_rad): compaction only, a few instructions per candidate;
//  C. the basis sums over the rows B produced.
// Splitting B from C keeps a warp from running the pair arithmetic for every candidate of
// the shell whenever one of its 32 atoms has that candidate inside the cutoff.  Rows are
// angular (r < rc_ang) or radial-only (rc_ang <= r < rc_rad), each grouped by neighbour
// species in candidate order (species 0 from candidate segments 0 and 2, then species 1
// from 1 and 3), for the angular and backward kernels and the gather.  The sums are
// contracted with the coefficients once per neighbour species (q^R, q^EX, q^DMI, q^ANI,
// q^SIA); q^O = |S|^2.

template <typename R>
struct RadSums {
    R b0[NK];
    v2<R> b12[NK], b34[NK];   // (EX, DMI) and (ANI, SIA) sums, two per packed multiply-add
};

template <typename R>
__device__ __forceinline__ void rad_accumulate(const NepDev<R> &P, const v4<R> &si, const v4<R> &cs, R dx, R dy,
                                               R dz, R d2, RadSums<R> &b) {
    const R ir = rsqrt_(d2), r = d2 * ir;
    const R ux = dx * ir, uy = dy * ir, uz = dz * ir;
    R f[NK];
    carrier_f(r, P.inv_rc_r, f);
    const R sij = si.x * cs.x + si.y * cs.y + si.z * cs.z;
    const R siu = si.x * ux + si.y * uy + si.z * uz;
    const R sju = cs.x * ux + cs.y * uy + cs.z * uz;
    const R dmi = (si.y * cs.z - si.z * cs.y) * ux + (si.z * cs.x - si.x * cs.z) * uy + (si.x * cs.y - si.y * cs.x) * uz;
    const R ani = siu * sju, sia = siu * siu;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        b.b0[k] += f[k];
        b.b12[k] = fma2(pair2<R>(f[k], f[k]), pair2<R>(sij, dmi), b.b12[k]);
        b.b34[k] = fma2(pair2<R>(f[k], f[k]), pair2<R>(ani, sia), b.b34[k]);
    }
}

// Row of an in-cutoff pair, or -1 (angular rows full: only after a list overflow, which ovf
// records; the atom reports it once its rows are written).
template <typename R>
__device__ __forceinline__ int take_row(const NepDev<R> &P, const Eval2Args<R> &a, R d2, int &na, int &nr,
                                        bool &ovf) {
    if (d2 < P.rc_a2) {
        if (na >= a.cap_ang) {
            ovf = true;
            return -1;
        }
        return na++;
    }
    return a.cap_ang + nr++;
}

// in-cutoff slot bits of this thread's atom, in shared memory (column threadIdx.x)
constexpr int MASKW_MAX = 8;
__device__ __forceinline__ void mark_slot(uint32_t (*sm)[128], int slot) {
    sm[slot >> 5][threadIdx.x] |= 1u << (slot & 31);
}

template <typename R, int TI, int TJ>
__device__ __forceinline__ void crad_species(const NepDev<R> &P, const Eval2Args<R> &a, int64_t i, const v4<R> &pi,
                                             const v4<R> &si, int lo0, int hi0, int lo1, int hi1, int &na, int &nr,
                                             bool &ovf, uint32_t (*smask)[128]) {
    RadSums<R> b;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        b.b0[k] = R(0);
        b.b12[k] = b.b34[k] = pair2<R>(R(0), R(0));
    }
    const int64_t N = a.n;
    // this atom's candidate list and reverse slots: one row each, read in aligned chunks of 4
    // entries (a 16-byte and a 4-byte load), two chunks ahead of the one being tested
    const int32_t *__restrict__ nrow = a.nbr + i * a.capr;
    const uint8_t *__restrict__ rrow = a.rev + i * a.capr;
    const v4<R> *__restrict__ pos = a.pos;
    const v4<R> *__restrict__ spin = a.spin;
    auto chunk = [&](int c, int hi, int4 &jq, uchar4 &tq) {
        if (c < hi) {
            jq = *reinterpret_cast<const int4 *>(nrow + c);
            tq = *reinterpret_cast<const uchar4 *>(rrow + c);
        }
    };

    // A: angular candidates, compaction and sums
    {
        int4 jq1 = make_int4(-1, -1, -1, -1), jq2 = jq1;
        uchar4 tq1 = make_uchar4(0, 0, 0, 0), tq2 = tq1;
        const int c0 = lo0 & ~3;
        chunk(c0, hi0, jq1, tq1);
        chunk(c0 + 4, hi0, jq2, tq2);
#pragma unroll 1
        for (int c = c0; c < hi0; c += 4) {
            int jj[4] = {jq1.x, jq1.y, jq1.z, jq1.w};
            const int tt[4] = {tq1.x, tq1.y, tq1.z, tq1.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c + u < lo0 || c + u >= hi0) jj[u] = -1;   // another segment's entry
            v4<R> pp[4], ss[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = jj[u] >= 0 ? jj[u] : (int)i;
                pp[u] = pos[j];
                ss[u] = spin[j];
            }
            jq1 = jq2;
            tq1 = tq2;
            chunk(c + 8, hi0, jq2, tq2);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (jj[u] < 0) continue;
                R dx, dy, dz;
                sep(a.box, pi, pp[u], dx, dy, dz);
                const R d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 < P.rc_r2)) continue;
                const int row = take_row(P, a, d2, na, nr, ovf);
                if (row < 0) continue;
                stg(a.clj + (int64_t)row * N + i, jj[u]);
                stg(a.cls + (int64_t)row * N + i, (uint16_t)((c + u) | (tt[u] << 8)));
                mark_slot(smask, c + u);
                rad_accumulate(P, si, ss[u], dx, dy, dz, d2, b);
            }
        }
    }
    // B: radial-shell candidates, compaction only
    const int naB = na, nrB = nr;
    {
        int4 jq1 = make_int4(-1, -1, -1, -1), jq2 = jq1;
        uchar4 tq1 = make_uchar4(0, 0, 0, 0), tq2 = tq1;
        const int c0 = lo1 & ~3;
        chunk(c0, hi1, jq1, tq1);
        chunk(c0 + 4, hi1, jq2, tq2);
#pragma unroll 1
        for (int c = c0; c < hi1; c += 4) {
            int jj[4] = {jq1.x, jq1.y, jq1.z, jq1.w};
            const int tt[4] = {tq1.x, tq1.y, tq1.z, tq1.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c + u < lo1 || c + u >= hi1) jj[u] = -1;
            v4<R> pp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) pp[u] = pos[jj[u] >= 0 ? jj[u] : (int)i];
            jq1 = jq2;
            tq1 = tq2;
            chunk(c + 8, hi1, jq2, tq2);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (jj[u] < 0) continue;
                R dx, dy, dz;
                sep(a.box, pi, pp[u], dx, dy, dz);
                const R d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 < P.rc_r2)) continue;
                const int row = take_row(P, a, d2, na, nr, ovf);
                if (row < 0) continue;
                stg(a.clj + (int64_t)row * N + i, jj[u]);
                stg(a.cls + (int64_t)row * N + i, (uint16_t)((c + u) | (tt[u] << 8)));
                mark_slot(smask, c + u);
            }
        }
    }
    // C: sums over the rows B wrote (angular rows naB..na, rare, then radial-only rows),
    // with the list entry two rows ahead and the coordinates of the next row in flight
    {
        const int nA = na - naB, len = nA + (nr - nrB);
        auto row_of = [&](int t) { return t < nA ? naB + t : a.cap_ang + nrB + (t - nA); };
        int j1 = 0, j2 = 0;
        v4<R> p1, s1;
        if (len > 0) j1 = a.clj[(int64_t)row_of(0) * N + i];
        if (len > 1) j2 = a.clj[(int64_t)row_of(1) * N + i];
        if (len > 0) { p1 = pos[j1]; s1 = spin[j1]; }
#pragma unroll 1
        for (int t = 0; t < len; ++t) {
            const v4<R> pj = p1, sj = s1;
            if (t + 1 < len) { p1 = pos[j2]; s1 = spin[j2]; }
            if (t + 2 < len) j2 = a.clj[(int64_t)row_of(t + 2) * N + i];
            R dx, dy, dz;
            sep(a.box, pi, pj, dx, dy, dz);
            rad_accumulate(P, si, sj, dx, dy, dz, dx * dx + dy * dy + dz * dz, b);
        }
    }
    // contraction of this species' sums; the second species adds onto the first's
    // values in q (the same thread wrote them), so no accumulator lives across the loops
    constexpr int GQ[5] = {Q_R, Q_EX, Q_DMI, Q_ANI, Q_SIA};
    constexpr int GG[5] = {G_R, G_EX, G_DMI, G_ANI, G_SIA};
#pragma unroll
    for (int g = 0; g < 5; ++g) {
#pragma unroll
        for (int n = 0; n < NCH; ++n) {
            R v = TJ == 0 ? R(0) : a.q[(GQ[g] + n) * a.qs + i];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const R bgk = g == 0 ? b.b0[k] : g == 1 ? b.b12[k].x : g == 2 ? b.b12[k].y : g == 3 ? b.b34[k].x
                                                                                                 : b.b34[k].y;
                v += P.c[TI][TJ][GG[g]][n][k] * bgk;
            }
            stg(a.q + (GQ[g] + n) * a.qs + i, v);
        }
    }
}

template <typename R, int TI>
__device__ __forceinline__ void crad_atom(const NepDev<R> &P, const Eval2Args<R> &a, int64_t i,
                                          uint32_t (*smask)[128]) {
    const int64_t N = a.n;
    const v4<R> pi = a.pos[i], si = a.spin[i];
    const int4 sg = a.seg[i];
    int na = 0, nr = 0;
    bool ovf = false;
    for (int w = 0; w < a.maskw; ++w) smask[w][threadIdx.x] = 0u;
    crad_species<R, TI, 0>(P, a, i, pi, si, 0, sg.x, sg.y, sg.z, na, nr, ovf, smask);
    const int na0 = na, nr0 = nr;
    crad_species<R, TI, 1>(P, a, i, pi, si, sg.x, sg.y, sg.z, sg.w, na, nr, ovf, smask);
    if (ovf) atomicOr(a.status, ST_NBR_OVERFLOW);
    stg(a.cnt + i, make_int4(na0, na, nr0, nr));
    for (int w = 0; w < a.maskw; ++w) stg(reinterpret_cast<int *>(a.mask) + (int64_t)w * N + i, (int)smask[w][threadIdx.x]);
    stg(a.q + Q_O * a.qs + i, si.x * si.x + si.y * si.y + si.z * si.z);
}

// MINB: minimum resident blocks per SM the register allocation is held to (the autotuner's
// register-budget dimension); the default is the first value of each kernel's list below.
template <typename R>
__device__ __forceinline__ void crad_body(const NepDev<R> &P, const Eval2Args<R> &args, int64_t blk,
                                          uint32_t (*smask)[128]) {
    // the arguments as values: read once from the block's copy, so nothing in the loops below
    // depends on where they are stored
    const Eval2Args<R> a = args;
    if (a.skip && *a.skip) return;
    const int64_t i = blk * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    if (i < a.n_fe) crad_atom<R, 0>(P, a, i, smask);
    else crad_atom<R, 1>(P, a, i, smask);
}


// ------------------------------------------------------------------ k_ang_fwd
// stage of one angular pair: (g_n, s g_n) interleaved for n = 0..4, pad (2), then the 24
// harmonics in lane-major order (position 12 + 6 ql + m holds p_lm of lm = ql + 4 m), so
// each quad lane reads its six harmonics with three 2-wide loads
constexpr int FSTAGE = 36;
constexpr int FQUAD = 4 * FSTAGE + 4;   // per quad, padded so quads start in different banks

template <typename R, int TI, int TJ>
__device__ __forceinline__ void ang_stage_fwd(const NepDev<R> &P, const Eval2Args<R> &a, const v4<R> &pi,
                                              const v4<R> &si, const v4<R> &pj, const v4<R> &sj, R *st) {
    R dx, dy, dz;
    sep(a.box, pi, pj, dx, dy, dz);
    const R d2 = dx * dx + dy * dy + dz * dz;
    const R ir = rsqrt_(d2), r = d2 * ir;
    R f[NK], g[NCH];
    carrier_f(r, P.inv_rc_a, f);
    contract_k<R, TI, TJ, G_A>(P, f, g);
    const R s = si.x * sj.x + si.y * sj.y + si.z * sj.z;
    v4<R> w0, w1;
    v2<R> w2;
    w0.x = g[0]; w0.y = g[0] * s; w0.z = g[1]; w0.w = g[1] * s;
    w1.x = g[2]; w1.y = g[2] * s; w1.z = g[3]; w1.w = g[3] * s;
    w2.x = g[4]; w2.y = g[4] * s;
    reinterpret_cast<v4<R> *>(st)[0] = w0;
    reinterpret_cast<v4<R> *>(st)[1] = w1;
    reinterpret_cast<v2<R> *>(st)[4] = w2;
    R p[NLM];
    harm_p(dx * ir, dy * ir, dz * ir, p);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v2<R> a0, a1, a2;
        a0.x = p[q]; a0.y = p[q + 4]; a1.x = p[q + 8]; a1.y = p[q + 12]; a2.x = p[q + 16]; a2.y = p[q + 20];
        v2<R> *d = reinterpret_cast<v2<R> *>(st + 12 + 6 * q);
        d[0] = a0; d[1] = a1; d[2] = a2;
    }
}

template <typename R>
__device__ __forceinline__ void ang_fwd_body(const NepDev<R> &P, const Eval2Args<R> &args, int64_t blk,
                                             unsigned char *smem_raw) {
    // the arguments as values: read once from the block's copy, so nothing in the loops below
    // depends on where they are stored
    const Eval2Args<R> a = args;
    if (a.skip && *a.skip) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int quad = lane >> 2, ql = lane & 3;
    const int64_t i = (blk * (blockDim.x >> 5) + warp) * 8 + quad;
    const bool valid = i < a.n;
    R *stage = reinterpret_cast<R *>(smem_raw) + (warp * 8 + quad) * FQUAD;
    const int64_t N = a.n;
    v4<R> pi, si;
    int na0 = 0, na = 0, ti = 0;
    if (valid) {
        pi = a.pos[i];
        si = a.spin[i];
        const int4 c = a.cnt[i];
        na0 = c.x;
        na = c.y;
        ti = i < a.n_fe ? 0 : 1;
    }
    v2<R> BB[6][NCH];   // (B_nlm, BS_nlm) of the lane's six harmonics
#pragma unroll
    for (int m = 0; m < 6; ++m)
#pragma unroll
        for (int n = 0; n < NCH; ++n) BB[m][n] = pair2<R>(R(0), R(0));
    const int nmax = __reduce_max_sync(0xffffffffu, na);
    // the lane's list entry three rounds ahead and its coordinates two rounds ahead are in flight
    v4<R> pjn, sjn, pjn2, sjn2;
    int jn3 = 0;
    if (ql < na) {
        const int j = a.clj[(int64_t)ql * N + i];
        pjn = a.pos[j];
        sjn = a.spin[j];
    }
    if (ql + 4 < na) {
        const int j = a.clj[(int64_t)(ql + 4) * N + i];
        pjn2 = a.pos[j];
        sjn2 = a.spin[j];
    }
    if (ql + 8 < na) jn3 = a.clj[(int64_t)(ql + 8) * N + i];
    for (int base = 0; base < nmax; base += 4) {
        const int p = base + ql;
        const v4<R> pj = pjn, sj = sjn;
        pjn = pjn2;
        sjn = sjn2;
        if (p + 8 < na) {
            pjn2 = a.pos[jn3];
            sjn2 = a.spin[jn3];
        }
        if (p + 12 < na) jn3 = a.clj[(int64_t)(p + 12) * N + i];
        if (p < na) {
            R *st = stage + ql * FSTAGE;
            if (ti == 0) {
                if (p < na0) ang_stage_fwd<R, 0, 0>(P, a, pi, si, pj, sj, st);
                else ang_stage_fwd<R, 0, 1>(P, a, pi, si, pj, sj, st);
            } else {
                if (p < na0) ang_stage_fwd<R, 1, 0>(P, a, pi, si, pj, sj, st);
                else ang_stage_fwd<R, 1, 1>(P, a, pi, si, pj, sj, st);
            }
        }
        __syncwarp();
        const int cnt = min(4, na - base);
        for (int q = 0; q < cnt; ++q) {
            const R *sp = stage + q * FSTAGE;
            const v4<R> w0 = reinterpret_cast<const v4<R> *>(sp)[0];
            const v4<R> w1 = reinterpret_cast<const v4<R> *>(sp)[1];
            const v2<R> w2 = reinterpret_cast<const v2<R> *>(sp)[4];
            const v2<R> gg[NCH] = {pair2<R>(w0.x, w0.y), pair2<R>(w0.z, w0.w), pair2<R>(w1.x, w1.y),
                                   pair2<R>(w1.z, w1.w), w2};
            const v2<R> *pp = reinterpret_cast<const v2<R> *>(sp + 12 + 6 * ql);
            const v2<R> p01 = pp[0], p23 = pp[1], p45 = pp[2];
            const R pv[6] = {p01.x, p01.y, p23.x, p23.y, p45.x, p45.y};
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const v2<R> pl = pair2<R>(pv[m], pv[m]);
#pragma unroll
                for (int n = 0; n < NCH; ++n) BB[m][n] = fma2(gg[n], pl, BB[m][n]);
            }
        }
        __syncwarp();
    }
    // angular sums for the backward pass, and the channel values
    R qa[NCH][4], qs[NCH][4];
#pragma unroll
    for (int n = 0; n < NCH; ++n)
#pragma unroll
        for (int l = 0; l < 4; ++l) { qa[n][l] = R(0); qs[n][l] = R(0); }
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const int lm = lm_of(ql, m);
        const int l = l_of_lm(lm) - 1;
        const R kap = kappa_of_lm<R>(lm);
        if (valid) {   // the harmonic's record: (B_n, BS_n) for n = 0..4, two zeros
            v4<R> *rec = reinterpret_cast<v4<R> *>(a.bsum + ((int64_t)i * NLM + lm) * BREC);
            v4<R> w0, w1, w2;
            w0.x = BB[m][0].x; w0.y = BB[m][0].y; w0.z = BB[m][1].x; w0.w = BB[m][1].y;
            w1.x = BB[m][2].x; w1.y = BB[m][2].y; w1.z = BB[m][3].x; w1.w = BB[m][3].y;
            w2.x = BB[m][4].x; w2.y = BB[m][4].y; w2.z = R(0); w2.w = R(0);
            stg(rec, w0); stg(rec + 1, w1); stg(rec + 2, w2);
        }
#pragma unroll
        for (int n = 0; n < NCH; ++n) {
            const R Bv = BB[m][n].x, BSv = BB[m][n].y;
            const R ka = kap * Bv * Bv, ks = kap * BSv * BSv;
            // l is 1..4 depending on the lane: add into the matching slot
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                qa[n][t] += (t == l) ? ka : R(0);
                qs[n][t] += (t == l) ? ks : R(0);
            }
        }
    }
#pragma unroll
    for (int n = 0; n < NCH; ++n)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            qa[n][t] += __shfl_xor_sync(0xffffffffu, qa[n][t], 1);
            qa[n][t] += __shfl_xor_sync(0xffffffffu, qa[n][t], 2);
            qs[n][t] += __shfl_xor_sync(0xffffffffu, qs[n][t], 1);
            qs[n][t] += __shfl_xor_sync(0xffffffffu, qs[n][t], 2);
        }
    if (valid) {
        // lane ql writes l = ql + 1
#pragma unroll
        for (int n = 0; n < NCH; ++n) {
            R va = qa[n][0], vs = qs[n][0];
#pragma unroll
            for (int t = 1; t < 4; ++t) {
                va = ql == t ? qa[n][t] : va;
                vs = ql == t ? qs[n][t] : vs;
            }
            stg(a.q + (int64_t)(Q_A + n * 4 + ql) * a.qs + i, va);
            stg(a.q + (int64_t)(Q_SA + n * 4 + ql) * a.qs + i, vs);
        }
    }
}


// ------------------------------------------------------------------ k_bwd (fused)
// Quad per atom, lanes over pairs.  Shared memory per atom: the angular adjoints
// dE/dB_nlm, dE/dBS_nlm as 24 records of 12 ((dE/dB, dE/dBS) interleaved per n, pad), then the precontracted
// radial coefficients C^G_k = sum_n Fp^G_n c^G_{n k t_i t_j} for both neighbour
// species (2 x 48).  Stride 388: 388 mod 32 = 4, so the eight atoms of a warp read
// disjoint bank groups.
constexpr int BW_C = 292;
constexpr int BW_ATOM = 388;

template <typename R>
struct BwdAcc2 {
    R fx, fy, fz, hx, hy, hz;
    R w[9];
};

template <typename R, int TI>
__device__ __forceinline__ void bwd_coeffs(const NepDev<R> &P, const R FR[NCH], const R FX[4][NCH], int ql, R *smc) {
#pragma unroll
    for (int tj = 0; tj < 2; ++tj)
#pragma unroll
        for (int g = 0; g < 5; ++g)
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                constexpr int G[5] = {G_R, G_EX, G_DMI, G_ANI, G_SIA};
                R v = R(0);
#pragma unroll
                for (int n = 0; n < NCH; ++n)
                    v += (g == 0 ? FR[n] : FX[g - 1][n]) * (tj == 0 ? P.c[TI][0][G[g]][n][k] : P.c[TI][1][G[g]][n][k]);
                if (((tj * 45 + g * 9 + k) & 3) == ql) smc[tj * 48 + g * 9 + k] = v;
            }
}

template <typename R, int TI, int TJ>
__device__ __forceinline__ void ang_gdg(const NepDev<R> &P, R r, R inv_rc, R g[NCH], R dg[NCH]) {
    R f[NK], df[NK];
    carrier_fd2(r, inv_rc, f, df);
    contract_k2<R, TI, TJ, G_A>(P, f, df, g, dg);
}

template <typename R, int LM>
__device__ __forceinline__ void bwd_harm(const R *__restrict__ bb, R ux, R uy, R uz, R ir, R s, const R g[NCH],
                                         const R dg[NCH], R &accu, R &avx, R &avy, R &avz, R &cj) {
    R p, gx, gy, gz;
    harm_one<R, LM>(ux, uy, uz, p, gx, gy, gz);
    const v4<R> *rec = reinterpret_cast<const v4<R> *>(bb + BREC * LM);
    const v4<R> r0 = rec[0], r1 = rec[1], r2 = rec[2];
    const v2<R> Bp[NCH] = {pair2<R>(r0.x, r0.y), pair2<R>(r0.z, r0.w), pair2<R>(r1.x, r1.y), pair2<R>(r1.z, r1.w),
                           pair2<R>(r2.x, r2.y)};   // (dE/dB_n, dE/dBS_n)
    v2<R> aa = pair2<R>(R(0), R(0)), bq = pair2<R>(R(0), R(0));
#pragma unroll
    for (int n = 0; n < NCH; ++n) {
        aa = fma2(Bp[n], pair2<R>(g[n], g[n]), aa);
        bq = fma2(Bp[n], pair2<R>(dg[n], dg[n]), bq);
    }
    const R aA = aa.x, aS = aa.y, bA = bq.x, bS = bq.y;
    const R av = aA + s * aS, bv = bA + s * bS;
    accu += p * (bv - R(harm_l(LM)) * ir * av);
    avx += av * gx;
    avy += av * gy;
    avz += av * gz;
    cj += aS * p;
    if constexpr (LM + 1 < NLM) bwd_harm<R, LM + 1>(bb, ux, uy, uz, ir, s, g, dg, accu, avx, avy, avz, cj);
}

// one pair record: FP32 as a single 256-bit store (the record is one 32-byte sector), FP64 as
// two 32-byte stores
__device__ __forceinline__ void store_rec(PairRec<float> *p, const float4 &a, const float4 &b) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}
__device__ __forceinline__ void store_rec(PairRec<double> *p, const double4 &a, const double4 &b) {
    stg(&p->a, a);
    stg(&p->b, b);
}

// VIR: the evaluation accumulates the virial parts (a compile-time switch, so the step's
// evaluation keeps no virial accumulators live across its row loops)
template <typename R, bool ANG, bool VIR>
__device__ __forceinline__ void bwd_pair(const NepDev<R> &P, const Eval2Args<R> &a, int ti, int tj, const v4<R> &pi,
                                         const v4<R> &si, const v4<R> &pj, const v4<R> &sj, int j, int t,
                                         const R *sm, BwdAcc2<R> &acc) {
    R dx, dy, dz;
    sep(a.box, pi, pj, dx, dy, dz);
    const R d2 = dx * dx + dy * dy + dz * dz;
    const R ir = rsqrt_(d2), r = d2 * ir;
    const R ux = dx * ir, uy = dy * ir, uz = dz * ir;
    // radial and pairwise-magnetic part with the precontracted coefficients
    R f[NK], df[NK];
    carrier_fd2(r, P.inv_rc_r, f, df);
    const v4<R> *cv = reinterpret_cast<const v4<R> *>(sm + BW_C + tj * 48);
    R C[48];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const v4<R> c4 = cv[q];
        C[4 * q] = c4.x; C[4 * q + 1] = c4.y; C[4 * q + 2] = c4.z; C[4 * q + 3] = c4.w;
    }
    R e0 = 0;
    v2<R> he[4];   // (h_G, e_G) of the four magnetic groups
#pragma unroll
    for (int q = 0; q < 4; ++q) he[q] = pair2<R>(R(0), R(0));
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        e0 += C[k] * df[k];
        const v2<R> fd = pair2<R>(f[k], df[k]);
#pragma unroll
        for (int q = 0; q < 4; ++q) he[q] = fma2(pair2<R>(C[9 * (q + 1) + k], C[9 * (q + 1) + k]), fd, he[q]);
    }
    const R h1 = he[0].x, e1 = he[0].y, h2 = he[1].x, e2 = he[1].y, h3 = he[2].x, e3 = he[2].y, h4 = he[3].x,
            e4 = he[3].y;
    const R sij = si.x * sj.x + si.y * sj.y + si.z * sj.z;
    const R siu = si.x * ux + si.y * uy + si.z * uz;
    const R sju = sj.x * ux + sj.y * uy + sj.z * uz;
    const R wx = si.y * sj.z - si.z * sj.y, wy = si.z * sj.x - si.x * sj.z, wz = si.x * sj.y - si.y * sj.x;
    const R wu = wx * ux + wy * uy + wz * uz;
    const R rad = e0 + e1 * sij + e2 * wu + e3 * siu * sju + e4 * siu * siu;
    const R cSi = (h3 * sju + R(2) * h4 * siu) * ir;
    const R cSj = h3 * siu * ir;
    const R cW = h2 * ir;
    const R along = rad - cSi * siu - cSj * sju - cW * wu;
    R Dx = along * ux + cSi * si.x + cSj * sj.x + cW * wx;
    R Dy = along * uy + cSi * si.y + cSj * sj.y + cW * wy;
    R Dz = along * uz + cSi * si.z + cSj * sj.z + cW * wz;
    R cg = h1;   // coefficient of S_i in dE_i/dS_j (exchange, plus the spin-angular weight below)
    const R cu = h3 * sju + R(2) * h4 * siu;
    acc.hx += h1 * sj.x + h2 * (sj.y * uz - sj.z * uy) + cu * ux;
    acc.hy += h1 * sj.y + h2 * (sj.z * ux - sj.x * uz) + cu * uy;
    acc.hz += h1 * sj.z + h2 * (sj.x * uy - sj.y * ux) + cu * uz;
    if constexpr (ANG) {
        R g[NCH], dg[NCH];
        if (ti == 0) {
            if (tj == 0) ang_gdg<R, 0, 0>(P, r, P.inv_rc_a, g, dg);
            else ang_gdg<R, 0, 1>(P, r, P.inv_rc_a, g, dg);
        } else {
            if (tj == 0) ang_gdg<R, 1, 0>(P, r, P.inv_rc_a, g, dg);
            else ang_gdg<R, 1, 1>(P, r, P.inv_rc_a, g, dg);
        }
        R accu = R(0), avx = R(0), avy = R(0), avz = R(0), cj = R(0);
        bwd_harm<R, 0>(sm, ux, uy, uz, ir, sij, g, dg, accu, avx, avy, avz, cj);
        Dx += accu * ux + ir * avx;
        Dy += accu * uy + ir * avy;
        Dz += accu * uz + ir * avz;
        cg += cj;
        acc.hx += cj * sj.x;
        acc.hy += cj * sj.y;
        acc.hz += cj * sj.z;
    }
    // dE_i/dS_j = (h_EX + c_ij) S_i + h_DMI (u x S_i) + h_ANI (S_i.u) u
    const R Gx = cg * si.x + h2 * (uy * si.z - uz * si.y) + h3 * siu * ux;
    const R Gy = cg * si.y + h2 * (uz * si.x - ux * si.z) + h3 * siu * uy;
    const R Gz = cg * si.z + h2 * (ux * si.y - uy * si.x) + h3 * siu * uz;
    acc.fx += Dx; acc.fy += Dy; acc.fz += Dz;
    if constexpr (VIR) {
        acc.w[0] -= dx * Dx; acc.w[1] -= dx * Dy; acc.w[2] -= dx * Dz;
        acc.w[3] -= dy * Dx; acc.w[4] -= dy * Dy; acc.w[5] -= dy * Dz;
        acc.w[6] -= dz * Dx; acc.w[7] -= dz * Dy; acc.w[8] -= dz * Dz;
    }
    PairRec<R> *rec = a.pd + (int64_t)t * a.n + j;
    v4<R> ra, rb;
    ra.x = Dx; ra.y = Dy; ra.z = Dz; ra.w = Gx;
    rb.x = Gy; rb.y = Gz; rb.z = R(0); rb.w = R(0);
    store_rec(rec, ra, rb);
}

// rows lo, lo+4, ... of one range for lane ql.  Two-level prefetch: the list entry of the
// row two steps ahead and the coordinates of the next row are in flight while a pair is
// computed, so no load waits on a load issued in the same step.
template <typename R, bool ANG, bool VIR>
__device__ __forceinline__ void bwd_rows(const NepDev<R> &P, const Eval2Args<R> &a, int64_t i, int ti, int lo, int hi,
                                         int split, const v4<R> &pi, const v4<R> &si, const R *sm,
                                         BwdAcc2<R> &acc) {
    const int64_t N = a.n;
    int j1 = 0, t1 = 0, j2 = 0, t2 = 0, j3 = 0, t3 = 0;
    v4<R> p1, s1, p2, s2;
    if (lo < hi) {
        j1 = ro(a.clj + (int64_t)lo * N + i);
        t1 = ro(a.cls + (int64_t)lo * N + i) >> 8;
    }
    if (lo + 4 < hi) {
        j2 = ro(a.clj + (int64_t)(lo + 4) * N + i);
        t2 = ro(a.cls + (int64_t)(lo + 4) * N + i) >> 8;
    }
    if (lo + 8 < hi) {
        j3 = ro(a.clj + (int64_t)(lo + 8) * N + i);
        t3 = ro(a.cls + (int64_t)(lo + 8) * N + i) >> 8;
    }
    if (lo < hi) {
        p1 = ro(a.pos + j1);
        s1 = ro(a.spin + j1);
    }
    if (lo + 4 < hi) {
        p2 = ro(a.pos + j2);
        s2 = ro(a.spin + j2);
    }
    for (int row = lo; row < hi; row += 4) {
        const int j = j1, t = t1;
        const v4<R> pj = p1, sj = s1;
        j1 = j2; t1 = t2; p1 = p2; s1 = s2;
        j2 = j3; t2 = t3;
        if (row + 8 < hi) {
            p2 = ro(a.pos + j2);
            s2 = ro(a.spin + j2);
        }
        if (row + 12 < hi) {
            j3 = ro(a.clj + (int64_t)(row + 12) * N + i);
            t3 = ro(a.cls + (int64_t)(row + 12) * N + i) >> 8;
        }
        bwd_pair<R, ANG, VIR>(P, a, ti, row < split ? 0 : 1, pi, si, pj, sj, j, t, sm, acc);
    }
}

template <typename R, bool VIR>
__device__ __forceinline__ void bwd_body(const NepDev<R> &P, const Eval2Args<R> &args, int64_t blk,
                                         unsigned char *smem_raw) {
    // the arguments as values: read once from the block's copy, so nothing in the loops below
    // depends on where they are stored
    const Eval2Args<R> a = args;
    if (a.skip && *a.skip) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int quad = lane >> 2, ql = lane & 3;
    const int64_t i = (blk * (blockDim.x >> 5) + warp) * 8 + quad;
    const bool valid = i < a.n;
    const int64_t N = a.n;
    R *sm = reinterpret_cast<R *>(smem_raw) + (warp * 8 + quad) * BW_ATOM;
    BwdAcc2<R> acc;
    acc.fx = acc.fy = acc.fz = acc.hx = acc.hy = acc.hz = R(0);
#pragma unroll
    for (int t = 0; t < 9; ++t) acc.w[t] = R(0);
    if (valid) {
        const int ti = i < a.n_fe ? 0 : 1;
        const v4<R> pi = ro(a.pos + i), si = ro(a.spin + i);
        const int4 c = ro(a.cnt + i);
        // angular adjoints of this lane's harmonics lm = ql + 4 m from their records (three
        // 16-byte loads each), the gradient entries straight from global memory
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int lm = lm_of(ql, m);
            const int l = l_of_lm(lm);
            const R k2 = R(2) * kappa_of_lm<R>(lm);
            const v4<R> *src = reinterpret_cast<const v4<R> *>(a.bsum + ((int64_t)i * NLM + lm) * BREC);
            v4<R> w0 = ro(src), w1 = ro(src + 1), w2 = ro(src + 2);
            const R *fa = a.fp + (int64_t)(Q_A + l - 1) * N + i, *fs = a.fp + (int64_t)(Q_SA + l - 1) * N + i;
            w0.x *= k2 * ro(fa); w0.y *= k2 * ro(fs); w0.z *= k2 * ro(fa + 4 * N); w0.w *= k2 * ro(fs + 4 * N);
            w1.x *= k2 * ro(fa + 8 * N); w1.y *= k2 * ro(fs + 8 * N); w1.z *= k2 * ro(fa + 12 * N);
            w1.w *= k2 * ro(fs + 12 * N);
            w2.x *= k2 * ro(fa + 16 * N); w2.y *= k2 * ro(fs + 16 * N); w2.z = R(0); w2.w = R(0);
            v4<R> *d = reinterpret_cast<v4<R> *>(sm + BREC * lm);
            d[0] = w0; d[1] = w1; d[2] = w2;
        }
        R FR[NCH], FX[4][NCH];
#pragma unroll
        for (int n = 0; n < NCH; ++n) {
            FR[n] = ro(a.fp + (int64_t)(Q_R + n) * N + i);
            FX[0][n] = ro(a.fp + (int64_t)(Q_EX + n) * N + i);
            FX[1][n] = ro(a.fp + (int64_t)(Q_DMI + n) * N + i);
            FX[2][n] = ro(a.fp + (int64_t)(Q_ANI + n) * N + i);
            FX[3][n] = ro(a.fp + (int64_t)(Q_SIA + n) * N + i);
        }
        if (ql == 0) {   // onsite term dE_i/dS_i = 2 Fp_O S_i, counted once per atom
            const R fo = R(2) * ro(a.fp + (int64_t)Q_O * N + i);
            acc.hx = fo * si.x; acc.hy = fo * si.y; acc.hz = fo * si.z;
        }
        if (ti == 0) bwd_coeffs<R, 0>(P, FR, FX, ql, sm + BW_C);
        else bwd_coeffs<R, 1>(P, FR, FX, ql, sm + BW_C);
        __syncwarp(0xfu << (quad * 4));
        const int ca = a.cap_ang;
        bwd_rows<R, true, VIR>(P, a, i, ti, ql, c.y, c.x, pi, si, sm, acc);
        bwd_rows<R, false, VIR>(P, a, i, ti, ca + ql, ca + c.w, ca + c.z, pi, si, sm, acc);
    }
    // per-atom sums over the quad
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        acc.fx += __shfl_xor_sync(0xffffffffu, acc.fx, o);
        acc.fy += __shfl_xor_sync(0xffffffffu, acc.fy, o);
        acc.fz += __shfl_xor_sync(0xffffffffu, acc.fz, o);
        acc.hx += __shfl_xor_sync(0xffffffffu, acc.hx, o);
        acc.hy += __shfl_xor_sync(0xffffffffu, acc.hy, o);
        acc.hz += __shfl_xor_sync(0xffffffffu, acc.hz, o);
    }
    if constexpr (VIR) {
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            acc.w[t] += __shfl_xor_sync(0xffffffffu, acc.w[t], 1);
            acc.w[t] += __shfl_xor_sync(0xffffffffu, acc.w[t], 2);
        }
    }
    if (valid && ql == 0) {
        v4<R> f4, g4;
        f4.x = acc.fx; f4.y = acc.fy; f4.z = acc.fz; f4.w = R(0);
        g4.x = acc.hx; g4.y = acc.hy; g4.z = acc.hz; g4.w = R(0);
        stg(a.fown + i, f4);
        stg(a.gii + i, g4);
        if constexpr (VIR) {
#pragma unroll
            for (int t = 0; t < 9; ++t) stg(a.wpart + (int64_t)t * N + i, acc.w[t]);
        }
    }
}


// The evaluation kernels over an argument table (sl_batch.h: a system's own table or a
// batch's).  MINB: the register budget, as the minimum resident blocks per SM.  The
// mixed-precision kernels default to 4 blocks (128 registers) and have a second budget each,
// which sl_autotune may choose: radial 3 blocks, angular unconstrained, backward 3 blocks.
template <typename R, int MINB = sizeof(R) == 4 ? 4 : 2>
__global__ void __launch_bounds__(128, MINB) k_crad(const __grid_constant__ NepDev<R> P,
                                                    const Eval2Args<R> *__restrict__ tab, SlotMap sm,
                                                    const __grid_constant__ Eval2Args<R> solo) {
    __shared__ uint32_t smask[MASKW_MAX][128];   // blocks have at most 128 threads
    one_work(tab, sm, solo, [&](const Eval2Args<R> &a, int64_t blk, int64_t) { crad_body(P, a, blk, smask); });
}
template <typename R, int MINB = sizeof(R) == 4 ? 4 : 1>
__global__ void __launch_bounds__(128, MINB) k_ang_fwd(const __grid_constant__ NepDev<R> P,
                                                       const Eval2Args<R> *__restrict__ tab, SlotMap sm,
                                                       const __grid_constant__ Eval2Args<R> solo) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    one_work(tab, sm, solo,
             [&](const Eval2Args<R> &a, int64_t blk, int64_t) { ang_fwd_body(P, a, blk, smem_raw); });
}
template <typename R, int MINB = sizeof(R) == 4 ? 4 : 1, bool VIR = false>
__global__ void __launch_bounds__(128, MINB) k_bwd(const __grid_constant__ NepDev<R> P,
                                                   const Eval2Args<R> *__restrict__ tab, SlotMap sm,
                                                   const __grid_constant__ Eval2Args<R> solo) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    one_work(tab, sm, solo,
             [&](const Eval2Args<R> &a, int64_t blk, int64_t) { bwd_body<R, VIR>(P, a, blk, smem_raw); });
}

// ------------------------------------------------------------------ launch
// The arguments of an evaluation at `at` (null members: the state).
template <typename R>
static Eval2Args<R> args2(Sys &s, const EvalAt &at, bool want_virial) {
    Eval2Args<R> a;
    if constexpr (sizeof(R) == 8) {
        a.pos = reinterpret_cast<const v4<R> *>(at.pos ? at.pos : s.pos);
        a.spin = reinterpret_cast<const v4<R> *>(at.spin ? at.spin : s.spin);
        a.box = *reinterpret_cast<const BoxDev<R> *>(&s.boxd);
    } else {
        a.pos = reinterpret_cast<const v4<R> *>(at.posf ? at.posf : s.posf);
        a.spin = reinterpret_cast<const v4<R> *>(at.spinf ? at.spinf : s.spinf);
        a.box = *reinterpret_cast<const BoxDev<R> *>(&s.boxf);
    }
    a.skip = at.skip;
    a.nbr = s.nbr; a.seg = s.seg; a.rev = s.rev; a.capr = nbr_stride(s.cap); a.n = s.n; a.n_fe = s.n_fe;
    a.cap = s.cap; a.cap_ang = s.cap_ang;
    a.clj = s.clj; a.cls = s.cls; a.cnt = s.cnt; a.mask = s.cmask; a.maskw = s.maskw;
    a.q = (R *)s.q; a.qs = s.qs; a.bsum = (R *)s.bsum; a.fp = (R *)s.fp; a.ei = (R *)s.ei;
    a.pd = (PairRec<R> *)s.pairs; a.fown = (v4<R> *)s.fown; a.gii = (v4<R> *)s.gii;
    a.wpart = (R *)s.wpart; a.want_virial = want_virial; a.status = s.status;
    return a;
}

template <typename R>
static constexpr int quad_block() { return sizeof(R) == 8 ? 64 : 128; }
template <typename R>
static constexpr size_t fwd_smem(int qb = quad_block<R>()) { return (size_t)(qb / 32) * 8 * FQUAD * sizeof(R); }
template <typename R>
static constexpr size_t bwdf_smem(int qb = quad_block<R>()) { return (size_t)(qb / 32) * 8 * BW_ATOM * sizeof(R); }

int default_quad_block(int prec) { return prec == 0 ? quad_block<double>() : quad_block<float>(); }

// Dynamic shared-memory limits of the quad kernels, set once per device (function
// attributes belong to the device's context), safe to call from several threads.
void eval2_init() {
    static std::mutex mu;
    static uint64_t done = 0;   // bit d: device d is set up
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && (done >> dev & 1u)) return;
    cudaFuncSetAttribute(k_ang_fwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<float>());
    cudaFuncSetAttribute(k_ang_fwd<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<float>());
    cudaFuncSetAttribute(k_ang_fwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<double>());
    cudaFuncSetAttribute(k_bwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwdf_smem<float>());
    cudaFuncSetAttribute(k_bwd<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwdf_smem<float>());
    cudaFuncSetAttribute(k_bwd<float, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwdf_smem<float>());
    cudaFuncSetAttribute(k_bwd<float, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwdf_smem<float>());
    cudaFuncSetAttribute(k_bwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwdf_smem<double>());
    cudaFuncSetAttribute(k_bwd<double, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwdf_smem<double>());
    if (dev < 64) done |= 1ull << dev;
}

// ---- argument tables (sl_batch.h)
size_t fused_eval_size(int prec) { return prec == 0 ? sizeof(Eval2Args<double>) : sizeof(Eval2Args<float>); }

// slot kinds: the step's evaluation (at the state, no virial), the full one (with the virial
// parts) and the midpoint iteration's (at its point, with its skip flag)
static EvalAt eval_point(const Sys &s, int kind) {
    EvalAt at;
    if (kind == SK_MID && s.mid_iters > 0) {
        at.pos = s.posmid; at.posf = s.posmidf; at.spin = s.mids; at.spinf = s.midsf;
        at.skip = reinterpret_cast<const int *>(reinterpret_cast<const char *>(s.md) + offsetof(MidDev, converged));
    }
    return at;
}

void fused_put_eval(Sys &s, int r, int kind, const FusedTables &t, unsigned char *img, int64_t *blocks) {
    const EvalAt at = eval_point(s, kind);
    if (s.prec == 0) reinterpret_cast<Eval2Args<double> *>(img + t.o_eval)[r] = args2<double>(s, at, kind == SK_FULL);
    else reinterpret_cast<Eval2Args<float> *>(img + t.o_eval)[r] = args2<float>(s, at, kind == SK_FULL);
    const int qb = default_quad_block(s.prec);
    blocks[FK_CRAD] = (s.n + 127) / 128;
    blocks[FK_ANG] = blocks[FK_BWD] = (s.n + qb / 4 - 1) / (qb / 4);
}

// Radial, angular, network and backward over a table, each launch in its own shape
// (L[k].block threads, 0: the default) and register budget (L[k].minb, 0: the default).
template <typename R>
void launch_eval_t(const FusedTables &t, const NepDev<R> &P, const Launch *L, cudaStream_t st, cudaEvent_t *ev) {
    // a system's own launch passes its argument block as a kernel parameter; a batch's reads
    // the table (the same for the four kernels of one launch group)
    const Eval2Args<R> *tab = L[0].solo ? nullptr : t.at<Eval2Args<R>>(t.o_eval);
    const Eval2Args<R> so = solo_args<Eval2Args<R>>(L[0]);
    const SlotMap s0 = L[0].slots(), s1 = L[1].slots(), s3 = L[3].slots();
    const int cb = L[0].block ? L[0].block : 128;
    const int qa = L[1].block ? L[1].block : quad_block<R>();
    const int qw = L[3].block ? L[3].block : quad_block<R>();
    if (ev) cudaEventRecord(ev[0], st);
    // compaction and radial channels in one kernel: the compaction group is empty
    if (ev) cudaEventRecord(ev[1], st);
    bool variant = false;
    if constexpr (sizeof(R) == 4) {
        variant = L[0].minb == 3;
        if (variant) k_crad<R, 3><<<L[0].grid, cb, 0, st>>>(P, tab, s0, so);
    }
    if (!variant) k_crad<R><<<L[0].grid, cb, 0, st>>>(P, tab, s0, so);
    if (ev) cudaEventRecord(ev[2], st);
    variant = false;
    if constexpr (sizeof(R) == 4) {
        variant = L[1].minb == 1;
        if (variant) k_ang_fwd<R, 1><<<L[1].grid, qa, fwd_smem<R>(qa), st>>>(P, tab, s1, so);
    }
    if (!variant) k_ang_fwd<R><<<L[1].grid, qa, fwd_smem<R>(qa), st>>>(P, tab, s1, so);
    if (ev) cudaEventRecord(ev[3], st);
    if constexpr (sizeof(R) == 4) launch_net_t_tc(t, P, L[2], st);
    else launch_net_t_fp64(t, P, L[2], st);
    if (ev) cudaEventRecord(ev[4], st);
    // the virial parts: only a system's own full evaluation asks for them (a batch's slots are
    // set up for the step's evaluation, which has none)
    const bool vir = L[3].solo && so.want_virial;
    variant = false;
    if constexpr (sizeof(R) == 4) {
        variant = L[3].minb == 3;
        if (variant && vir) k_bwd<R, 3, true><<<L[3].grid, qw, bwdf_smem<R>(qw), st>>>(P, tab, s3, so);
        else if (variant) k_bwd<R, 3><<<L[3].grid, qw, bwdf_smem<R>(qw), st>>>(P, tab, s3, so);
    }
    if (!variant && vir) k_bwd<R, sizeof(R) == 4 ? 4 : 1, true><<<L[3].grid, qw, bwdf_smem<R>(qw), st>>>(P, tab, s3, so);
    else if (!variant) k_bwd<R><<<L[3].grid, qw, bwdf_smem<R>(qw), st>>>(P, tab, s3, so);
    if (ev) cudaEventRecord(ev[5], st);
}
template void launch_eval_t<float>(const FusedTables &, const NepDev<float> &, const Launch *, cudaStream_t,
                                   cudaEvent_t *);
template void launch_eval_t<double>(const FusedTables &, const NepDev<double> &, const Launch *, cudaStream_t,
                                    cudaEvent_t *);

// The system's own evaluation: at the midpoint point while s.at is set (the midpoint
// iteration), else at the state, with the virial parts when asked for.
void launch_eval(Sys &s, bool want_virial, cudaEvent_t *ev) {
    if (s.n == 0) return;
    const int kind = s.at.pos ? SK_MID : want_virial ? SK_FULL : SK_STEP;
    const Launch L[4] = {solo_launch(s, FK_CRAD, kind), solo_launch(s, FK_ANG, kind), solo_launch(s, FK_NET, kind),
                         solo_launch(s, FK_BWD, kind)};
    if (s.prec == 0) launch_eval_t<double>(s.solo->t, s.pd, L, s.stream, ev);
    else launch_eval_t<float>(s.solo->t, s.pf, L, s.stream, ev);
}

}  // namespace sl
