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
// This file holds the per-atom forward (one thread per atom, used by the
// no-allocation entry point) and the CUDA-core network k_mlp:
//   E_i and Fp = dE_i/dq_i.
// The step's evaluation kernels are in sl_eval2.cu; forces and fields are gathered
// without atomics (sl_integrate.cu):
//   F_k = sum_j (dE_k/dr_kj - dE_j/dr_jk),  H_k = -dE_k/dS_k - sum_j dE_j/dS_k + Zeeman.
//
// Atoms are stored species-major, so a warp almost always has one centre species;
// the neighbour list is segmented by neighbour species, so inside a segment both
// species are compile-time constants and every coefficient is a constant operand.
#include <cstddef>
#include <mutex>

#include "sl_internal.h"
#include "sl_batch.h"
#include "sl_fused.cuh"

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

// ------------------------------------------------------------------ network
// E_i = sum_h w1_h tanh(z_h) - b1, z_h = sum_v W0_hv s_v q_v - b0_h;
// Fp_v = s_v sum_h w1_h (1 - tanh^2 z_h) W0_hv.
template <typename R>
__device__ __forceinline__ void mlp_atom(const NepDev<R> &P, const R *__restrict__ q, R *__restrict__ fp,
                                         R *__restrict__ ei, int64_t n, int64_t qs, int64_t i) {
    R x[DIM];
#pragma unroll
    for (int v = 0; v < DIM; ++v) x[v] = q[(int64_t)v * qs + i] * P.scal[v];
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

// over an argument table (sl_batch.h), one 128-thread block per 128 atoms of a slot
template <typename R>
__global__ void __launch_bounds__(128) k_mlp(const __grid_constant__ NepDev<R> P, const NetArgs<R> *__restrict__ tab,
                                             SlotMap sm, const __grid_constant__ NetArgs<R> solo) {
    one_work(tab, sm, solo, [&](const NetArgs<R> &a, int64_t blk, int64_t) {
        if (a.skip && *a.skip) return;
        const int64_t i = blk * 128 + threadIdx.x;
        if (i < a.n) mlp_atom(P, a.q, a.fp, a.ei, a.n, a.qs, i);
    });
}

// ---- argument tables (sl_batch.h): the FP64 network over NetArgs, the mixed one
// (sl_mlp_tc.cu) over MlpArgs holding each slot's TMA map
size_t fused_net_size(int prec) { return prec == 0 ? sizeof(NetArgs<double>) : sizeof(MlpArgs); }

void fused_put_net(Sys &s, int r, int kind, const FusedTables &t, unsigned char *img, int64_t *blocks) {
    // the midpoint iteration's evaluations stop once it has converged
    const int *skip = kind == SK_MID && s.md ? reinterpret_cast<const int *>(reinterpret_cast<const char *>(s.md) +
                                                                             offsetof(MidDev, converged))
                                             : nullptr;
    if (s.prec == 0) {
        NetArgs<double> a;
        a.q = (const double *)s.q; a.fp = (double *)s.fp; a.ei = (double *)s.ei; a.n = s.n; a.qs = s.qs;
        a.skip = skip;
        reinterpret_cast<NetArgs<double> *>(img + t.o_net)[r] = a;
    } else {
        MlpArgs a;
        a.qmap = s.qmap; a.n = s.n; a.fp = (float *)s.fp; a.ei = (float *)s.ei; a.status = s.status;
        a.skip = skip; a.wimg = s.mlp_img;
        reinterpret_cast<MlpArgs *>(img + t.o_net)[r] = a;
    }
    blocks[FK_NET] = (s.n + 127) / 128;   // atoms of 128-thread blocks, or 128-atom tensor-core tiles
}

void launch_net_t_fp64(const FusedTables &t, const NepDev<double> &P, const Launch &L, cudaStream_t st) {
    k_mlp<double><<<L.grid, 128, 0, st>>>(P, L.solo ? nullptr : t.at<NetArgs<double>>(t.o_net), L.slots(),
                                          solo_args<NetArgs<double>>(L));
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
    // species index the per-species coefficient tables: a value outside [0, NS) in this
    // atom or in any atom it would pair with is reported and the atom is skipped (the
    // host then rejects the whole call)
    const int ti = species[i];
    if (ti < 0 || ti >= NS) {
        atomicOr(status, ST_BAD_SPECIES);
        return;
    }
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
        const int tj = species[j];
        if (tj < 0 || tj >= NS) {
            atomicOr(status, ST_BAD_SPECIES);
            return;
        }
        if (m >= MAX_NBR) { overflow = true; continue; }
        const int key = ((d2 < P.rc_a2 ? 0 : 2) + tj) * MAX_ATOMS + j;
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
    // descriptor by fwd_atom (one thread per atom, harmonic form of the angular channels;
    // the step's kernels in sl_eval2.cu compute the same sums with another work split)
    EvalArgs<double> a;
    a.pos = pos; a.spin = spin; a.nbr = nbr; a.seg = seg; a.n = n; a.n_fe = 0; a.box = box;
    a.q = q; a.bsum = bsum;
    if (ti == 0) fwd_atom<double, 0>(P, a, i);
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
