// sl_texture.cu -- on-device texture diagnostics of a film (arXiv 2606.14073, Fig. 7 and
// Section 8: helix-to-skyrmion textures in a thin FeGe stripe).
//
//   in-plane grid  the two axes other than the film normal, n = max(1, floor(L / cell))
//                  equal cells each; atoms beyond a non-periodic edge go to the edge cell
//   m(cell)        normalised sum of the spins of the column (zero when it vanishes)
//   Q              Berg-Luescher lattice topological charge: every plaquette
//                  (a,b) -> (a+1,b) -> (a+1,b+1) -> (a,b+1) gives the counter-clockwise
//                  triangles (m00, m10, m11) and (m00, m11, m01), each contributing its
//                  signed solid angle 2 atan2(m1.(m2 x m3), 1 + m1.m2 + m2.m3 + m3.m1);
//                  Q = sum / 4 pi; plaquettes wrap across periodic axes only; triangles
//                  touching an empty cell add nothing.
// Determinism: the column sums are accumulated as 2^-40 fixed-point integers (integer
// atomics are exact and order-free); the charge is a fixed-grid tree reduction summed
// in block order.
#include <cmath>

#include "sl_internal.h"

namespace sl {
namespace {

constexpr int TEX_BLOCKS = 256;
constexpr double TEX_SCALE = 1099511627776.0;   // 2^40

struct TexGrid {
    int a, b;            // in-plane axes
    int na, nb;
    double wa, wb;
    int pa, pb;          // periodic flags
};

__device__ __forceinline__ int cell_index(double x, double w, int n, int per) {
    long long k = (long long)floor(x / w);
    if (per) {
        k %= n;
        if (k < 0) k += n;
    } else {
        k = k < 0 ? 0 : (k >= n ? n - 1 : k);
    }
    return (int)k;
}

__global__ void __launch_bounds__(256) k_tex_bin(const double4 *__restrict__ pos, const double4 *__restrict__ spin,
                                                 int64_t n, TexGrid g, unsigned long long *__restrict__ acc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 p = pos[i], s = spin[i];
    const double pc[3] = {p.x, p.y, p.z};
    const int ia = cell_index(pc[g.a], g.wa, g.na, g.pa);
    const int ib = cell_index(pc[g.b], g.wb, g.nb, g.pb);
    const int64_t c = (int64_t)ib * g.na + ia;
    atomicAdd(acc + 3 * c, (unsigned long long)llrint(s.x * TEX_SCALE));
    atomicAdd(acc + 3 * c + 1, (unsigned long long)llrint(s.y * TEX_SCALE));
    atomicAdd(acc + 3 * c + 2, (unsigned long long)llrint(s.z * TEX_SCALE));
}

__global__ void __launch_bounds__(256) k_tex_norm(const unsigned long long *__restrict__ acc, int64_t cells,
                                                  double4 *__restrict__ m) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= cells) return;
    const double x = (double)(long long)acc[3 * c] / TEX_SCALE;
    const double y = (double)(long long)acc[3 * c + 1] / TEX_SCALE;
    const double z = (double)(long long)acc[3 * c + 2] / TEX_SCALE;
    const double nn = sqrt(x * x + y * y + z * z);
    if (nn > 0) m[c] = make_double4(x / nn, y / nn, z / nn, 1.0);
    else m[c] = make_double4(0.0, 0.0, 0.0, 0.0);   // .w = 0: empty column
}

__device__ __forceinline__ double tri_angle(const double4 &p, const double4 &q, const double4 &r) {
    if (p.w == 0.0 || q.w == 0.0 || r.w == 0.0) return 0.0;
    const double cx = q.y * r.z - q.z * r.y, cy = q.z * r.x - q.x * r.z, cz = q.x * r.y - q.y * r.x;
    const double num = p.x * cx + p.y * cy + p.z * cz;
    const double den = 1.0 + (p.x * q.x + p.y * q.y + p.z * q.z) + (q.x * r.x + q.y * r.y + q.z * r.z) +
                       (r.x * p.x + r.y * p.y + r.z * p.z);
    return 2.0 * atan2(num, den);
}

__global__ void __launch_bounds__(256) k_tex_charge(const double4 *__restrict__ m, TexGrid g,
                                                    double *__restrict__ part) {
    __shared__ double red[256];
    const int ra = g.pa ? g.na : g.na - 1, rb = g.pb ? g.nb : g.nb - 1;
    const int64_t np = (int64_t)(ra > 0 ? ra : 0) * (rb > 0 ? rb : 0);
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % ra), j = (int)(p / ra);
        const int i1 = (i + 1) % g.na, j1 = (j + 1) % g.nb;
        const double4 m00 = m[(int64_t)j * g.na + i], m10 = m[(int64_t)j * g.na + i1];
        const double4 m11 = m[(int64_t)j1 * g.na + i1], m01 = m[(int64_t)j1 * g.na + i];
        acc += tri_angle(m00, m10, m11) + tri_angle(m00, m11, m01);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

}  // namespace

int texture_grid(const Sys &s, int normal, double cell, int *na, int *nb) {
    const int a = normal == 0 ? 1 : 0, b = normal == 2 ? 1 : 2;
    *na = (int)std::max(1.0, std::floor(s.box[a] / cell));
    *nb = (int)std::max(1.0, std::floor(s.box[b] / cell));
    return 0;
}

// Fills m (host, [nb][na][3], may be null) and Q (may be null).  Scratch is kept in the
// system and grown on demand.
cudaError_t launch_texture(Sys &s, int normal, double cell, double *h_m, double *Q) {
    TexGrid g;
    g.a = normal == 0 ? 1 : 0;
    g.b = normal == 2 ? 1 : 2;
    texture_grid(s, normal, cell, &g.na, &g.nb);
    g.wa = s.box[g.a] / g.na;
    g.wb = s.box[g.b] / g.nb;
    g.pa = s.per[g.a];
    g.pb = s.per[g.b];
    const int64_t cells = (int64_t)g.na * g.nb;
    cudaError_t e;
    if (cells > s.tex_cells) {
        if (s.tex_acc) cudaFree(s.tex_acc);
        if (s.tex_m) cudaFree(s.tex_m);
        s.tex_acc = nullptr;
        s.tex_m = nullptr;
        s.tex_cells = 0;
        if ((e = cudaMalloc((void **)&s.tex_acc, sizeof(unsigned long long) * 3 * cells)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void **)&s.tex_m, sizeof(double4) * cells)) != cudaSuccess) return e;
        s.tex_cells = cells;
    }
    if (!s.tex_part && (e = cudaMalloc((void **)&s.tex_part, sizeof(double) * TEX_BLOCKS)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(s.tex_acc, 0, sizeof(unsigned long long) * 3 * cells, s.stream)) != cudaSuccess) return e;
    if (s.n > 0)
        k_tex_bin<<<(unsigned)((s.n + 255) / 256), 256, 0, s.stream>>>(s.pos, s.spin, s.n, g, s.tex_acc);
    k_tex_norm<<<(unsigned)((cells + 255) / 256), 256, 0, s.stream>>>(s.tex_acc, cells, s.tex_m);
    k_tex_charge<<<TEX_BLOCKS, 256, 0, s.stream>>>(s.tex_m, g, s.tex_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<double> part(TEX_BLOCKS);
    if ((e = cudaMemcpyAsync(part.data(), s.tex_part, sizeof(double) * TEX_BLOCKS, cudaMemcpyDeviceToHost,
                             s.stream)) != cudaSuccess)
        return e;
    std::vector<double4> hm;
    if (h_m) {
        hm.resize((size_t)cells);
        if ((e = cudaMemcpyAsync(hm.data(), s.tex_m, sizeof(double4) * cells, cudaMemcpyDeviceToHost, s.stream)) !=
            cudaSuccess)
            return e;
    }
    if ((e = cudaStreamSynchronize(s.stream)) != cudaSuccess) return e;
    if (Q) {
        double sum = 0.0;
        for (int b = 0; b < TEX_BLOCKS; ++b) sum += part[b];
        *Q = sum / (4.0 * M_PI);
    }
    if (h_m)
        for (int64_t c = 0; c < cells; ++c) {
            h_m[3 * c] = hm[c].x;
            h_m[3 * c + 1] = hm[c].y;
            h_m[3 * c + 2] = hm[c].z;
        }
    return cudaSuccess;
}

}  // namespace sl
