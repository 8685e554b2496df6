// sl_neighbors.cu -- cell binning and neighbour lists on the device.
//
// The paper's workload includes cutoff-based neighbour construction every step
// it is needed (Sections 5.1.1, 6.2); here the lists carry a skin and are rebuilt
// when an atom has moved more than skin/2 since the last build.
//
// List definition (bit-exact): j is a candidate of i when
//   t_a = x_ja - x_ia;  t_a -= L_a * rint(t_a / L_a)  (periodic dims)
//   d2 = (t_x*t_x + t_y*t_y) + t_z*t_z  <  (rc_rad + skin)^2
// in FP64 with no contraction.  An FP32 pre-test settles pairs far from the
// cutoff; only pairs within a margin of it take the exact FP64 test.
// Each list is split in four segments -- angular candidates (d2 < (rc_ang+skin)^2)
// of neighbour species 0 and 1, then the remaining radial candidates of species
// 0 and 1 -- and each segment is ordered by the neighbour's caller index, so every
// per-atom sum runs in an order that does not depend on the internal atom order.
#include <algorithm>
#include <cstdio>

#include "sl_internal.h"
#include "sl_batch.h"
#include "sl_fused.cuh"
#include "sl_rebuild.cuh"

namespace sl {

namespace {

__device__ __forceinline__ double exact_d2(double xi, double yi, double zi, double xj, double yj, double zj,
                                           const BoxDev<double> &b, const int per[3]) {
    double t[3] = {__dsub_rn(xj, xi), __dsub_rn(yj, yi), __dsub_rn(zj, zi)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (per[a]) {
            const double q = rint(__ddiv_rn(t[a], b.L[a]));
            t[a] = __dsub_rn(t[a], __dmul_rn(b.L[a], q));
        }
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(t[0], t[0]), __dmul_rn(t[1], t[1])), __dmul_rn(t[2], t[2]));
}



__device__ __forceinline__ void bin_body(const BinArgs &r, int64_t blk, int64_t nblk) {
    if (r.flag && *r.flag == 0) return;
    const GridArgs &g = r.g;
    for (int64_t i = blk * (int64_t)blockDim.x + threadIdx.x; i < r.n; i += nblk * blockDim.x) {
    const double4 p = r.pos[i];
    const double x[3] = {p.x, p.y, p.z};
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int ci = (int)floor(x[a] / g.w[a]);
        c[a] = min(max(ci, 0), g.nc[a] - 1);
    }
    const int cell = (c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0];
    r.of[i] = cell;
    atomicAdd(r.count + cell, 1);
    }
}

// Exclusive scan of count[0..m) into start[0..m] by one whole block (s_part: blockDim.x ints).
__device__ __forceinline__ void scan_body(const BinArgs &r, int *s_part, int &s_carry) {
    if (r.flag && *r.flag == 0) return;
    const int *__restrict__ count = r.count;
    int *__restrict__ start = r.start;
    const int m = r.ncell;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < m; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < m ? count[i] : 0;
        s_part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < blockDim.x; off <<= 1) {
            const int t = threadIdx.x >= off ? s_part[threadIdx.x - off] : 0;
            __syncthreads();
            s_part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < m) start[i] = s_carry + s_part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += s_part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) start[m] = s_carry;
    __syncthreads();   // the block's next work item reuses s_part and s_carry
}

// Atoms into their cells, with a cell-ordered copy of the FP32 position and of the
// key (species << 30 | caller index) so the list build reads candidates contiguously.
__device__ __forceinline__ void scatter_body(const BinArgs &r, int64_t blk, int64_t nblk) {
    if (r.flag && *r.flag == 0) return;
    for (int64_t i = blk * (int64_t)blockDim.x + threadIdx.x; i < r.n; i += nblk * blockDim.x) {
        const int c = r.of[i];
        const int p = r.start[c] + atomicAdd(r.fill + c, 1);
        r.atoms[p] = (int)i;
        r.cposf[p] = r.posf[i];
        r.ckey[p] = ((uint32_t)r.species[i] << 30) | (uint32_t)r.orig[i];
    }
}




// Warp per atom.  Lanes take the candidates of the stencil cells 32 at a time;
// pairs inside the list cutoff are appended to a per-warp shared-memory buffer
// (ballot/popc, so the append order is the scan order), the buffer is sorted
// by (segment, caller index) with a warp bitonic sort, and written out.

// Ascending bitonic sort of 32*E keys held E per lane (element r*32 + lane in
// register r): strides below 32 exchange through shuffles, larger ones inside the lane.
template <int E>
__device__ __forceinline__ void warp_bitonic(uint32_t (&k)[E], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int e = r * 32 + lane;
                const bool asc = (e & size) == 0;
                if (stride >= 32) {
                    const int rp = r ^ (stride >> 5);
                    if (rp > r) {
                        const uint32_t u = k[r], v = k[rp];
                        const bool sw = (u > v) == asc;
                        k[r] = sw ? v : u;
                        k[rp] = sw ? u : v;
                    }
                } else {
                    const uint32_t v = __shfl_xor_sync(0xffffffffu, k[r], stride);
                    const bool lower = (lane & stride) == 0;
                    k[r] = (lower == asc) ? min(k[r], v) : max(k[r], v);
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void sort_and_store(const uint32_t *key, int mm, int lane, uint32_t *out) {
    uint32_t k[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int e = r * 32 + lane;
        k[r] = e < mm ? key[e] : 0xFFFFFFFFu;
    }
    warp_bitonic<E>(k, lane);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < E; ++r) out[r * 32 + lane] = k[r];
    __syncwarp();
}

__device__ __forceinline__ int wrap_cell(int x, int nc) { return x < 0 ? x + nc : (x >= nc ? x - nc : x); }

constexpr int SORT_MAX = 256;

struct ListSmem {
    uint32_t key[LB_WARPS][SORT_MAX];
    int off[LB_WARPS][32], p0[LB_WARPS][32];   // stencil cells of each warp's atom
};

__device__ __forceinline__ void lists_body(const ListArgs &args, int64_t blk, int64_t nblk, ListSmem &sm) {
    const ListArgs a = args;   // as values: the stores below cannot make the compiler re-read them
    if (a.flag && *a.flag == 0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *key = sm.key[w];
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t i = blk * LB_WARPS + w; i < a.n; i += nblk * LB_WARPS) {
        const double4 pi = a.pos[i];
        const float4 pfi = a.posf[i];
        const int cc = a.cell_of[i];
        int ci[3] = {cc % a.g.nc[0], (cc / a.g.nc[0]) % a.g.nc[1], cc / (a.g.nc[0] * a.g.nc[1])};
        int lo[3], hi[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (a.g.per[d] && a.g.nc[d] < 3) { lo[d] = 0; hi[d] = a.g.nc[d] - 1; }
            else if (a.g.per[d]) { lo[d] = ci[d] - 1; hi[d] = ci[d] + 1; }
            else { lo[d] = max(ci[d] - 1, 0); hi[d] = min(ci[d] + 1, a.g.nc[d] - 1); }
        }
        const uint32_t self = (uint32_t)a.orig[i];
        // The stencil cells' candidates are walked as one flattened sequence in the cell order
        // below (z, y, x), 32 per round, with the next round's keys and positions in flight
        // while the current round is tested.  Lane c < nst holds cell c's first cell-ordered
        // position and its exclusive offset in the sequence.
        const int sx = hi[0] - lo[0] + 1, sy = hi[1] - lo[1] + 1, sz = hi[2] - lo[2] + 1;
        const int nst = sx * sy * sz;   // at most 27 cells
        int my_p0 = 0, my_len = 0;
        if (lane < nst) {
            const int x = lo[0] + lane % sx, y = lo[1] + (lane / sx) % sy, z = lo[2] + lane / (sx * sy);
            const int c = (wrap_cell(z, a.g.nc[2]) * a.g.nc[1] + wrap_cell(y, a.g.nc[1])) * a.g.nc[0] +
                          wrap_cell(x, a.g.nc[0]);
            my_p0 = a.cell_start[c];
            my_len = a.cell_start[c + 1] - my_p0;
        }
        int incl = my_len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int *off = sm.off[w], *p0 = sm.p0[w];
        if (lane < nst) {
            off[lane] = incl - my_len;
            p0[lane] = my_p0;
        }
        __syncwarp();
        // cell-ordered position of candidate f of the sequence: the last cell whose offset is
        // <= f holds it (empty cells share the offset of the cell after them).  f grows by 32
        // per round, so each lane moves its cell pointer forward instead of searching.
        int cl = 0;
        auto position_of = [&](int f) {
            while (cl + 1 < nst && off[cl + 1] <= f) ++cl;
            return p0[cl] + (f - off[cl]);
        };
        int pn = -1;
        uint32_t kn = 0;
        float4 fn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < total) {
            pn = position_of(lane);
            kn = a.ckey[pn];
            fn = a.cposf[pn];
        }
        int m = 0, nang = 0;
        for (int base = 0; base < total; base += 32) {
            const int p = pn;
            const uint32_t k = kn;
            const float4 pfj = fn;
            pn = -1;
            if (base + 32 + lane < total) {   // the next round's candidates in flight
                pn = position_of(base + 32 + lane);
                kn = a.ckey[pn];
                fn = a.cposf[pn];
            }
            bool in_r = false, in_a = false;
            if (p >= 0 && (k & 0x3FFFFFFFu) != self) {
                float dx = pfj.x - pfi.x, dy = pfj.y - pfi.y, dz = pfj.z - pfi.z;
                minimg(a.bf, dx, dy, dz);
                const float d2f = dx * dx + dy * dy + dz * dz;
                if (d2f < a.cut_r2f_hi) {
                    if (d2f < a.cut_r2f_lo && (d2f < a.cut_a2f_lo || d2f >= a.cut_a2f_hi)) {
                        in_r = true;
                        in_a = d2f < a.cut_a2f_lo;
                    } else {   // near a cutoff: the exact FP64 test decides
                        const double4 pj = a.pos[a.cell_atoms[p]];
                        const double d2 = exact_d2(pi.x, pi.y, pi.z, pj.x, pj.y, pj.z, a.bd, a.g.per);
                        in_r = d2 < a.cut_r2;
                        in_a = d2 < a.cut_a2;
                    }
                }
            }
            const unsigned mr = __ballot_sync(0xffffffffu, in_r);
            const unsigned ma = __ballot_sync(0xffffffffu, in_a);
            if (in_r) {
                const int pos = m + __popc(mr & lt);
                // segment (angular? 0 : 2) + species of j in bits 30-31 above the caller index;
                // species is 0 or 1, so (seg << 30) fits with the caller index below 2^30
                const uint32_t sg = (in_a ? 0u : 2u) + (k >> 30);
                if (pos < SORT_MAX) key[pos] = (sg << 30) | (k & 0x3FFFFFFFu);
            }
            m += __popc(mr);
            nang += __popc(ma);
        }
        const bool overflow = m > a.cap || nang > a.cap_ang;
        const int mm = min(m, SORT_MAX);
        __syncwarp();
        if (mm <= 64) sort_and_store<2>(key, mm, lane, key);
        else if (mm <= 128) sort_and_store<4>(key, mm, lane, key);
        else sort_and_store<8>(key, mm, lane, key);
        const int cnt = min(mm, a.cap);
        int ends[4] = {0, 0, 0, 0};
        for (int s0 = 0; s0 < cnt; s0 += 32) {
            const int s = s0 + lane;
            unsigned sg = 4u;
            if (s < cnt) {
                const uint32_t k = key[s];
                sg = k >> 30;
                a.nbr[i * a.capr + s] = a.inv[k & 0x3FFFFFFFu];
                a.nbr_orig[i * a.capr + s] = (int32_t)(k & 0x3FFFFFFFu);   // atom-major: one row per atom
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) ends[t] += __popc(__ballot_sync(0xffffffffu, sg <= (unsigned)t));
        }
        if (lane == 0) {
            a.seg[i] = make_int4(ends[0], ends[1], ends[2], ends[3]);
            if (overflow) atomicOr(a.status, ST_NBR_OVERFLOW);
        }
        __syncwarp();
    }
}

// Slot of caller index oi inside [lo, hi) of the atom-major list row `row` (16-byte aligned),
// or -1.  The segment is read with independent 16-byte loads, 32 entries per round (a binary
// search needs one memory round trip per halving); the entries of a sorted segment are
// distinct, so at most one matches.  `first` holds the first round's 32 entries from
// lo & ~3, already loaded by the caller.
__device__ __forceinline__ int match_round(const int4 (&v)[8], int b, int lo, int hi, int oi) {
    int found = -1;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int k = b + 4 * u + c;
            if (e[c] == oi && k >= lo && k < hi) found = k;
        }
    }
    return found;
}
__device__ __forceinline__ void load_round(const int32_t *__restrict__ row, int b, int hi, int4 (&v)[8]) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
        v[u] = b + 4 * u < hi ? *reinterpret_cast<const int4 *>(row + b + 4 * u) : make_int4(-1, -1, -1, -1);
}
__device__ __forceinline__ int find_rest(const int32_t *__restrict__ row, int b, int lo, int hi, int oi) {
    int found = -1;
    for (; b < hi && found < 0; b += 32) {
        int4 v[8];
        load_round(row, b, hi, v);
        found = match_round(v, b, lo, hi, oi);
    }
    return found;
}

// Warp per atom, lanes over slots: for every list entry j = nbr[i][s] with j > i, the slot t
// of i in the list of j is found and both reverse slots are written, rev[i][s] = t and
// rev[j][t] = s (the entries with j < i are written by j's warp): one search per unordered
// pair.  The lists are symmetric and so is each pair's segment kind (the cutoff test gives the
// same result for (i, j) and (j, i)), so i sits in the segment of j's list for (kind of slot
// s, t_i).  Each lane takes four slots 32 apart: their list entries, then their neighbours'
// segment bounds, then two first search rounds at a time are in flight together.  A pair
// found in one list only (a list cut at its capacity) raises the overflow status.
__device__ __forceinline__ void rev_body(const RevArgs &args, int64_t blk, int64_t nblk) {
    const RevArgs a = args;   // as values: the stores below cannot make the compiler re-read them
    if (a.flag && *a.flag == 0) return;
    const int lane = threadIdx.x & 31;
    for (int64_t i = blk * 4 + (threadIdx.x >> 5); i < a.n; i += nblk * 4) {
        const int4 sg = a.seg[i];
        const int oi = a.orig[i];
        const int ti = a.species[i];
        for (int s0 = 0; s0 < sg.w; s0 += 128) {
            int j[4];
            int4 sj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int s = s0 + lane + 32 * u;
                const int jj = s < sg.w ? a.nbr[i * a.capr + s] : -1;
                j[u] = jj > i ? jj : -1;   // the lower-indexed atom of the pair searches
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) sj[u] = j[u] >= 0 ? a.seg[j[u]] : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 4; u += 2) {
                int lo[2], hi[2], b[2];
                int4 v[2][8];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int s = s0 + lane + 32 * (u + h);
                    const int sgi = (s < sg.y ? 0 : 2) + ti;
                    const int e[4] = {sj[u + h].x, sj[u + h].y, sj[u + h].z, sj[u + h].w};
                    lo[h] = sgi == 0 ? 0 : e[sgi - 1];
                    hi[h] = j[u + h] >= 0 ? e[sgi] : 0;
                    b[h] = lo[h] & ~3;
                    load_round(a.nbr_orig + (int64_t)max(j[u + h], 0) * a.capr, b[h], hi[h], v[h]);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (j[u + h] < 0) continue;
                    const int s = s0 + lane + 32 * (u + h);
                    int found = match_round(v[h], b[h], lo[h], hi[h], oi);
                    if (found < 0 && b[h] + 32 < hi[h])
                        found = find_rest(a.nbr_orig + (int64_t)j[u + h] * a.capr, b[h] + 32, lo[h], hi[h], oi);
                    if (found < 0) {
                        atomicOr(a.status, ST_NBR_OVERFLOW);
                        a.rev[i * a.capr + s] = 0;
                        continue;
                    }
                    a.rev[i * a.capr + s] = (uint8_t)found;
                    a.rev[(int64_t)j[u + h] * a.capr + found] = (uint8_t)s;
                }
            }
        }
    }
}

__device__ __forceinline__ void finish_body(const BinArgs &r, int64_t blk, int64_t nblk) {
    if (r.flag && *r.flag == 0) return;
    const int64_t m = r.n > r.ncell ? r.n : r.ncell;
    for (int64_t i = blk * (int64_t)blockDim.x + threadIdx.x; i < m; i += nblk * blockDim.x) {
        if (i < r.n) r.posref[i] = r.pos[i];
        if (i < r.ncell) { r.count[i] = 0; r.fill[i] = 0; }
    }
    if (blk == 0 && threadIdx.x == 0) *r.builds += 1ULL;
    // the flag itself is cleared by the last kernel of the group, after everything that reads it
}

// The group over an argument table (sl_batch.h: a system's own table or a batch's), one
// launch per kernel.  LOOP: a batch's persistent grid walks the work map, passing over a slot
// with no rebuild due as a whole; otherwise (a system's own launch, whose grid is its block
// count) one item per block, which keeps the loop's state out of the latency-bound bodies'
// registers.  The lists do not depend on the form: integer work, an FP32 pre-test that decides
// only far from the cutoffs, and an FP64 test in explicitly rounded operations.
// quick (a system's own conditional launch: its rebuild flag): return at once, before any
// table lookup, when no rebuild is due.
template <typename A>
__device__ __forceinline__ bool no_rebuild(const A &a) { return a.flag && *a.flag == 0; }

template <bool LOOP, typename A, typename Body>
__device__ __forceinline__ void rebuild_items(const A *__restrict__ tab, const WorkMap &m, Body body) {
    if constexpr (LOOP) for_each_work_unless(tab, m, no_rebuild<A>, body);
    else map_item(tab, m, body);
}

// register budget of a system's own list build: the latency-bound walk wants occupancy
#ifndef LISTS_MINB
#define LISTS_MINB 8
#endif

template <bool LOOP>
__global__ void k_bin(const BinArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    rebuild_items<LOOP>(tab, m, [](const BinArgs &r, int64_t blk, int64_t nblk) { bin_body(r, blk, nblk); });
}
template <bool LOOP>
__global__ void k_scan(const BinArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    __shared__ int s_part[1024];
    __shared__ int s_carry;
    rebuild_items<LOOP>(tab, m, [&](const BinArgs &r, int64_t, int64_t) { scan_body(r, s_part, s_carry); });
}
template <bool LOOP>
__global__ void k_scatter(const BinArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    rebuild_items<LOOP>(tab, m, [](const BinArgs &r, int64_t blk, int64_t nblk) { scatter_body(r, blk, nblk); });
}
template <bool LOOP>
__global__ void __launch_bounds__(LB_WARPS * 32, LOOP ? 4 : LISTS_MINB) k_lists(const ListArgs *__restrict__ tab,
                                                                              WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    __shared__ ListSmem sm;
    rebuild_items<LOOP>(tab, m, [&](const ListArgs &a, int64_t blk, int64_t nblk) { lists_body(a, blk, nblk, sm); });
}
template <bool LOOP>
__global__ void __launch_bounds__(128) k_rev(const RevArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    rebuild_items<LOOP>(tab, m, [](const RevArgs &a, int64_t blk, int64_t nblk) { rev_body(a, blk, nblk); });
}
template <bool LOOP>
__global__ void k_finish(const BinArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    rebuild_items<LOOP>(tab, m, [](const BinArgs &r, int64_t blk, int64_t nblk) { finish_body(r, blk, nblk); });
}
// clears the rebuild flag of every slot with a conditional rebuild in the launch (after the
// whole group has read it); m is the binning kernel's map, in which every such slot has blocks
__global__ void k_clear_flags(const BinArgs *__restrict__ tab, WorkMap m) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m.nrep; r += gridDim.x * blockDim.x)
        if (m.w0[r + 1] > m.w0[r] && tab[r].flag) *tab[r].rebuild = 0;
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void nbr_setup(Sys &s) {
    const double cut = s.pd.rc_r + s.skin;
    for (int a = 0; a < 3; ++a) {
        int nc = (int)floor(s.box[a] / (cut * (1.0 + 1e-9)));
        s.cells.nc[a] = nc < 1 ? 1 : nc;
    }
    s.cells.ncell = s.cells.nc[0] * s.cells.nc[1] * s.cells.nc[2];
}

// The rebuild group's argument blocks of system s and each kernel's block count for it.
RebuildPlan rebuild_plan(Sys &s, bool conditional) {
    RebuildPlan pl;
    const int *flag = conditional ? s.rebuild : nullptr;
    GridArgs g;
    for (int a = 0; a < 3; ++a) {
        g.nc[a] = s.cells.nc[a];
        g.w[a] = s.box[a] / s.cells.nc[a];
        g.per[a] = s.per[a];
    }
    const int64_t n = s.n;
    BinArgs &r = pl.bin;
    r.pos = s.pos; r.posf = s.posf; r.species = s.species; r.orig = s.orig; r.n = n; r.g = g;
    r.ncell = s.cells.ncell; r.count = s.cells.count; r.start = s.cells.start; r.fill = s.cells.fill;
    r.atoms = s.cells.atoms; r.of = s.cells.of; r.cposf = s.cells.posf; r.ckey = s.cells.key;
    r.posref = s.posref; r.builds = s.d_builds; r.rebuild = s.rebuild; r.flag = flag;
    ListArgs &la = pl.lists;
    la.pos = s.pos; la.posf = s.posf; la.species = s.species; la.orig = s.orig; la.inv = s.inv;
    la.cell_start = s.cells.start; la.cell_atoms = s.cells.atoms; la.cell_of = s.cells.of;
    la.cposf = s.cells.posf; la.ckey = s.cells.key; la.nbr_orig = s.nbr_orig;
    la.n = n; la.cap = s.cap; la.cap_ang = s.cap_ang; la.capr = nbr_orig_stride(s.cap);
    la.cut_r2 = s.cut_r2; la.cut_a2 = s.cut_a2;
    // FP32 separations of positions below 1e4 A carry an absolute d2 error far
    // below 0.05 A^2 at these distances; pairs inside that band take the FP64 test.
    la.cut_r2f_lo = (float)(s.cut_r2 - 0.05); la.cut_r2f_hi = (float)(s.cut_r2 + 0.05);
    la.cut_a2f_lo = (float)(s.cut_a2 - 0.05); la.cut_a2f_hi = (float)(s.cut_a2 + 0.05);
    la.bd = s.boxd; la.bf = s.boxf; la.g = g;
    la.nbr = s.nbr; la.seg = s.seg; la.status = s.status; la.flag = flag;
    RevArgs &ra = pl.rev;
    ra.species = s.species; ra.orig = s.orig; ra.nbr = s.nbr; ra.nbr_orig = s.nbr_orig; ra.seg = s.seg;
    ra.n = n; ra.cap = s.cap; ra.capr = nbr_orig_stride(s.cap);
    ra.rev = s.rev; ra.status = s.status; ra.flag = flag;
    // grids are capped (grid-stride loops): when no rebuild is due every kernel returns at once
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto capped = [&](int64_t items, int per_block) -> int64_t {
        const int64_t b = (items + per_block - 1) / per_block;
        return b < (int64_t)sms * 16 ? (b > 0 ? b : 1) : (int64_t)sms * 16;
    };
    const int64_t m = n > s.cells.ncell ? n : s.cells.ncell;
    pl.blocks[RB_BIN] = capped(n, RB_THREADS);
    pl.blocks[RB_SCAN] = 1;
    pl.blocks[RB_SCATTER] = capped(n, RB_THREADS);
    pl.blocks[RB_LISTS] = capped(n, LB_WARPS);
    pl.blocks[RB_REV] = capped(n, 4);
    pl.blocks[RB_FINISH] = capped(m, RB_THREADS);
    return pl;
}

// The system's own rebuild group: conditional (a step's, on the flag the first half raised;
// the flag is cleared afterwards) or unconditional.
void launch_rebuild(Sys &s, bool conditional) {
    const int kind = conditional ? SK_STEP : SK_FULL;
    Launch L[RB_KERNELS];
    for (int k = 0; k < RB_KERNELS; ++k) L[k] = solo_launch(s, FK_BIN + k, kind);
    launch_rebuild_t(s.solo->t, L, conditional, false, s.stream);
}

// ---- argument tables (sl_batch.h)
void fused_put_rebuild(Sys &s, int r, int kind, const FusedTables &t, unsigned char *img, int64_t *blocks) {
    const RebuildPlan pl = rebuild_plan(s, kind != SK_FULL);
    reinterpret_cast<BinArgs *>(img + t.o_bin)[r] = pl.bin;
    reinterpret_cast<ListArgs *>(img + t.o_lists)[r] = pl.lists;
    reinterpret_cast<RevArgs *>(img + t.o_rev)[r] = pl.rev;
    for (int k = 0; k < RB_KERNELS; ++k) blocks[FK_BIN + k] = pl.blocks[k];
}

// persistent grids: every SM filled to the kernel's occupancy (the scan: one block per slot)
void fused_grids_rebuild(FusedTables &t) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto full = [&](const void *fn, int threads) -> unsigned {
        int per = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0) != cudaSuccess || per < 1) per = 1;
        return (unsigned)(sms * per);
    };
    t.grid[FK_BIN] = full((const void *)k_bin<true>, RB_THREADS);
    t.grid[FK_SCAN] = std::min<unsigned>((unsigned)t.cap, full((const void *)k_scan<true>, 1024));
    t.grid[FK_SCATTER] = full((const void *)k_scatter<true>, RB_THREADS);
    t.grid[FK_LISTS] = full((const void *)k_lists<true>, LB_WARPS * 32);
    t.grid[FK_REV] = full((const void *)k_rev<true>, 128);
    t.grid[FK_FINISH] = full((const void *)k_finish<true>, RB_THREADS);
}

template <bool LOOP>
static void rebuild_t(const FusedTables &t, const Launch *L, bool clear, cudaStream_t st) {
    const BinArgs *bin = t.at<BinArgs>(t.o_bin);
    k_bin<LOOP><<<L[RB_BIN].grid, RB_THREADS, 0, st>>>(bin, L[RB_BIN].m, L[RB_BIN].quick);
    k_scan<LOOP><<<L[RB_SCAN].grid, 1024, 0, st>>>(bin, L[RB_SCAN].m, L[RB_SCAN].quick);
    k_scatter<LOOP><<<L[RB_SCATTER].grid, RB_THREADS, 0, st>>>(bin, L[RB_SCATTER].m, L[RB_SCATTER].quick);
    k_lists<LOOP><<<L[RB_LISTS].grid, LB_WARPS * 32, 0, st>>>(t.at<ListArgs>(t.o_lists), L[RB_LISTS].m,
                                                              L[RB_LISTS].quick);
    k_rev<LOOP><<<L[RB_REV].grid, 128, 0, st>>>(t.at<RevArgs>(t.o_rev), L[RB_REV].m, L[RB_REV].quick);
    k_finish<LOOP><<<L[RB_FINISH].grid, RB_THREADS, 0, st>>>(bin, L[RB_FINISH].m, L[RB_FINISH].quick);
    if (clear) k_clear_flags<<<1, 128, 0, st>>>(bin, L[RB_BIN].m);
}
void launch_rebuild_t(const FusedTables &t, const Launch *L, bool clear, bool loop, cudaStream_t st) {
    if (loop) rebuild_t<true>(t, L, clear, st);
    else rebuild_t<false>(t, L, clear, st);
}

}  // namespace sl
