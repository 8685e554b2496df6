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
// 0 and 1 -- and each segment is in the order of the list build's walk (the half-width
// sub-cells around the atom z-major, or the whole stencil's cells z-major in a box with
// fewer than 3 cells along a periodic axis; each sub-cell's or cell's atoms by species,
// then caller index), so every per-atom sum runs in an order set by the positions and caller indices
// alone, never by the internal atom order.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "sl_internal.h"
#include "sl_batch.h"
#include "sl_fused.cuh"
#include "sl_rebuild.cuh"

namespace sl {

namespace {

// The list definition's d2.  |t| <= L/2 gives |t/L| <= 1/2, so the rounded quotient lies in
// [-1/2, 1/2] and rint (ties to even) returns a zero: t is then left as it is, without the
// division, and the result (up to the sign of a zero, which squaring removes) is the same.
__device__ __forceinline__ double exact_d2(double xi, double yi, double zi, double xj, double yj, double zj,
                                           const BoxDev<double> &b, const int per[3]) {
    double t[3] = {__dsub_rn(xj, xi), __dsub_rn(yj, yi), __dsub_rn(zj, zi)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (per[a] && fabs(t[a]) > 0.5 * b.L[a]) {
            const double q = rint(__ddiv_rn(t[a], b.L[a]));
            t[a] = __dsub_rn(t[a], __dmul_rn(b.L[a], q));
        }
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(t[0], t[0]), __dmul_rn(t[1], t[1])), __dmul_rn(t[2], t[2]));
}

// Cell of each atom and its half-width sub-cell inside it (bit 0 x, 1 y, 2 z): the sub-cell
// index along an axis is floor(x * 2/w) clamped to [0, 2 nc), and the cell is half of it.  A
// position within a rounding of a boundary may land on either side; the cells are at least
// (1 + 1e-9) times the list cutoff wide, far more than that, so the stencil still holds every
// pair.
__device__ __forceinline__ void bin_body(const BinArgs &r, int64_t blk, int64_t nblk) {
    if (r.flag && *r.flag == 0) return;
    const GridArgs &g = r.g;
    for (int64_t i = blk * (int64_t)blockDim.x + threadIdx.x; i < r.n; i += nblk * blockDim.x) {
        const double4 p = r.pos[i];
        const double x[3] = {p.x, p.y, p.z};
        int c[3], sb = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // the conversion saturates, so far outside positions clamp too
            const int hi = min(max((int)floor(x[a] * g.inv2w[a]), 0), 2 * g.nc[a] - 1);
            c[a] = hi >> 1;
            sb |= (hi & 1) << a;
        }
        const int cell = (c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0];
        r.of[i] = (cell << 3) | sb;
        atomicAdd(r.count + cell, 1);
    }
}

// Exclusive scan of count[0..m) into start[0..m] by one whole block (s_part: 32 ints): warp w
// takes the w-th contiguous chunk (a multiple of 32 cells) and reads it 32 cells at a time,
// coalesced, twice: once for its total, then, after the warps' totals are scanned through
// shared memory, for the starts it writes (a shuffle scan per 32 cells with a running carry).
__device__ __forceinline__ void scan_body(const BinArgs &r, int *s_part) {
    if (r.flag && *r.flag == 0) return;
    const int *__restrict__ count = r.count;
    int *__restrict__ start = r.start;
    const int m = r.ncell, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int chunk = ((m + nw - 1) / nw + 31) & ~31;
    const int b0 = min(wid * chunk, m), b1 = min(b0 + chunk, m);
    int sum = 0;
    for (int k = b0 + lane; k < b1; k += 32) sum += count[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) s_part[wid] = sum;
    __syncthreads();
    if (wid == 0) {
        int v = lane < nw ? s_part[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane < nw) s_part[lane] = v;   // inclusive warp totals
    }
    __syncthreads();
    int carry = wid > 0 ? s_part[wid - 1] : 0;
    for (int k0 = b0; k0 < b1; k0 += 32) {
        const int k = k0 + lane;
        const int c = k < b1 ? count[k] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (k < b1) start[k] = carry + incl - c;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (threadIdx.x == 0) start[m] = s_part[nw - 1];
    __syncthreads();   // the block's next work item reuses s_part
}

// Atoms into their cells, with a cell-ordered copy of the key (species << 30 | caller index)
// and of the position relative to the cell's corner in FP32 (NaN for an atom more than a
// cell width outside its cell, which only a non-periodic axis can hold); w carries the
// species (bit 0) and the sub-cell (bits 1-3) as integer bits.  The list build reads the
// candidates contiguously.
__device__ __forceinline__ void scatter_body(const BinArgs &r, int64_t blk, int64_t nblk) {
    if (r.flag && *r.flag == 0) return;
    const GridArgs &g = r.g;
    for (int64_t i = blk * (int64_t)blockDim.x + threadIdx.x; i < r.n; i += nblk * blockDim.x) {
        const int cs = r.of[i], c = cs >> 3;
        const int p = r.start[c] + atomicAdd(r.fill + c, 1);
        const double4 x = r.pos[i];
        const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
        const double u[3] = {x.x - cx * g.w[0], x.y - cy * g.w[1], x.z - cz * g.w[2]};
        bool near = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) near = near && u[d] >= -g.w[d] && u[d] <= 2.0 * g.w[d];
        r.atoms[p] = (int)i;
        const float tag = __int_as_float(r.species[i] | ((cs & 7) << 1));
        r.cposf[p] = near ? make_float4((float)u[0], (float)u[1], (float)u[2], tag)
                          : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, tag);
        r.ckey[p] = ((uint32_t)r.species[i] << 30) | (uint32_t)r.orig[i];
    }
}

// Ascending bitonic sort of 32*E 64-bit keys held E per lane (element r*32 + lane in
// register r): strides below 32 exchange through shuffles, larger ones inside the lane.
template <int E>
__device__ __forceinline__ void warp_bitonic64(uint64_t (&k)[E], int lane) {
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
                        const uint64_t u = k[r], v = k[rp];
                        const bool sw = (u > v) == asc;
                        k[r] = sw ? v : u;
                        k[rp] = sw ? u : v;
                    }
                } else {
                    const uint64_t v = __shfl_xor_sync(0xffffffffu, k[r], stride);
                    const bool lower = (lane & stride) == 0;
                    k[r] = (lower == asc) ? min(k[r], v) : max(k[r], v);
                }
            }
        }
    }
}

__device__ __forceinline__ int sub_of(const float4 &pf) { return (__float_as_int(pf.w) >> 1) & 7; }

// One cell of up to 32 E atoms sorted in registers (E per lane), its sub-cell starts recorded.
template <int E>
__device__ __forceinline__ void cellsort_regs(const BinArgs &r, int64_t c, int p0, int len, int lane) {
    // (sub-cell << 61) | (key << 29) | element: distinct, so the order is unique
    uint64_t v[E];
    int at[E];
    float4 pf[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int e = q * 32 + lane;
        v[q] = ~0ull;
        at[q] = 0;
        pf[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < len) {
            at[q] = r.atoms[p0 + e];
            pf[q] = r.cposf[p0 + e];
            v[q] = ((uint64_t)sub_of(pf[q]) << 61) | ((uint64_t)r.ckey[p0 + e] << 29) | (uint64_t)e;
        }
    }
    warp_bitonic64<E>(v, lane);
    int below[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // sorted elements of a sub-cell below k
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int e = q * 32 + lane;
        const int src = (int)(v[q] & 63u), sl = src & 31, sq = src >> 5;
        int an = 0;
        float4 fn = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < E; ++u) {   // element src sits in register sq of lane sl
            const int a = __shfl_sync(0xffffffffu, at[u], sl);
            float4 f;
            f.x = __shfl_sync(0xffffffffu, pf[u].x, sl);
            f.y = __shfl_sync(0xffffffffu, pf[u].y, sl);
            f.z = __shfl_sync(0xffffffffu, pf[u].z, sl);
            f.w = __shfl_sync(0xffffffffu, pf[u].w, sl);
            if (sq == u) {
                an = a;
                fn = f;
            }
        }
        const int sub = e < len ? (int)(v[q] >> 61) : 8;
#pragma unroll
        for (int k = 1; k < 8; ++k) below[k] += __popc(__ballot_sync(0xffffffffu, sub < k));
        if (e < len) {
            r.ckey[p0 + e] = (uint32_t)(v[q] >> 29);
            r.atoms[p0 + e] = an;
            r.cposf[p0 + e] = fn;
        }
    }
    if (lane < 8) {
        int mine = 0;
#pragma unroll
        for (int k = 1; k < 8; ++k) mine = lane == k ? below[k] : mine;
        r.sub[c * 8 + lane] = mine;
    }
}

// Each cell's atoms in ascending (sub-cell, key) order (key: species << 30 | caller index),
// one warp per cell, and the first position of each sub-cell relative to the cell's start:
// the scatter fills a cell in the order of its atomic increments, and the list build walks
// the cells' atoms in their stored order, so sorted cells make every list independent of that
// order and of the internal atom order.  Cells of up to 32 or 64 atoms are sorted in registers; a
// larger one (only in boxes of very few cells) by lane 0 in place.
__device__ __forceinline__ void cellsort_body(const BinArgs &r, int64_t blk, int64_t nblk) {
    if (r.flag && *r.flag == 0) return;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t c = blk * wpb + (threadIdx.x >> 5); c < r.ncell; c += nblk * wpb) {
        const int p0 = r.start[c], len = r.start[c + 1] - p0;
        if (len <= 32) {
            cellsort_regs<1>(r, c, p0, len, lane);
        } else if (len <= 64) {
            cellsort_regs<2>(r, c, p0, len, lane);
        } else if (lane == 0) {
            auto before = [&](int s1, uint32_t k1, int s2, uint32_t k2) { return s1 < s2 || (s1 == s2 && k1 < k2); };
            for (int x = 1; x < len; ++x) {
                const uint32_t k = r.ckey[p0 + x];
                const int at = r.atoms[p0 + x];
                const float4 pf = r.cposf[p0 + x];
                int y = x - 1;
                for (; y >= 0 && before(sub_of(pf), k, sub_of(r.cposf[p0 + y]), r.ckey[p0 + y]); --y) {
                    r.ckey[p0 + y + 1] = r.ckey[p0 + y];
                    r.atoms[p0 + y + 1] = r.atoms[p0 + y];
                    r.cposf[p0 + y + 1] = r.cposf[p0 + y];
                }
                r.ckey[p0 + y + 1] = k;
                r.atoms[p0 + y + 1] = at;
                r.cposf[p0 + y + 1] = pf;
            }
            int k = 0;
            for (int e = 0; e < len; ++e)
                for (const int s = sub_of(r.cposf[p0 + e]); k <= s; ++k) r.sub[c * 8 + k] = e;
            for (; k < 8; ++k) r.sub[c * 8 + k] = len;
        }
        __syncwarp();
    }
}

// The lists are built cell by cell: a block takes one cell, copies the candidates of its
// stencil (the 27 surrounding cells, each cell's atoms contiguous and sorted by sub-cell and
// key) into shared memory once, and its warps build the lists of the cell's atoms from there,
// one atom per warp: lanes take the candidates 32 at a time, pairs inside the list cutoff are
// appended to a per-warp buffer in walk order (ballot/popc), and the buffer is written out
// partitioned by segment, each segment in walk order.
//
// With at least 3 cells along every periodic axis an atom walks only the 5 x 5 x 5 half-width
// sub-cells around its own (a neighbour within the cutoff, at most two sub-cell widths away,
// lies in one of them: about 58% of the 27 cells' candidates): the block lists the staged
// indices of that walk once for each of the 8 sub-cell positions in the centre cell, sub-cells
// z-major, each by key.  Otherwise the walk is the whole stencil (lo..hi per axis, z-major,
// each cell by sub-cell and key).  Either order depends on the positions and caller indices
// only.
//
// FP32 pre-test.  The scatter stores each atom's position relative to its own cell's corner
// (FP64 difference, then rounded), so the FP32 separation of a pair is the difference of two
// numbers below two cell widths plus the stencil cell's corner offset (a whole number of cell
// widths, which with at least 3 cells along every periodic axis already carries the periodic
// image; with fewer the minimum image is taken in FP32).  Its error is a few FP32 roundings
// of a cell width, independent of the box size, and the host sets the band around each cutoff
// from that bound (rebuild_plan); pairs inside the band, and any pair with an atom more than a
// cell width outside its cell (stored as NaN, which fails every comparison), take the exact
// FP64 test.

__device__ __forceinline__ int wrap_cell(int x, int nc) { return x < 0 ? x + nc : (x >= nc ? x - nc : x); }

// 8-bit hash of an atom index, stored beside each list entry so that the reverse-slot search
// reads one byte per entry: the low byte (a row's entries are atoms near each other in the
// Morton-ordered internal order, so their low bytes seldom coincide)
__device__ __forceinline__ uint32_t index_hash8(int x) { return (uint32_t)x & 0xFFu; }

constexpr int SORT_MAX = 256;
constexpr int STAGE_MAX = 1024;   // staged candidates; a larger stencil is walked in global memory
constexpr int WALK_MAX = 640;     // a sub-cell walk's staged indices (a longer one takes the whole stencil)

struct ListSmem {
    // FP32 positions of the stencil's candidates relative to the centre cell's corner, with the
    // species and sub-cell bits in w; padded past the end with candidates far away
    float4 p[STAGE_MAX];
    int j[STAGE_MAX];         // their internal indices
    uint32_t key[LB_WARPS][SORT_MAX];
    uint16_t walk[8][WALK_MAX];   // per sub-cell position of the centre cell: its walk's staged indices
    int wlen[8];
    int off[32], p0[32];      // stencil cells: offset in the walk, first cell-ordered position
    int soff[27][9];          // stencil cells (27-cell form): sub-cell starts relative to the cell, and its size
    float4 org[32];           // stencil cells: corner relative to the centre cell's corner (its image)
    int nst, total, self0;    // self0: walk offset of the centre cell
};

// One atom's list from its walk fw = 0 .. nwalk-1 over the staged or stencil candidates
// (total of them; fself: the atom's own candidate index).  pfi: the atom's FP32 position
// relative to its cell's corner; cand(fw, f) gives walk step fw's candidate index f (f >= total:
// none) and FP32 position relative to the same corner with the species in bit 0 of w, and
// jof(f) its internal index (the exact test and the list entry).  The FP32 decision is branch-free; a warp takes the exact test's branch only
// when one of its lanes is in a band.
template <typename Cand, typename Jof>
__device__ __forceinline__ void list_atom(const ListArgs &a, int64_t i, float4 pfi, int fself, uint32_t *key,
                                          int lane, int nwalk, int total, bool image_placed, Cand cand, Jof jof) {
    const unsigned lt = (1u << lane) - 1u;
    int m = 0;
    auto classify = [&](int f, const float4 &pj, bool &in_r, bool &in_a, bool &near) {
        float dx = pj.x - pfi.x, dy = pj.y - pfi.y, dz = pj.z - pfi.z;
        if (!image_placed) minimg(a.bf, dx, dy, dz);
        const float d2f = dx * dx + dy * dy + dz * dz;
        const bool other = f != fself && f < total;   // a real candidate, not the atom itself
        in_r = d2f < a.cut_r2f_lo && other;
        in_a = d2f < a.cut_a2f_lo;
        // inside a band, or NaN (an atom far outside its cell): the exact FP64 test decides
        near = other && !(d2f >= a.cut_r2f_hi) && !(d2f < a.cut_r2f_lo && (d2f < a.cut_a2f_lo || d2f >= a.cut_a2f_hi));
    };
    auto exact = [&](int f, bool &in_r, bool &in_a) {
        const double4 qi = a.pos[i], qj = a.pos[jof(f)];
        const double d2 = exact_d2(qi.x, qi.y, qi.z, qj.x, qj.y, qj.z, a.bd, a.g.per);
        in_r = d2 < a.cut_r2;
        in_a = d2 < a.cut_a2;
    };
    auto append = [&](int f, const float4 &pj, bool in_r, bool in_a) {
        const unsigned mr = __ballot_sync(0xffffffffu, in_r);
        const int pos = m + __popc(mr & lt);
        // segment (angular? 0 : 2) + species of j in bits 30-31 above the candidate index
        if (in_r && pos < SORT_MAX)
            key[pos] = (((in_a ? 0u : 2u) + ((uint32_t)__float_as_int(pj.w) & 1u)) << 30) | (uint32_t)f;
        m += __popc(mr);
    };
    for (int base = 0; base < nwalk; base += 64) {   // two chunks of 32 candidates at a time
        int f0, f1;
        float4 p0, p1;
        cand(base + lane, f0, p0);
        cand(base + 32 + lane, f1, p1);
        bool r0, a0, n0, r1, a1, n1;
        classify(f0, p0, r0, a0, n0);
        classify(f1, p1, r1, a1, n1);
        if (__any_sync(0xffffffffu, n0 || n1)) {
            if (n0) exact(f0, r0, a0);
            if (n1) exact(f1, r1, a1);
        }
        append(f0, p0, r0, a0);
        append(f1, p1, r1, a1);
    }
    const int mm = min(m, SORT_MAX);
    __syncwarp();
    // entries per segment, then each segment's entries in walk order from its offset (a stable
    // partition); an overflowing list keeps its first `cap` entries and raises the status
    int cnt4[4] = {0, 0, 0, 0};
    for (int s0 = 0; s0 < mm; s0 += 32) {
        const int e = s0 + lane;
        const unsigned sg = e < mm ? key[e] >> 30 : 4u;
#pragma unroll
        for (int t = 0; t < 4; ++t) cnt4[t] += __popc(__ballot_sync(0xffffffffu, sg == (unsigned)t));
    }
    const bool overflow = m > a.cap || cnt4[0] + cnt4[1] > a.cap_ang;
    int run[4] = {0, cnt4[0], cnt4[0] + cnt4[1], cnt4[0] + cnt4[1] + cnt4[2]};
    const int ends_all[4] = {run[1], run[2], run[3], run[3] + cnt4[3]};
    for (int s0 = 0; s0 < mm; s0 += 32) {
        const int e = s0 + lane;
        const uint32_t k = e < mm ? key[e] : 0u;
        const unsigned sg = e < mm ? k >> 30 : 4u;
        int pos = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const unsigned b = __ballot_sync(0xffffffffu, sg == (unsigned)t);
            if (sg == (unsigned)t) pos = run[t] + __popc(b & lt);
            run[t] += __popc(b);
        }
        if (e < mm && pos < a.cap) {
            const int jx = jof((int)(k & 0x3FFFFFFFu));
            a.nbr[i * a.capr + pos] = jx;   // atom-major rows
            a.hash[i * a.capr + pos] = (uint8_t)index_hash8(jx);
        }
    }
    if (lane == 0) {
        a.seg[i] = make_int4(min(ends_all[0], a.cap), min(ends_all[1], a.cap), min(ends_all[2], a.cap),
                             min(ends_all[3], a.cap));
        if (overflow) atomicOr(a.status, ST_NBR_OVERFLOW);
    }
    __syncwarp();
}

// Cells blk, blk + nblk, ... of the grid (a block-uniform loop).
__device__ __forceinline__ void lists_body(const ListArgs &args, int64_t blk, int64_t nblk, ListSmem &sm) {
    const ListArgs a = args;   // as values: the stores below cannot make the compiler re-read them
    if (a.flag && *a.flag == 0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ncell = a.g.nc[0] * a.g.nc[1] * a.g.nc[2];
    // with at least 3 cells along every periodic axis each stencil cell is one image, placed by
    // its corner offset, and the sub-cell walks apply; otherwise the walk takes the minimum image
    bool image_placed = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) image_placed = image_placed && (!a.g.per[d] || a.g.nc[d] >= 3);
    const float4 far = make_float4(1e30f, 1e30f, 1e30f, 0.f);
    for (int64_t c = blk; c < ncell; c += nblk) {
        // the stencil and each cell's offset in it (warp 0): the 27 cells around (an empty one
        // past a non-periodic face) when the images are placed, else lo..hi per axis, z-major
        if (w == 0) {
            const int ci[3] = {(int)(c % a.g.nc[0]), (int)((c / a.g.nc[0]) % a.g.nc[1]),
                               (int)(c / ((int64_t)a.g.nc[0] * a.g.nc[1]))};
            int lo[3], sx, sy, nst, centre;
            if (image_placed) {
                lo[0] = ci[0] - 1; lo[1] = ci[1] - 1; lo[2] = ci[2] - 1;
                sx = sy = 3;
                nst = 27;
                centre = 13;
            } else {
                int hi[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (a.g.per[d] && a.g.nc[d] < 3) { lo[d] = 0; hi[d] = a.g.nc[d] - 1; }
                    else if (a.g.per[d]) { lo[d] = ci[d] - 1; hi[d] = ci[d] + 1; }
                    else { lo[d] = max(ci[d] - 1, 0); hi[d] = min(ci[d] + 1, a.g.nc[d] - 1); }
                }
                sx = hi[0] - lo[0] + 1;
                sy = hi[1] - lo[1] + 1;
                nst = sx * sy * (hi[2] - lo[2] + 1);   // at most 27 cells
                centre = ((ci[2] - lo[2]) * sy + (ci[1] - lo[1])) * sx + (ci[0] - lo[0]);
            }
            int my_p0 = 0, my_len = 0;
            if (lane < nst) {
                const int x = lo[0] + lane % sx, y = lo[1] + (lane / sx) % sy, z = lo[2] + lane / (sx * sy);
                const int xyz[3] = {x, y, z};
                bool inside = true;   // false only past a non-periodic face
#pragma unroll
                for (int d = 0; d < 3; ++d) inside = inside && (a.g.per[d] || (xyz[d] >= 0 && xyz[d] < a.g.nc[d]));
                const int wx = wrap_cell(x, a.g.nc[0]), wy = wrap_cell(y, a.g.nc[1]), wz = wrap_cell(z, a.g.nc[2]);
                const int cc = (wz * a.g.nc[1] + wy) * a.g.nc[0] + wx;
                if (inside) {
                    my_p0 = a.cell_start[cc];
                    my_len = a.cell_start[cc + 1] - my_p0;
                }
                if (image_placed) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) sm.soff[lane][k] = inside ? a.cell_sub[(int64_t)cc * 8 + k] : 0;
                    sm.soff[lane][8] = my_len;
                }
                // x, y, z are unwrapped: a cell across a periodic face sits one box length away
                sm.org[lane] = make_float4((float)(x - ci[0]) * a.wf[0], (float)(y - ci[1]) * a.wf[1],
                                           (float)(z - ci[2]) * a.wf[2], 0.f);
            }
            int incl = my_len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane < nst) {
                sm.off[lane] = incl - my_len;
                sm.p0[lane] = my_p0;
            }
            if (lane == centre) sm.self0 = incl - my_len;
            if (lane == 31) {
                sm.total = incl;
                sm.nst = nst;
            }
        }
        __syncthreads();
        const int total = sm.total, nst = sm.nst, self0 = sm.self0;
        auto placed = [&](int cl, float4 pf) {
            const float4 o = sm.org[cl];
            pf.x += o.x; pf.y += o.y; pf.z += o.z;
            return pf;
        };
        // staged when the candidates and a far one after them fit
        const bool staged = ((total + 64) & ~63) <= STAGE_MAX;
        if (staged) {   // a warp per stencil cell, a lane per atom
            for (int cl = w; cl < nst; cl += LB_WARPS) {
                const int o = sm.off[cl], p0 = sm.p0[cl], len = (cl + 1 < nst ? sm.off[cl + 1] : total) - o;
                for (int e = lane; e < len; e += 32) {
                    sm.p[o + e] = placed(cl, a.cposf[p0 + e]);
                    sm.j[o + e] = a.cell_atoms[p0 + e];
                }
            }
            for (int f = total + threadIdx.x; f < ((total + 64) & ~63); f += blockDim.x) sm.p[f] = far;
        }
        // the sub-cell walks: for sub-cell position sb = (bz, by, bx) of the centre cell, the
        // sub-cells (X, Y, Z) in [b - 2, b + 2] per axis (in sub-cell units from the centre
        // cell's corner), z-major; sub-cell X lies in stencil cell X >> 1 (floor), half X & 1
        bool walks = staged && image_placed;
        if (walks) {
            for (int sb = w; sb < 8; sb += LB_WARPS) {
                const int bx = sb & 1, by = (sb >> 1) & 1, bz = sb >> 2;
                const int X = bx - 2 + lane % 5, Y = by - 2 + lane / 5;   // lanes 0..24: one z-layer
                int run = 0;
                for (int Z = bz - 2; Z <= bz + 2; ++Z) {
                    int start = 0, len = 0;
                    if (lane < 25) {
                        const int cl = (((Z >> 1) + 1) * 3 + ((Y >> 1) + 1)) * 3 + ((X >> 1) + 1);
                        const int h = ((Z & 1) << 2) | ((Y & 1) << 1) | (X & 1);
                        start = sm.off[cl] + sm.soff[cl][h];
                        len = sm.soff[cl][h + 1] - sm.soff[cl][h];
                    }
                    int incl = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += t;
                    }
                    const int o = run + incl - len;
                    for (int t = 0; t < len; ++t)
                        if (o + t < WALK_MAX) sm.walk[sb][o + t] = (uint16_t)(start + t);
                    run += __shfl_sync(0xffffffffu, incl, 31);
                }
                // padded to whole pairs of chunks with the far candidate at index total
                for (int t = run + lane; t < ((run + 63) & ~63) && t < WALK_MAX; t += 32) sm.walk[sb][t] = (uint16_t)total;
                if (lane == 0) sm.wlen[sb] = run;
            }
        }
        __syncthreads();
        if (walks) {
#pragma unroll
            for (int sb = 0; sb < 8; ++sb) walks = walks && ((sm.wlen[sb] + 63) & ~63) <= WALK_MAX;
        }
        // stencil cell of candidate f: the last one whose offset is <= f (empty cells share the
        // offset of the cell after them)
        auto cell_of = [&](int f) {
            int cl = 0;
            while (cl + 1 < nst && sm.off[cl + 1] <= f) ++cl;
            return cl;
        };
        // the cell's own atoms, one per warp
        const int c0 = a.cell_start[c], nc0 = a.cell_start[c + 1] - c0;
        for (int q = w; q < nc0; q += LB_WARPS) {
            const int64_t i = a.cell_atoms[c0 + q];
            const float4 pfi = a.cposf[c0 + q];
            auto jof = [&](int f) { return sm.j[f]; };
            if (walks) {
                const int sb = sub_of(pfi);
                const uint16_t *wk = sm.walk[sb];
                list_atom(
                    a, i, pfi, self0 + q, sm.key[w], lane, sm.wlen[sb], total, true,
                    [&](int fw, int &f, float4 &pf) {
                        f = wk[fw];
                        pf = sm.p[f];
                    },
                    jof);
            } else if (staged) {
                list_atom(
                    a, i, pfi, self0 + q, sm.key[w], lane, total, total, image_placed,
                    [&](int fw, int &f, float4 &pf) {
                        f = fw;
                        pf = sm.p[fw];
                    },
                    jof);
            } else {
                auto position_of = [&](int f) {
                    const int cl = cell_of(f);
                    return sm.p0[cl] + (f - sm.off[cl]);
                };
                list_atom(
                    a, i, pfi, self0 + q, sm.key[w], lane, total, total, image_placed,
                    [&](int fw, int &f, float4 &pf) {
                        f = fw;
                        if (fw >= total) {
                            pf = far;
                            return;
                        }
                        const int cl = cell_of(fw);
                        pf = placed(cl, a.cposf[sm.p0[cl] + (fw - sm.off[cl])]);
                    },
                    [&](int f) { return a.cell_atoms[position_of(f)]; });
            }
        }
        __syncthreads();   // the next cell reuses the staging
    }
}

// 32 bytes of a row at p (32-byte aligned) in one 256-bit load.
__device__ __forceinline__ void ld_v8u(const uint8_t *p, uint32_t *r) {
    asm("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "l"(p));
}

// Bit k (k = 0..3) set where byte k of x is zero.  Adding 0x7F to the low seven bits of a
// byte sets its top bit unless they are all zero (no carry leaves the byte); with the byte's
// own top bit that marks the nonzero bytes.  The four top bits are then gathered by one
// multiplication whose partial products fall on distinct bits.
__device__ __forceinline__ uint32_t zero_bytes4(uint32_t x) {
    const uint32_t hb = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);   // 0x80 in each zero byte
    return (((hb >> 7) * 0x00204081u) >> 21) & 0xFu;
}

// Slot of atom index ai in [lo, hi) of a list row, or -1.  The row's hash bytes are read from
// lo & ~31 in windows of 64 (two 32-byte loads), and the entries whose hash equals ai's are
// the candidates.  An atom appears at most once in a row's entries [0, seg.w), and when the
// search runs the atom is in the segment unless a list was cut at its capacity (which the list
// build has already reported): so a window that holds the whole segment and a single candidate
// gives the slot; otherwise each candidate's entry is compared, in order.
__device__ __forceinline__ int find_slot(const int32_t *__restrict__ row, const uint8_t *__restrict__ hrow, int lo,
                                         int hi, int ai) {
    const uint32_t hh = index_hash8(ai) * 0x01010101u;
    for (int b = lo & ~31; b < hi; b += 64) {
        uint32_t w[16];
        ld_v8u(hrow + b, w);
        if (b + 32 < hi) {
            ld_v8u(hrow + b + 32, w + 8);
        } else {
#pragma unroll
            for (int q = 8; q < 16; ++q) w[q] = ~hh;   // no byte matches
        }
        uint64_t m = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) m |= (uint64_t)zero_bytes4(w[q] ^ hh) << (4 * q);
        const int l0 = max(lo - b, 0), h0 = min(hi - b, 64);
        m &= (h0 >= 64 ? ~0ull : ((1ull << h0) - 1ull)) & ~((1ull << l0) - 1ull);
        if (hi <= b + 64 && __popcll(m) == 1) return b + __ffsll(m) - 1;
        while (m) {
            const int k = __ffsll(m) - 1;
            m &= m - 1;
            if (row[b + k] == ai) return b + k;
        }
    }
    return -1;
}

constexpr int REV_WARPS = 4;
struct RevSmem {
    int s[REV_WARPS][256];   // each warp's pairs: slot in the atom's list (the capacity is at most 256)
    int j[REV_WARPS][256];   //   and the neighbour's internal index
};

// Warp per atom i.  The entries j = nbr[i][s] with j > i are compacted (ballot) into the warp's
// pair list; each lane then takes one pair, reads j's segment bounds for the kind of slot s,
// finds the slot t of i in that segment of j's list row (through the row's hash bytes) and
// writes both reverse slots,
// rev[i][s] = t and rev[j][t] = s (the entries with j < i are written by j's warp): one search
// per unordered pair.  The lists are symmetric and so is each pair's segment kind (the cutoff
// test gives the same result for (i, j) and (j, i)), so i sits in the segment of j's list for
// (kind of slot s, species of i).  A pair found in one list only (a list cut at its capacity)
// raises the overflow status.
__device__ __forceinline__ void rev_body(const RevArgs &args, int64_t blk, int64_t nblk, RevSmem &sm) {
    const RevArgs a = args;   // as values: the stores below cannot make the compiler re-read them
    if (a.flag && *a.flag == 0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t i = blk * REV_WARPS + w; i < a.n; i += nblk * REV_WARPS) {
        const int4 sg = a.seg[i];
        const int ti = a.species[i];
        int cnt = 0;
        for (int s0 = 0; s0 < sg.w; s0 += 32) {
            const int s = s0 + lane;
            const int jj = s < sg.w ? a.nbr[i * a.capr + s] : -1;
            const bool act = jj > i;   // the lower-indexed atom of the pair searches
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (act) {
                sm.s[w][cnt + __popc(bal & lt)] = s;
                sm.j[w][cnt + __popc(bal & lt)] = jj;
            }
            cnt += __popc(bal);
        }
        __syncwarp();
        for (int p = lane; p < cnt; p += 32) {
            const int s = sm.s[w][p], j = sm.j[w][p];
            const int4 sj = a.seg[j];
            const int sgi = (s < sg.y ? 0 : 2) + ti;
            const int lo = sgi == 0 ? 0 : sgi == 1 ? sj.x : sgi == 2 ? sj.y : sj.z;
            const int hi = sgi == 0 ? sj.x : sgi == 1 ? sj.y : sgi == 2 ? sj.z : sj.w;
            const int t = find_slot(a.nbr + (int64_t)j * a.capr, a.hash + (int64_t)j * a.capr, lo, hi, (int)i);
            if (t < 0) {
                atomicOr(a.status, ST_NBR_OVERFLOW);
                a.rev[i * a.capr + s] = 0;
                continue;
            }
            a.rev[i * a.capr + s] = (uint8_t)t;
            a.rev[(int64_t)j * a.capr + t] = (uint8_t)s;
        }
        __syncwarp();   // the next atom reuses the pair list
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

// register budget of a system's own list build (its 29 KB of staging allow 7 blocks per SM)
constexpr int LISTS_MINB = 6;

template <bool LOOP>
__global__ void k_bin(const BinArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    rebuild_items<LOOP>(tab, m, [](const BinArgs &r, int64_t blk, int64_t nblk) { bin_body(r, blk, nblk); });
}
template <bool LOOP>
__global__ void k_scan(const BinArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    __shared__ int s_part[32];
    rebuild_items<LOOP>(tab, m, [&](const BinArgs &r, int64_t, int64_t) { scan_body(r, s_part); });
}
template <bool LOOP>
__global__ void k_scatter(const BinArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    rebuild_items<LOOP>(tab, m, [](const BinArgs &r, int64_t blk, int64_t nblk) { scatter_body(r, blk, nblk); });
}
template <bool LOOP>
__global__ void k_cellsort(const BinArgs *__restrict__ tab, WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    rebuild_items<LOOP>(tab, m, [](const BinArgs &r, int64_t blk, int64_t nblk) { cellsort_body(r, blk, nblk); });
}
template <bool LOOP>
__global__ void __launch_bounds__(LB_WARPS * 32, LOOP ? 4 : LISTS_MINB) k_lists(const ListArgs *__restrict__ tab,
                                                                              WorkMap m, const int *quick) {
    if (quick && *quick == 0) return;
    __shared__ ListSmem sm;
    rebuild_items<LOOP>(tab, m, [&](const ListArgs &a, int64_t blk, int64_t nblk) { lists_body(a, blk, nblk, sm); });
}
template <bool LOOP>
__global__ void __launch_bounds__(REV_WARPS * 32, LOOP ? 6 : 8) k_rev(const RevArgs *__restrict__ tab, WorkMap m,
                                                                     const int *quick) {
    if (quick && *quick == 0) return;
    __shared__ RevSmem sm;
    rebuild_items<LOOP>(tab, m, [&](const RevArgs &a, int64_t blk, int64_t nblk) { rev_body(a, blk, nblk, sm); });
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
        g.inv2w[a] = 2.0 / g.w[a];
        g.per[a] = s.per[a];
    }
    const int64_t n = s.n;
    BinArgs &r = pl.bin;
    r.pos = s.pos; r.species = s.species; r.orig = s.orig; r.n = n; r.g = g;
    r.ncell = s.cells.ncell; r.count = s.cells.count; r.start = s.cells.start; r.fill = s.cells.fill;
    r.atoms = s.cells.atoms; r.of = s.cells.of; r.cposf = s.cells.posf; r.ckey = s.cells.key;
    r.sub = s.cells.sub;
    r.posref = s.posref; r.builds = s.d_builds; r.rebuild = s.rebuild; r.flag = flag;
    ListArgs &la = pl.lists;
    la.pos = s.pos;
    la.cell_start = s.cells.start; la.cell_atoms = s.cells.atoms; la.cell_sub = s.cells.sub;
    la.cposf = s.cells.posf;
    la.cap = s.cap; la.cap_ang = s.cap_ang; la.capr = nbr_stride(s.cap);
    la.cut_r2 = s.cut_r2; la.cut_a2 = s.cut_a2;
    // Band of the FP32 pre-test.  Each FP32 separation component is (u_j + o) - u_i with
    // |u| <= 2w (positions relative to their cells' corners, rounded once from FP64) and o a
    // corner offset of at most one cell width (one rounding of w); every rounding is at most
    // 2^-24 of a value below 5w, and the FP32 minimum image (fewer than 3 cells along a
    // periodic axis) adds roundings below 2^-24 of 2L.  So each component is off by at most
    // E = 2^-24 (16 w + 4 L'), with w the largest cell width and L' the largest periodic box
    // length where the minimum image is taken (else 0), and d2 (at most R^2, R the list
    // cutoff plus a margin) by at most 2 sqrt(3) R E + 3 E^2 + 4 2^-24 R^2.  The band is twice
    // that; pairs inside it take the FP64 test.
    {
        const double u32 = std::ldexp(1.0, -24);
        double wmax = 0.0, lmin = 0.0;
        bool placed = true;
        for (int a = 0; a < 3; ++a) placed = placed && (!s.per[a] || s.cells.nc[a] >= 3);
        for (int a = 0; a < 3; ++a) {
            wmax = std::max(wmax, g.w[a]);
            if (!placed && s.per[a]) lmin = std::max(lmin, s.box[a]);
        }
        const double E = u32 * (16.0 * wmax + 4.0 * lmin);
        const double R = std::sqrt(std::max(s.cut_r2, s.cut_a2)) + 1.0;
        const double band = 2.0 * (2.0 * std::sqrt(3.0) * R * E + 3.0 * E * E + 4.0 * u32 * R * R);
        la.cut_r2f_lo = (float)(s.cut_r2 - band); la.cut_r2f_hi = (float)(s.cut_r2 + band);
        la.cut_a2f_lo = (float)(s.cut_a2 - band); la.cut_a2f_hi = (float)(s.cut_a2 + band);
        for (int a = 0; a < 3; ++a) la.wf[a] = (float)g.w[a];
    }
    la.bd = s.boxd; la.bf = s.boxf; la.g = g;
    la.nbr = s.nbr; la.hash = s.nbr_hash; la.seg = s.seg; la.status = s.status; la.flag = flag;
    RevArgs &ra = pl.rev;
    ra.species = s.species; ra.nbr = s.nbr; ra.hash = s.nbr_hash; ra.seg = s.seg;
    ra.n = n; ra.cap = s.cap; ra.capr = nbr_stride(s.cap);
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
    pl.blocks[RB_CELLSORT] = capped(s.cells.ncell, RB_THREADS / 32);   // a warp per cell
    pl.blocks[RB_LISTS] = capped(s.cells.ncell, 1);   // one cell per block and item
    pl.blocks[RB_REV] = capped(n, REV_WARPS);
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
    t.grid[FK_CELLSORT] = full((const void *)k_cellsort<true>, RB_THREADS);
    t.grid[FK_LISTS] = full((const void *)k_lists<true>, LB_WARPS * 32);
    t.grid[FK_REV] = full((const void *)k_rev<true>, REV_WARPS * 32);
    t.grid[FK_FINISH] = full((const void *)k_finish<true>, RB_THREADS);
}

template <bool LOOP>
static void rebuild_t(const FusedTables &t, const Launch *L, bool clear, cudaStream_t st) {
    const BinArgs *bin = t.at<BinArgs>(t.o_bin);
    k_bin<LOOP><<<L[RB_BIN].grid, RB_THREADS, 0, st>>>(bin, L[RB_BIN].m, L[RB_BIN].quick);
    k_scan<LOOP><<<L[RB_SCAN].grid, 1024, 0, st>>>(bin, L[RB_SCAN].m, L[RB_SCAN].quick);
    k_scatter<LOOP><<<L[RB_SCATTER].grid, RB_THREADS, 0, st>>>(bin, L[RB_SCATTER].m, L[RB_SCATTER].quick);
    k_cellsort<LOOP><<<L[RB_CELLSORT].grid, RB_THREADS, 0, st>>>(bin, L[RB_CELLSORT].m, L[RB_CELLSORT].quick);
    k_lists<LOOP><<<L[RB_LISTS].grid, LB_WARPS * 32, 0, st>>>(t.at<ListArgs>(t.o_lists), L[RB_LISTS].m,
                                                              L[RB_LISTS].quick);
    k_rev<LOOP><<<L[RB_REV].grid, REV_WARPS * 32, 0, st>>>(t.at<RevArgs>(t.o_rev), L[RB_REV].m, L[RB_REV].quick);
    k_finish<LOOP><<<L[RB_FINISH].grid, RB_THREADS, 0, st>>>(bin, L[RB_FINISH].m, L[RB_FINISH].quick);
    if (clear) k_clear_flags<<<1, 128, 0, st>>>(bin, L[RB_BIN].m);
}
void launch_rebuild_t(const FusedTables &t, const Launch *L, bool clear, bool loop, cudaStream_t st) {
    if (loop) rebuild_t<true>(t, L, clear, st);
    else rebuild_t<false>(t, L, clear, st);
}

}  // namespace sl
