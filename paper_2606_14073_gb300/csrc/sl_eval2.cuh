// sl_eval2.cuh -- argument block and pair record shared by the evaluation kernels and the gather.
#pragma once

#include "sl_common.cuh"

namespace sl {

template <typename R> struct V2s;
template <> struct V2s<float> { using t = float2; };
template <> struct V2s<double> { using t = double2; };
template <typename R> using v2 = typename V2s<R>::t;

// Record of one ordered pair (i -> j) for neighbour j: (dE_i/dr_ij, dE_i/dS_j), 32 bytes
// in FP32 (one DRAM sector), stored in j's own list slot of i.
template <typename R>
struct PairRec {
    v4<R> a;   // dE_i/dr_ij (x, y, z), dE_i/dS_j .x
    v4<R> b;   // dE_i/dS_j .y, .z, 0, 0
};

template <typename R>
struct Eval2Args {
    const v4<R> *pos, *spin;
    const int32_t *nbr;   // [n][capr] candidate list of atom i (internal indices), atom-major
    const uint8_t *rev;   // [n][capr] rev[i][s] = slot of i in the list of nbr[i][s]
    int capr;             // row stride of nbr and rev: cap rounded up to a multiple of 32
    const int4 *seg;
    int64_t n, n_fe;
    BoxDev<R> box;
    int cap, cap_ang;
    int32_t *clj;      // compact in-cutoff rows [cap_ang + cap][n]: neighbour index
    uint16_t *cls;     // ... its candidate slot s (low byte) and the reverse slot rev[s][i] (high byte)
    int4 *cnt;         // (angular rows of species 0, angular rows, radial-only rows of species 0, radial-only rows)
    uint32_t *mask;    // [maskw][n]: bit s of word s/32 set when candidate slot s is inside rc_rad
    int maskw;
    R *q, *bsum, *fp, *ei;
    int64_t qs;        // row stride of q ([DIM][qs])
    PairRec<R> *pd;    // [cap][n]
    v4<R> *fown, *gii;
    R *wpart;
    int want_virial;
    int *status;
    const int *skip;   // non-null and set: every evaluation kernel returns at once
};

}  // namespace sl
